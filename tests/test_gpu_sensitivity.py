"""GPU parity of the sensitivities S_i^2 and the truncation N-hat (Sec. 3.1) against
the FP64 oracle, through the C ABI (hmc_sensitivity, hmc_select_subset).

The oracle takes every data term's full reverse pass and squares it; the GPU forms
the same sums as GEMMs of squared activations with squared (or, for a DeepONet,
Gram-weighted) adjoints.  Tolerances: 1e-10 relative per parameter in FP64 (the
terms are non-negative, so there is no cancellation), 1e-4 in FP32.  The ranking
and the mask are integer results: on the same S2 input they must be identical.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "case1_table1.json")
NAMES = ["omega1", "omega2", "phi1", "phi2", "a", "b"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


def _mu_sd(P, seed):
    rng = np.random.default_rng(seed)
    return 0.4 * rng.standard_normal(P), rng.uniform(0.01, 0.3, P)


def _gpu_sens(prob, mu, sd, prec):
    if prob.kind == W.KIND_MLP:
        S2 = hmc.sensitivity_mlp(prob.net.widths, prob.x, mu, sd, prec=prec, act=prob.net.act, bias=prob.net.bias)
    else:
        S2 = hmc.sensitivity_deeponet(prob.branch.widths, prob.trunk.widths, prob.u, prob.yq, mu, sd, prec=prec,
                                      out_bias=prob.out_bias, branch_act=prob.branch.act, trunk_act=prob.trunk.act,
                                      branch_bias=prob.branch.bias, trunk_bias=prob.trunk.bias)
    return S2.cpu().numpy()


CASES = {
    # multi-output, mixed activations and biases, ragged tiles
    "mlp_ragged": lambda: W.small_mlp(n=300, widths=(3, 70, 33, 2), acts=[W.ACT_TANH, W.ACT_SIN, W.ACT_IDENTITY],
                                      bias=[True, False, True], seed=81),
    "mlp_wide": lambda: W.small_mlp(n=700, widths=(2, 128, 128, 1), seed=82),
    "deeponet": lambda: W.small_deeponet(n_u=37, n_y=29, seed=83),
    "deeponet_no_b0": lambda: W.small_deeponet(n_u=70, n_y=45, du=5, width=40, latent=20, seed=84, out_bias=False),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_sensitivity_parity(case, prec):
    prob = CASES[case]()
    mu, sd = _mu_sd(prob.P, 5)
    S2r = oracle.Oracle(prob).sensitivity(mu, sd)
    S2 = _gpu_sens(prob, mu, sd, prec)
    tol = 1e-10 if prec == hmc.PREC_FP64 else 1e-4
    rel = np.abs(S2 - S2r) / np.maximum(np.abs(S2r), 1e-300)
    assert np.all(np.abs(S2 - S2r) <= tol * np.abs(S2r) + 1e-30), (rel.max(), int(rel.argmax()))


def test_sensitivity_full_size_wide_mlp():
    # MLP 2-256-256-256-256-1 on 8192 points, FP32, against the term-by-term oracle
    prob = W.wide_mlp()
    mu, sd = prob.frozen.copy(), np.full(prob.P, 0.05)
    S2 = _gpu_sens(prob, mu, sd, hmc.PREC_FP32)
    S2r = oracle.Oracle(prob).sensitivity(mu, sd)
    rel = np.abs(S2 - S2r) / np.maximum(S2r, 1e-300)
    assert np.all(np.abs(S2 - S2r) <= 1e-4 * S2r + 1e-30), (rel.max(), int(rel.argmax()))


def _clear_of_cut(S2, tau, band=1e-9):
    """tau is not within rounding of any prefix share (the FP64 sums run in different orders)."""
    order = sorted(range(len(S2)), key=lambda i: (-S2[i], i))
    c = np.cumsum(S2[order]) / S2.sum()
    return np.all(np.abs(c - tau) > band)


@pytest.mark.parametrize("P,ties", [(1, False), (7, True), (300, False), (5000, True), (70001, True)])
def test_select_subset_is_exact(P, ties):
    rng = np.random.default_rng(P)
    S2 = rng.exponential(1.0, P) ** 2
    if ties:
        S2[rng.integers(0, P, max(1, P // 4))] = S2[0]
        S2[rng.integers(0, P, max(1, P // 10))] = 0.0
    for tau in (0.0, 0.05, 0.3, 0.5, 0.9, 0.999, 1.0):
        if not _clear_of_cut(S2, tau):
            continue
        n, mask, order = hmc.select_subset(torch.from_numpy(S2), tau)
        nr, maskr, orderr = oracle.truncate(S2, tau)
        assert n == nr, (P, tau, n, nr)
        assert np.array_equal(mask.cpu().numpy(), maskr)
        assert np.array_equal(order.cpu().numpy(), orderr)


def test_select_subset_edges():
    n, mask, _ = hmc.select_subset(torch.zeros(9, dtype=torch.float64), 0.9)
    assert n == 0 and int(mask.sum()) == 0
    with pytest.raises(hmc.HmcError):
        hmc.select_subset(torch.tensor([1.0, -1.0], dtype=torch.float64), 0.5)
    with pytest.raises(hmc.HmcError):
        hmc.select_subset(torch.tensor([1.0, float("nan")], dtype=torch.float64), 0.5)


def test_case1_pipeline_on_the_gpu():
    # Sec. 4.1.1 end to end through the C ABI: sensitivities at the Table 1 VI values,
    # the tau = 0.9 subset, then FP64 HMC on it with App. C's step and L; the samples
    # reproduce Table 1's VI-HMC row (tolerances as in the oracle's Case I test)
    g = json.load(open(GOLD))
    mu = np.array([g["vi"]["mean"][n] for n in NAMES])
    sd = np.array([g["vi"]["std"][n] for n in NAMES])
    base = W.case1_sine(mu)
    S2 = hmc.sensitivity_mlp([1, 2, 1], base.x, base.frozen, sd, prec=hmc.PREC_FP64,
                             act=[W.ACT_SIN, W.ACT_IDENTITY], bias=[True, False])
    n, mask, _ = hmc.select_subset(S2, g["vi_hmc_subset"]["tau"])
    mask = mask.cpu().numpy()
    assert n == 4
    assert sorted(NAMES[i] for i in np.flatnonzero(mask)) == sorted(g["vi_hmc_subset"]["sampled"])
    h = g["hyper"]
    L = int(round(np.pi * h["posterior_variance"] / (2 * h["step_size_hmc"])))
    prob = W.case1_sine(mu, mask=mask, chains=16, eps=h["step_size_hmc"], L=L)
    s = hmc.Sampler.mlp([1, 2, 1], prob.x, prob.y, prob.mask, prob.frozen, 16, prior_sigma=1.0,
                        noise_sigma=prob.noise_sigma, prec=hmc.PREC_FP64, act=[W.ACT_SIN, W.ACT_IDENTITY],
                        bias=[True, False])
    S, acc, _, _ = s.sample(torch.from_numpy(prob.q0), prob.eps, L, 160, seed=77)
    assert acc.float().mean().item() > 0.8
    X = S.cpu().numpy()[40:].reshape(-1, 4)
    names = [NAMES[i] for i in np.flatnonzero(mask)]
    for j, nm in enumerate(names):
        m, sdv = g["vi_hmc"]["mean"][nm], g["vi_hmc"]["std"][nm]
        assert abs(X[:, j].mean() - m) <= 3 * np.sqrt(2.0) * sdv + 0.005, (nm, X[:, j].mean(), m)
        assert abs(X[:, j].std() / sdv - 1) <= 0.15, (nm, X[:, j].std(), sdv)
