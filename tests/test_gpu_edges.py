"""GPU edge cases of the energy, the gradient and the sampler, through the C ABI.

* No data terms (zero training points, or a DeepONet without input functions): the
  potential is the prior alone, U = |q|^2 / (2 alpha^2), in every precision; the
  leapfrog is then the harmonic oscillator, whose L-step map is the L-th power of the
  one-step kick-drift-kick matrix (a closed form, not the oracle); the sampler draws
  the N(0, alpha^2) prior, checked on its moments.
* Subsets confined to one part of the network: the output layer only (the adjoint stops
  at once), the first layer only (it runs through every layer), the biases only.
* Data sizes at and below the 128-row tile: N = 1, 127, 128, 129, 255, 257, one chain.
Tolerances as for the other parity tests: FP64 1e-10, FP32 1e-5, BF16 2e-2, FP16 5e-3.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, grad_ok_bf16, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu

PRECS = [hmc.PREC_FP64, hmc.PREC_FP32, hmc.PREC_BF16, hmc.PREC_FP16]
TOL16 = {hmc.PREC_BF16: 2e-2, hmc.PREC_FP16: 5e-3}


def _f32(a):
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def _with_mask(prob, mask, chains=None, seed=0, jitter=0.05):
    """The same network and data with another subset (and fresh chain states)."""
    mask = np.asarray(mask, dtype=np.uint8)
    C = prob.chains if chains is None else chains
    rng = np.random.default_rng(seed)
    base = prob.frozen[mask.astype(bool)]
    q0 = _f32(base[None, :] + jitter * rng.standard_normal((C, base.size)))
    return dataclasses.replace(prob, mask=mask, q0=q0)


def _layer_mask(prob, which):
    m = np.zeros(prob.P, dtype=np.uint8)
    sl = prob.net.layer_slices()
    widths = prob.net.widths
    for l, (woff, boff) in enumerate(sl):
        nw = widths[l] * widths[l + 1]
        if which == "output" and l == len(sl) - 1 or which == "first" and l == 0:
            m[woff:woff + nw] = 1
            if boff >= 0:
                m[boff:boff + widths[l + 1]] = 1
        if which == "bias" and boff >= 0:
            m[boff:boff + widths[l + 1]] = 1
    return m


def _check(prob, prec, q=None):
    o = oracle.Oracle(prob)
    s = sampler_from(prob, prec)
    q = prob.q0 if q is None else q
    U, g = s.energy_grad(torch.from_numpy(q))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    Ur, gr = o.energy_grad_batch(q)
    for c in range(prob.chains):
        if prec in TOL16:
            assert abs(U[c] - Ur[c]) <= TOL16[prec] * abs(Ur[c]), (c, U[c], Ur[c])
            ok, re, rinf = grad_ok_bf16(g[c], gr[c], TOL16[prec])
        else:
            tol = 1e-10 if prec == hmc.PREC_FP64 else 1e-5
            assert abs(U[c] - Ur[c]) <= tol * abs(Ur[c]), (c, U[c], Ur[c])
            ok, re, rinf = grad_ok(g[c], gr[c], tol)
        assert ok, (c, re, rinf)


# ---- no data terms --------------------------------------------------------------------

def _no_data_mlp(prior=0.7, chains=3):
    # a deep MLP with every hidden layer, but no training points
    prob = W.small_mlp(n=1, widths=(2, 256, 256, 1), frac=0.05, chains=chains, prior=prior, seed=41)
    return dataclasses.replace(prob, x=np.zeros((0, 2)), y=np.zeros((0, 1)))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["harmonic", "mlp", "deeponet"])
def test_no_data_energy_is_the_prior(which, prec):
    if which == "harmonic":
        prob = W.harmonic(k=50, prior=0.7, chains=3)
    elif which == "mlp":
        prob = _no_data_mlp()
    else:
        prob = W.small_deeponet(frac=0.2, chains=3)
        prob = dataclasses.replace(prob, u=np.zeros((0, prob.u.shape[1])), t=np.zeros((0, prob.t.shape[1])))
    s = sampler_from(prob, prec)
    U, g = s.energy_grad(torch.from_numpy(prob.q0))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    a2 = prob.prior_sigma ** 2
    for c in range(prob.chains):
        q = prob.q0[c]
        # the closed form: U up to the FP64 summation order, g up to its final rounding
        assert abs(U[c] - 0.5 * q @ q / a2) <= 1e-12 * (0.5 * q @ q / a2), (c, U[c])
        rtol = 1e-15 if prec == hmc.PREC_FP64 else 2 ** -23
        assert np.all(np.abs(g[c] - q / a2) <= rtol * np.abs(q / a2) + 1e-300), c


@pytest.mark.parametrize("prec", PRECS)
def test_no_data_leapfrog_is_the_harmonic_oscillator(prec):
    alpha, eps, L = 0.7, 0.1, 13
    prob = W.harmonic(k=64, prior=alpha, chains=2, eps=eps, L=L)
    s = sampler_from(prob, prec)
    rng = np.random.default_rng(1)
    q = _f32(rng.standard_normal(prob.q0.shape))
    p = _f32(rng.standard_normal(prob.q0.shape))
    q1, p1 = s.leapfrog(torch.from_numpy(q), torch.from_numpy(p), eps, L)
    q1, p1 = q1.cpu().double().numpy(), p1.cpu().double().numpy()
    w2 = 1.0 / alpha ** 2
    M = np.array([[1 - eps ** 2 * w2 / 2, eps], [-eps * w2 * (1 - eps ** 2 * w2 / 4), 1 - eps ** 2 * w2 / 2]])
    ML = np.linalg.matrix_power(M, L)
    qe, pe = ML[0, 0] * q + ML[0, 1] * p, ML[1, 0] * q + ML[1, 1] * p
    tol = 1e-12 if prec == hmc.PREC_FP64 else 1e-5
    assert np.max(np.abs(q1 - qe)) <= tol * np.max(np.abs(qe)), np.max(np.abs(q1 - qe))
    assert np.max(np.abs(p1 - pe)) <= tol * np.max(np.abs(pe)), np.max(np.abs(p1 - pe))


@pytest.mark.parametrize("prec", PRECS)
def test_no_data_sampler_draws_the_prior(prec):
    # eps L ~ 0.46 pi alpha: nearly independent draws of N(0, alpha^2) per coordinate
    alpha, n = 0.7, 300
    prob = W.harmonic(k=40, prior=alpha, chains=2)
    s = sampler_from(prob, prec)
    S, acc, dH, _ = s.sample(torch.from_numpy(prob.q0), 0.1 * alpha, 14, n, seed=3)
    S = S.cpu().double().numpy()[50:]          # 250 kept draws x 2 chains x 40 coordinates
    assert acc.float().mean().item() > 0.95
    draws = S.reshape(-1)
    m, v = draws.mean(), draws.var()
    # 20,000 draws, mildly autocorrelated: 6-sigma bands with a factor 3 for the correlation
    assert abs(m) <= 6 * 3 * alpha / np.sqrt(draws.size), m
    assert abs(v / alpha ** 2 - 1) <= 6 * 3 * np.sqrt(2.0 / draws.size), v


def test_no_data_is_rejected_by_split_handles():
    prob = _no_data_mlp(chains=1)
    with pytest.raises(hmc.HmcError, match="n_splits"):
        sampler_from(prob, hmc.PREC_FP32, n_splits=2)


# ---- subsets confined to one part of the network ------------------------------------

@pytest.mark.parametrize("which", ["output", "first", "bias"])
@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_subset_in_one_part_cuda_cores(which, prec):
    prob = W.small_mlp(n=300, widths=(3, 40, 33, 2), chains=2, seed=42)
    _check(_with_mask(prob, _layer_mask(prob, which)), prec)


@pytest.mark.parametrize("prec", [hmc.PREC_BF16, hmc.PREC_FP16])
@pytest.mark.parametrize("which", ["output", "first", "bias"])
@pytest.mark.parametrize("widths", [(2, 256, 256, 256, 1), (2, 128, 128, 1)])
def test_subset_in_one_part_tensor_cores(which, widths, prec):
    prob = W.small_mlp(n=300, widths=widths, frac=0.05, chains=2, seed=43)
    _check(_with_mask(prob, _layer_mask(prob, which), jitter=0.02), prec)


# ---- row counts around the 128-row tile ---------------------------------------------

@pytest.mark.parametrize("n", [1, 127, 128, 129, 255, 257])
@pytest.mark.parametrize("prec,widths", [(hmc.PREC_FP32, (2, 48, 40, 1)), (hmc.PREC_BF16, (2, 256, 256, 256, 1)),
                                         (hmc.PREC_BF16, (2, 128, 128, 1)), (hmc.PREC_FP16, (2, 256, 256, 256, 1))])
def test_row_counts_around_a_tile(n, prec, widths):
    prob = W.small_mlp(n=n, widths=widths, frac=0.1, chains=1, seed=44)
    _check(prob, prec)


# ---- training data passed as float32 ----------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("which", ["mlp", "deeponet"])
def test_float32_training_data_is_the_float64_data(which, prec):
    # the workloads' data are float32-representable: both element types give the same problem
    if which == "mlp":
        prob = W.small_mlp(n=300, widths=(2, 128, 128, 1), frac=0.1, chains=2, seed=45)
        arrays = {"x": prob.x, "y": prob.y}
    else:
        prob = W.small_deeponet(chains=2)
        arrays = {"u": prob.u, "yq": prob.yq, "t": prob.t}
    if prec in TOL16 and which == "deeponet":
        prob = W.small_deeponet(n_u=40, n_y=130, du=8, width=64, latent=64, frac=0.1, chains=2, seed=46)
        arrays = {"u": prob.u, "yq": prob.yq, "t": prob.t}
    q = torch.from_numpy(prob.q0)
    U64, g64 = sampler_from(prob, prec).energy_grad(q)
    f32 = dataclasses.replace(prob, **{k: v.astype(np.float32) for k, v in arrays.items()})
    s32 = sampler_from(f32, prec)
    U32, g32 = s32.energy_grad(q)
    assert torch.equal(U32, U64) and torch.equal(g32, g64)
    # device tensors take the same route
    dev = dataclasses.replace(prob, **{k: torch.from_numpy(v.astype(np.float32)).cuda() for k, v in arrays.items()})
    Ud, gd = sampler_from(dev, prec).energy_grad(q)
    assert torch.equal(Ud, U64) and torch.equal(gd, g64)


# ---- a bounded device-side wait that runs out ------------------------------------------

def test_a_wait_that_runs_out_is_reported_and_the_handle_stays_usable():
    prob = W.small_mlp(n=300, widths=(2, 128, 128, 1), frac=0.1, chains=2, seed=47)
    s = sampler_from(prob, hmc.PREC_BF16)
    q = torch.from_numpy(prob.q0)
    U0, g0 = s.energy_grad(q)
    s.check()                                   # no wait gave up
    L = hmc.lib()
    # a 1 ms wait on a barrier that nothing arrives at: recorded, no fault, no hang
    assert L.hmc_diag_expire_wait(s._h, 1_000_000) == 0
    with pytest.raises(hmc.HmcError, match="HMC_ERR_TIMEOUT"):
        s.check()
    s.check()                                   # the record was cleared
    U1, g1 = s.energy_grad(q)                   # and the context still works
    assert torch.equal(U1, U0) and torch.equal(g1, g0)
    s.check()
    # the CUDA-core engines have no such waits and keep no flag
    s32 = sampler_from(prob, hmc.PREC_FP32)
    assert L.hmc_diag_expire_wait(s32._h, 1_000_000) == 6
    s32.check()
