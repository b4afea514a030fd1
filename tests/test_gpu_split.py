"""GPU parity of the symmetric split integrator (hmc_create_split) against the FP64
oracle's split integrator, through the C ABI.

The GPU fuses every kick with the drift after it and the last kick of a step with
the first of the next; the oracle applies the sweeps one sub-step at a time.  The
tolerances are those of the unsplit tests: 1e-10 (FP64), FP32 rounding (1e-5 on
the energy and gradient, 1e-4 on a trajectory's displacement), 2e-2 for BF16 and
5e-3 for FP16.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, grad_ok_bf16, rel_err, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


def _problem(which):
    return {
        "mlp": lambda: W.small_mlp(n=301, chains=3),
        "deeponet": lambda: W.small_deeponet(n_u=41, n_y=23, chains=2),
        "wide_mlp": lambda: W.small_mlp(n=700, widths=(2, 128, 128, 1), frac=0.2, chains=2, seed=7101),
        "wide_deeponet": lambda: W.small_deeponet(n_u=150, n_y=90, du=12, width=64, latent=64, frac=0.3,
                                                  chains=2, seed=41),
    }[which]()


@pytest.mark.parametrize("which", ["mlp", "deeponet"])
@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_split_handle_energy_grad_is_the_full_one(which, prec):
    prob = _problem(which)
    s = sampler_from(prob, prec, n_splits=4)
    U, g = s.energy_grad(torch.from_numpy(prob.q0))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    tol = 1e-10 if prec == hmc.PREC_FP64 else 1e-5
    Ur, gr = oracle.Oracle(prob).energy_grad_batch(prob.q0)
    for c in range(prob.chains):
        assert abs(U[c] - Ur[c]) <= tol * abs(Ur[c]), (c, U[c], Ur[c])
        ok, re, comp = grad_ok(g[c], gr[c], tol)
        assert ok, (c, re, comp)


@pytest.mark.parametrize("which", ["mlp", "deeponet"])
@pytest.mark.parametrize("M", [2, 5])
def test_split_leapfrog_parity_fp64(which, M):
    prob = _problem(which)
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_FP64, n_splits=M)
    rng = np.random.default_rng(11)
    p0 = rng.standard_normal(prob.q0.shape)
    eps, L = 4e-4, 7
    q1, p1 = s.leapfrog(torch.from_numpy(prob.q0), torch.from_numpy(p0), eps, L)
    q1, p1 = q1.cpu().numpy(), p1.cpu().numpy()
    for c in range(prob.chains):
        qr, pr = o.split_leapfrog(prob.q0[c], p0[c], eps, L, M)
        assert np.max(np.abs(q1[c] - qr)) <= 1e-10 * max(1.0, np.max(np.abs(qr))), c
        assert np.max(np.abs(p1[c] - pr)) <= 1e-9 * max(1.0, np.max(np.abs(pr))), c
        # and the split flow is not the leapfrog flow
        ql, _, _, _ = o.leapfrog(prob.q0[c], p0[c], eps, L)
        assert np.max(np.abs(ql - qr)) > 1e3 * np.max(np.abs(q1[c] - qr)) + 1e-14


# FP32 positions carry an absolute rounding of about ulp(|q|) per drift, so the FP32
# cases take a step whose displacement is large against it
@pytest.mark.parametrize("which,prec,tol,eps", [("mlp", hmc.PREC_FP32, 1e-4, 3e-4),
                                                ("deeponet", hmc.PREC_FP32, 1e-4, 3e-4),
                                                ("wide_mlp", hmc.PREC_BF16, 2e-2, 2e-5),
                                                ("wide_deeponet", hmc.PREC_BF16, 2e-2, 2e-5),
                                                ("wide_mlp", hmc.PREC_FP16, 5e-3, 2e-5),
                                                ("wide_deeponet", hmc.PREC_FP16, 5e-3, 2e-5)])
def test_split_leapfrog_parity_reduced_precision(which, prec, tol, eps):
    prob = _problem(which)
    o = oracle.Oracle(prob)
    s = sampler_from(prob, prec, n_splits=3)
    rng = np.random.default_rng(12)
    q0 = prob.q0.astype(np.float32).astype(np.float64)
    p0 = rng.standard_normal(prob.q0.shape).astype(np.float32).astype(np.float64)
    L = 6
    q1, p1 = s.leapfrog(torch.from_numpy(q0), torch.from_numpy(p0), eps, L)
    q1, p1 = q1.cpu().double().numpy(), p1.cpu().double().numpy()
    for c in range(prob.chains):
        qr, pr = o.split_leapfrog(q0[c], p0[c], eps, L, 3)
        assert rel_err(q1[c] - q0[c], qr - q0[c]) < tol, c
        assert rel_err(p1[c] - p0[c], pr - p0[c]) < tol, c


@pytest.mark.parametrize("which", ["mlp", "deeponet"])
def test_split_sample_parity_fp64(which):
    prob = _problem(which)
    o = oracle.Oracle(prob)
    M, n, eps, L, seed = 3, 4, 3e-4, 5, 17
    s = sampler_from(prob, hmc.PREC_FP64, n_splits=M)
    S, acc, dH, ql = s.sample(torch.from_numpy(prob.q0), eps, L, n, seed=seed, first_traj=3)
    S, acc, dH = S.cpu().numpy(), acc.cpu().numpy(), dH.cpu().numpy()
    Sr, accr, dHr, qlr = o.split_sample(prob.q0, eps, L, n, M, seed=seed, first_traj=3)
    lu = np.array([[oracle.log(oracle.mh_uniform(seed, c, 3 + t)) for c in range(prob.chains)] for t in range(n)])
    clear = np.abs(lu + dHr) > 1e-8 * (1 + np.abs(dHr))
    assert np.array_equal(acc[clear], accr[clear])
    assert np.allclose(dH, dHr, rtol=1e-6, atol=1e-7)
    assert np.max(np.abs(S - Sr)) <= 1e-9 * max(1.0, np.max(np.abs(Sr)))


@pytest.mark.parametrize("prec", [hmc.PREC_BF16, hmc.PREC_FP16])
@pytest.mark.parametrize("which", ["wide_mlp", "wide_deeponet"])
def test_split_16bit_sampler_energy_and_resume(which, prec):
    prob = _problem(which)
    M, eps, L = 3, 2e-5, 4
    s = sampler_from(prob, prec, n_splits=M)
    q0 = torch.from_numpy(prob.q0)
    # the Metropolis energy of a split handle is the sum of its batches' accurate energies
    Um = s.metropolis_energy(q0).cpu().numpy()
    Ur, _ = oracle.Oracle(prob).energy_grad_batch(prob.q0)
    assert np.all(np.abs(Um - Ur) <= 1e-4 * np.abs(Ur)), (Um, Ur)
    S, acc, dH, ql = s.sample(q0, eps, L, 4, seed=3)
    assert np.all(np.isfinite(dH.cpu().numpy()))
    S1, _, dH1, q1 = s.sample(q0, eps, L, 2, seed=3)
    S2, _, dH2, q2 = s.sample(q1, eps, L, 2, seed=3, first_traj=2)
    assert torch.equal(torch.cat([S1, S2]), S) and torch.equal(torch.cat([dH1, dH2]), dH)
    if which != "wide_mlp":
        return   # far from its mode this DeepONet's |dH| is ~1e4 per step: no dH check there
    # dH inherits the Metropolis energy's error at both ends (each within about 5e-6 of
    # U for the hi/lo forward; the unsplit BF16 path shows the same) and the BF16
    # force error integrated along the path (a few percent of dH)
    _, _, dHr, _ = oracle.Oracle(prob).split_sample(prob.q0, eps, L, 1, M, seed=7)
    _, _, dHg, _ = s.sample(q0, eps, L, 1, seed=7)
    bound = 0.05 + 0.05 * np.abs(dHr) + 1e-5 * np.abs(Ur)
    assert np.all(np.abs(dHg.cpu().numpy() - dHr) <= bound), (dHg, dHr, bound)


def test_split_rejects_more_batches_than_rows():
    prob = W.small_mlp(n=5, chains=1)
    with pytest.raises(hmc.HmcError):
        sampler_from(prob, hmc.PREC_FP32, n_splits=6)
    with pytest.raises(hmc.HmcError):
        sampler_from(prob, hmc.PREC_FP32, n_splits=65)
