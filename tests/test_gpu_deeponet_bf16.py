"""GPU parity of the DeepONet on the tensor cores (BF16 GEMMs, FP32 accumulate, FP64
energy) against the FP64 oracle, through the C ABI.

The operator output S = B T^T + b0 (Sec. 4.2) is formed on 128 x N tiles; dB and dT
are GEMMs over the bf16 residual dS; branch and trunk run the MLP kernels.  The
tolerance is the BF16 one of the MLP path: per gradient evaluation, relative 2-norm
and infinity-norm errors within 2e-2, and U within 2e-2 relative.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok_bf16, rel_err, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


def _check(prob, chains=None, tol=2e-2):
    s = sampler_from(prob, hmc.PREC_BF16)
    q = prob.q0
    U, g = s.energy_grad(torch.from_numpy(q))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(g))
    o = oracle.Oracle(prob)
    for c in (range(prob.chains) if chains is None else chains):
        Ur, gr = o.energy_grad(q[c])
        assert abs(U[c] - Ur) <= tol * abs(Ur), (c, U[c], Ur)
        ok, r2, rinf = grad_ok_bf16(g[c], gr, tol)
        assert ok, (c, r2, rinf)
    return s, U, g


@pytest.mark.parametrize("case", ["gemm_first_ragged", "cuda_core_first_no_b0", "wide_latent"])
def test_deeponet_bf16_parity_small(case):
    prob = {
        # branch input width 12 (> 8): the first layer is a GEMM on bf16 inputs; ragged tiles
        "gemm_first_ragged": lambda: W.small_deeponet(n_u=150, n_y=90, du=12, width=64, latent=64, frac=0.3,
                                                      chains=3, seed=41),
        # both first layers on CUDA cores, no output bias, a single-hidden-layer trunk
        "cuda_core_first_no_b0": lambda: W.small_deeponet(n_u=300, n_y=200, du=5, width=128, latent=64, frac=0.2,
                                                          chains=2, seed=42, out_bias=False),
        "wide_latent": lambda: W.small_deeponet(n_u=130, n_y=260, du=3, width=256, latent=128, frac=0.1,
                                                chains=2, seed=43),
    }[case]()
    _check(prob)


def test_deeponet_grf_full_size_bf16():
    # branch 100-128-128-128-64, trunk 2-128-128-128-64, 500 x 100, 32 chains
    prob = W.deeponet_grf()
    _check(prob, chains=(0, 17, 31))


def test_cone_deeponet_bf16_full_grid():
    # branch 6-256-256-256-128, trunk 2-256-256-256-128 on the full 64 x 128 grid, 16 conditions
    prob = W.cone_deeponet(n_u=16, chains=2)
    _check(prob)


def test_deeponet_bf16_deterministic_and_close_to_fp32():
    prob = W.small_deeponet(n_u=200, n_y=120, du=7, width=128, latent=64, frac=0.25, chains=3, seed=44)
    s16 = sampler_from(prob, hmc.PREC_BF16)
    s32 = sampler_from(prob, hmc.PREC_FP32)
    q = torch.from_numpy(prob.q0)
    U1, g1 = s16.energy_grad(q)
    U2, g2 = s16.energy_grad(q)
    assert torch.equal(U1, U2) and torch.equal(g1, g2)
    U3, g3 = s32.energy_grad(q)
    for c in range(prob.chains):
        ok, r2, rinf = grad_ok_bf16(g1[c].cpu().numpy(), g3[c].cpu().numpy())
        assert ok, (c, r2, rinf)


def test_deeponet_bf16_trajectory_parity():
    # a shared (q, p) integrated for L steps: positions and momenta follow the oracle's
    prob = W.small_deeponet(n_u=160, n_y=96, du=10, width=128, latent=64, frac=0.2, chains=2, seed=46)
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_BF16)
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal(prob.q0.shape).astype(np.float32).astype(np.float64)
    eps, L = 2e-5, 10
    q1, p1 = s.leapfrog(torch.from_numpy(prob.q0), torch.from_numpy(p0), eps, L)
    q1, p1 = q1.cpu().double().numpy(), p1.cpu().double().numpy()
    for c in range(prob.chains):
        qr, pr, Ur, gr = o.leapfrog(prob.q0[c], p0[c], eps, L)
        assert rel_err(q1[c] - prob.q0[c], qr - prob.q0[c]) < 2e-2, c
        assert rel_err(p1[c] - p0[c], pr - p0[c]) < 2e-2, c


def test_deeponet_bf16_sampler_runs_and_resumes():
    prob = W.small_deeponet(n_u=120, n_y=64, du=4, width=64, latent=64, frac=0.3, chains=2, seed=45)
    s = sampler_from(prob, hmc.PREC_BF16)
    q0 = torch.from_numpy(prob.q0)
    S, acc, dH, ql = s.sample(q0, 2e-5, 5, 4, seed=3)
    assert np.all(np.isfinite(dH.cpu().numpy()))
    # the same trajectories in two calls: identical
    S1, acc1, dH1, q1 = s.sample(q0, 2e-5, 5, 2, seed=3)
    S2, acc2, dH2, q2 = s.sample(q1, 2e-5, 5, 2, seed=3, first_traj=2)
    assert torch.equal(torch.cat([S1, S2]), S) and torch.equal(torch.cat([dH1, dH2]), dH)
    assert torch.equal(q2, ql)


def test_deeponet_bf16_metropolis_energy_is_accurate():
    # hi/lo-activation forward of branch and trunk and S^T from hi/lo outputs
    prob = W.small_deeponet(n_u=150, n_y=90, du=12, width=64, latent=64, frac=0.3, chains=3, seed=41)
    s = sampler_from(prob, hmc.PREC_BF16)
    o = oracle.Oracle(prob)
    Um = s.metropolis_energy(torch.from_numpy(prob.q0)).cpu().numpy()
    Ur, _ = o.energy_grad_batch(prob.q0)
    assert np.all(np.abs(Um - Ur) <= 1e-4 * np.abs(Ur)), (Um, Ur)
    eps, L = 2e-5, 6
    _, _, dH, _ = s.sample(torch.from_numpy(prob.q0), eps, L, 1, seed=7)
    _, _, dHr, _ = o.sample(prob.q0, eps, L, 1, seed=7)
    dH = dH.cpu().numpy()
    assert np.all(np.abs(dH - dHr) <= 0.05 + 0.05 * np.abs(dHr)), (dH, dHr)
