"""GPU parity of the DeepONet on the tensor cores at FP16 (FP16 GEMMs, FP32 accumulate,
FP64 energy) against the FP64 oracle, through the C ABI.

FP16 keeps 11 significant bits but tops out at 65504.  The output-layer deltas
dB = dS T and dT = dS^T B (the gradient of the data term of Sec. 4.2 with respect to
the two nets' outputs) are sums over all query points and all input functions, so at
a state far from the data they exceed that range unless they are scaled down; the
cases below include such states.  Tolerance: per gradient evaluation, relative 2-norm
and infinity-norm errors within 5e-3, and U within 5e-3 relative.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok_bf16, rel_err, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu

TOL = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


def _check(prob, chains=None, tol=TOL):
    s = sampler_from(prob, hmc.PREC_FP16)
    q = prob.q0
    U, g = s.energy_grad(torch.from_numpy(q))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(g))
    o = oracle.Oracle(prob)
    errs = []
    for c in (range(prob.chains) if chains is None else chains):
        Ur, gr = o.energy_grad(q[c])
        assert abs(U[c] - Ur) <= tol * abs(Ur), (c, U[c], Ur)
        ok, r2, rinf = grad_ok_bf16(g[c], gr, tol)
        assert ok, (c, r2, rinf)
        errs.append(r2)
    return s, U, g, errs


@pytest.mark.parametrize("case", ["gemm_first_ragged", "cuda_core_first_no_b0", "wide_latent", "wide_unfitted"])
def test_deeponet_fp16_parity_small(case):
    prob = {
        "gemm_first_ragged": lambda: W.small_deeponet(n_u=150, n_y=90, du=12, width=64, latent=64, frac=0.3,
                                                      chains=3, seed=41),
        "cuda_core_first_no_b0": lambda: W.small_deeponet(n_u=300, n_y=200, du=5, width=128, latent=64, frac=0.2,
                                                          chains=2, seed=42, out_bias=False),
        "wide_latent": lambda: W.small_deeponet(n_u=130, n_y=260, du=3, width=256, latent=128, frac=0.1,
                                                chains=2, seed=43),
        # frozen weights N(0, 0.3^2) at width 256: |S| reaches 150 against targets of order
        # one, so the unscaled dB = dS T would reach about 6e5
        "wide_unfitted": lambda: W.small_deeponet(n_u=300, n_y=260, du=3, dy=2, width=256, latent=128, frac=0.1,
                                                  chains=2, seed=77),
    }[case]()
    _check(prob)


def test_deeponet_grf_full_size_fp16():
    # branch 100-128-128-128-64, trunk 2-128-128-128-64, 500 x 100, 32 chains
    prob = W.deeponet_grf()
    _check(prob, chains=(0, 17, 31))


def test_cone_deeponet_fp16_full_grid():
    # branch 6-256-256-256-128, trunk 2-256-256-256-128 on the full 64 x 128 grid: dB adds
    # 8192 products per entry, dT 16
    prob = W.cone_deeponet(n_u=16, chains=2)
    _check(prob)


def test_deeponet_fp16_is_more_accurate_than_bf16():
    prob = W.small_deeponet(n_u=200, n_y=120, du=7, width=128, latent=64, frac=0.25, chains=3, seed=44)
    o = oracle.Oracle(prob)
    q = torch.from_numpy(prob.q0)
    err = {}
    for name, prec in (("fp16", hmc.PREC_FP16), ("bf16", hmc.PREC_BF16)):
        s = sampler_from(prob, prec)
        U, g = s.energy_grad(q)
        g = g.cpu().double().numpy()
        err[name] = max(grad_ok_bf16(g[c], o.energy_grad(prob.q0[c])[1], 1.0)[1] for c in range(prob.chains))
    assert err["fp16"] < 0.5 * err["bf16"], err


def test_deeponet_fp16_deterministic():
    prob = W.small_deeponet(n_u=300, n_y=260, du=3, dy=2, width=256, latent=128, frac=0.1, chains=2, seed=77)
    s = sampler_from(prob, hmc.PREC_FP16)
    q = torch.from_numpy(prob.q0)
    U1, g1 = s.energy_grad(q)
    U2, g2 = s.energy_grad(q)
    assert torch.equal(U1, U2) and torch.equal(g1, g2)


def test_deeponet_fp16_trajectory_parity():
    # a shared (q, p) integrated for L steps: positions and momenta follow the oracle's
    prob = W.small_deeponet(n_u=160, n_y=96, du=10, width=128, latent=64, frac=0.2, chains=2, seed=46)
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_FP16)
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal(prob.q0.shape).astype(np.float32).astype(np.float64)
    eps, L = 2e-5, 10
    q1, p1 = s.leapfrog(torch.from_numpy(prob.q0), torch.from_numpy(p0), eps, L)
    q1, p1 = q1.cpu().double().numpy(), p1.cpu().double().numpy()
    for c in range(prob.chains):
        qr, pr, Ur, gr = o.leapfrog(prob.q0[c], p0[c], eps, L)
        assert rel_err(q1[c] - prob.q0[c], qr - prob.q0[c]) < TOL, c
        assert rel_err(p1[c] - p0[c], pr - p0[c]) < TOL, c


def test_deeponet_fp16_sampler_energy_and_resume():
    # the Metropolis energy from the hi/lo forward pass, dH against the oracle's, and the
    # same trajectories in one call or two
    prob = W.small_deeponet(n_u=150, n_y=90, du=12, width=64, latent=64, frac=0.3, chains=3, seed=41)
    s = sampler_from(prob, hmc.PREC_FP16)
    o = oracle.Oracle(prob)
    q0 = torch.from_numpy(prob.q0)
    Um = s.metropolis_energy(q0).cpu().numpy()
    Ur, _ = o.energy_grad_batch(prob.q0)
    assert np.all(np.abs(Um - Ur) <= 1e-4 * np.abs(Ur)), (Um, Ur)
    eps, L = 2e-5, 6
    _, _, dH, _ = s.sample(q0, eps, L, 1, seed=7)
    _, _, dHr, _ = o.sample(prob.q0, eps, L, 1, seed=7)
    dH = dH.cpu().numpy()
    assert np.all(np.abs(dH - dHr) <= 0.05 + 0.05 * np.abs(dHr)), (dH, dHr)
    S, acc, dH4, ql = s.sample(q0, eps, L, 4, seed=3)
    S1, _, dH1, q1 = s.sample(q0, eps, L, 2, seed=3)
    S2, _, dH2, q2 = s.sample(q1, eps, L, 2, seed=3, first_traj=2)
    assert torch.equal(torch.cat([S1, S2]), S) and torch.equal(torch.cat([dH1, dH2]), dH4)
    assert torch.equal(q2, ql)
