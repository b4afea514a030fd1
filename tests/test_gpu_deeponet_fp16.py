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
from _adapt import grad_ok_bf16, sampler_from

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
