"""GPU parity of the DeepONet whose input functions carry their own query points
(HMC_NET_DEEPONET_UNALIGNED) against the FP64 oracle, through the C ABI.

Every function's queries go through the trunk as rows of their own; S_jk is a
row-wise dot product with B_j, dB_j sums over the function's queries and dT_jk is
dS_jk B_j.  Tolerances as for the aligned DeepONet: 1e-10 (FP64), 1e-5 (FP32).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


CASES = {
    "ragged": lambda: W.small_deeponet_unaligned(n_u=37, n_q=13, chains=3),
    "no_b0_tanh_out": lambda: W.small_deeponet_unaligned(n_u=20, n_q=70, du=3, width=40, latent=20, chains=2,
                                                         out_bias=False, seed=8109),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_unaligned_energy_grad_parity(case, prec):
    prob = CASES[case]()
    s = sampler_from(prob, prec)
    U, g = s.energy_grad(torch.from_numpy(prob.q0))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    Ur, gr = oracle.Oracle(prob).energy_grad_batch(prob.q0)
    tol = 1e-10 if prec == hmc.PREC_FP64 else 1e-5
    for c in range(prob.chains):
        assert abs(U[c] - Ur[c]) <= tol * abs(Ur[c]), (c, U[c], Ur[c])
        ok, re, comp = grad_ok(g[c], gr[c], tol)
        assert ok, (c, re, comp)


def test_unaligned_with_shared_queries_is_the_aligned_one():
    pu = W.small_deeponet_unaligned(shared=True, chains=2)
    pa = W.Problem("aligned", W.KIND_DEEPONET, pu.noise_sigma, pu.prior_sigma, pu.frozen, pu.mask, pu.q0,
                   eps=pu.eps, L=pu.L, branch=pu.branch, trunk=pu.trunk, out_bias=pu.out_bias,
                   u=pu.u, yq=pu.yq[0], t=pu.t)
    q = torch.from_numpy(pu.q0)
    Uu, gu = sampler_from(pu, hmc.PREC_FP64).energy_grad(q)
    Ua, ga = sampler_from(pa, hmc.PREC_FP64).energy_grad(q)
    assert torch.allclose(Uu, Ua, rtol=1e-13, atol=0)
    assert torch.allclose(gu, ga, rtol=1e-11, atol=1e-11 * ga.abs().max().item())


def test_unaligned_sample_parity_fp64_and_split():
    prob = CASES["ragged"]()
    o = oracle.Oracle(prob)
    n, eps, L, seed = 3, 2e-4, 5, 19
    for M in (1, 3):
        s = sampler_from(prob, hmc.PREC_FP64, n_splits=M)
        S, acc, dH, _ = s.sample(torch.from_numpy(prob.q0), eps, L, n, seed=seed)
        S, acc, dH = S.cpu().numpy(), acc.cpu().numpy(), dH.cpu().numpy()
        if M == 1:
            Sr, accr, dHr, _ = o.sample(prob.q0, eps, L, n, seed=seed)
        else:
            Sr, accr, dHr, _ = o.split_sample(prob.q0, eps, L, n, M, seed=seed)
        lu = np.array([[oracle.log(oracle.mh_uniform(seed, c, t)) for c in range(prob.chains)] for t in range(n)])
        clear = np.abs(lu + dHr) > 1e-8 * (1 + np.abs(dHr))
        assert np.array_equal(acc[clear], accr[clear]), M
        assert np.allclose(dH, dHr, rtol=1e-6, atol=1e-7), M
        assert np.max(np.abs(S - Sr)) <= 1e-9 * max(1.0, np.max(np.abs(Sr))), M


def test_unaligned_grf_sized_fp32():
    # 500 GRF-like functions, each with its own 100 query points, GRF-workload widths
    prob = W.small_deeponet_unaligned(n_u=500, n_q=100, du=100, width=128, latent=64, frac=0.1, chains=4,
                                      seed=8110)
    s = sampler_from(prob, hmc.PREC_FP32)
    U, g = s.energy_grad(torch.from_numpy(prob.q0))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    o = oracle.Oracle(prob)
    for c in (0, 3):
        Ur, gr = o.energy_grad(prob.q0[c])
        assert abs(U[c] - Ur) <= 1e-5 * abs(Ur)
        ok, re, comp = grad_ok(g[c], gr, 1e-5)
        assert ok, (c, re, comp)


def test_unaligned_rejections():
    prob = CASES["ragged"]()
    with pytest.raises(hmc.HmcError):
        sampler_from(prob, hmc.PREC_BF16)
    s = sampler_from(prob, hmc.PREC_FP32)
    with pytest.raises(hmc.HmcError):
        s.predict(torch.from_numpy(prob.q0), u=prob.u, yq=prob.yq)
