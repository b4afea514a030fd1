"""GPU tests of the tcgen05 tensor-core path, through the C ABI.

* The GEMM core (TMA -> smem -> tcgen05.mma -> TMEM) in all four operand
  layouts against a float32 product of the same bf16 inputs.
* BF16 U and grad U against the FP64 oracle: for every gradient evaluation the
  relative 2-norm error and the relative infinity-norm error within 2e-2; U within
  2e-2 relative.
* Full-size 2-256-256-256-256-1 network on 8192 points, 16 chains, sampled chains
  checked one by one against the oracle, in the launch configuration the
  benchmark times.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, grad_ok_bf16, rel_err, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


def _gemm(M, N, K, batch, a_mn, b_mn, seed=0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn((batch, K, M) if a_mn else (batch, M, K), generator=g).to(torch.bfloat16).cuda()
    B = torch.randn((batch, K, N) if b_mn else (batch, N, K), generator=g).to(torch.bfloat16).cuda()
    C = torch.full((batch, M, N), float("nan"), dtype=torch.float32, device="cuda")
    L = hmc.lib()
    L.hmc_diag_umma_gemm.argtypes = [ctypes.c_int] * 6 + [ctypes.c_void_p] * 3
    st = L.hmc_diag_umma_gemm(M, N, K, batch, a_mn, b_mn, A.data_ptr(), B.data_ptr(), C.data_ptr())
    assert st == 0, L.hmc_last_error()
    Am = (A.transpose(1, 2) if a_mn else A).float()
    Bn = (B.transpose(1, 2) if b_mn else B).float()
    ref = torch.bmm(Am, Bn.transpose(1, 2))
    return C, ref


@pytest.mark.parametrize("a_mn", [0, 1])
@pytest.mark.parametrize("b_mn", [0, 1])
@pytest.mark.parametrize("shape", [(128, 64, 64), (256, 256, 512), (200, 128, 200), (136, 192, 1000)])
def test_umma_gemm_layouts(a_mn, b_mn, shape):
    M, N, K = shape
    C, ref = _gemm(M, N, K, 2, a_mn, b_mn)
    assert torch.isfinite(C).all()
    err = (C - ref).abs().max().item()
    assert err <= 1e-3 * max(1.0, ref.abs().max().item()), err


def _bf16_check(prob, q, tol=2e-2):
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_BF16)
    U, g = s.energy_grad(torch.from_numpy(q))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    return s, o, U, g


@pytest.mark.parametrize("case", ["one_hidden", "ragged", "deep64", "w192_dx4"])
def test_bf16_energy_grad_parity_small(case):
    prob = {
        "one_hidden": lambda: W.small_mlp(n=300, widths=(2, 128, 128, 1), frac=0.2, chains=3, seed=21),
        "ragged": lambda: W.small_mlp(n=517, widths=(3, 256, 256, 256, 1), frac=0.05, chains=2, seed=22),
        "deep64": lambda: W.small_mlp(n=129, widths=(1, 64, 64, 64, 64, 1), frac=0.3, chains=2, seed=23),
        "w192_dx4": lambda: W.small_mlp(n=1000, widths=(4, 192, 192, 1), frac=0.1, chains=2, seed=24),
    }[case]()
    q = prob.q0
    s, o, U, g = _bf16_check(prob, q)
    Ur, gr = o.energy_grad_batch(q)
    for c in range(prob.chains):
        assert abs(U[c] - Ur[c]) <= 2e-2 * abs(Ur[c]), (c, U[c], Ur[c])
        ok, re, rinf = grad_ok_bf16(g[c], gr[c])
        assert ok, (case, c, re, rinf)


def test_bf16_full_size_wide_mlp_sampled_chains():
    # 2-256-256-256-256-1, N = 8192, 5% subset, 16 chains: the benchmark's configuration
    prob = W.wide_mlp()
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_BF16)
    U, g = s.energy_grad(torch.from_numpy(prob.q0))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(g))
    for c in (0, 15):
        Ur, gr = o.energy_grad(prob.q0[c])
        assert abs(U[c] - Ur) <= 2e-2 * abs(Ur), (c, U[c], Ur)
        ok, re, rinf = grad_ok_bf16(g[c], gr)
        assert ok, (c, re, rinf)
    # property at any size: chains that share a state agree exactly (batched launch = solo launch)
    q = np.repeat(prob.q0[3:4], 16, axis=0)
    U2, g2 = s.energy_grad(torch.from_numpy(q))
    assert torch.equal(U2, U2[0].expand(16)) and torch.equal(g2, g2[0:1].expand(16, -1))


def test_bf16_matches_fp32_engine_and_is_deterministic():
    prob = W.small_mlp(n=700, widths=(2, 256, 256, 256, 1), frac=0.05, chains=4, seed=31)
    s16 = sampler_from(prob, hmc.PREC_BF16)
    s32 = sampler_from(prob, hmc.PREC_FP32)
    q = torch.from_numpy(prob.q0)
    U16, g16 = s16.energy_grad(q)
    U16b, g16b = s16.energy_grad(q)
    assert torch.equal(U16, U16b) and torch.equal(g16, g16b)
    U32, g32 = s32.energy_grad(q)
    for c in range(4):
        ok, re, rinf = grad_ok_bf16(g16[c].cpu().numpy(), g32[c].cpu().numpy())
        assert ok, (c, re, rinf)


def test_bf16_trajectory_parity():
    prob = W.small_mlp(n=400, widths=(2, 128, 128, 128, 1), frac=0.1, chains=2, seed=41)
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_BF16)
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal(prob.q0.shape).astype(np.float32).astype(np.float64)
    eps, L = 5e-4, 10
    q1, p1 = s.leapfrog(torch.from_numpy(prob.q0), torch.from_numpy(p0), eps, L)
    q1, p1 = q1.cpu().double().numpy(), p1.cpu().double().numpy()
    for c in range(2):
        qr, pr, Ur, gr = o.leapfrog(prob.q0[c], p0[c], eps, L)
        # the position moves by eps * L * |p| ~ 5e-3; its error is bounded by the force error
        assert rel_err(q1[c] - prob.q0[c], qr - prob.q0[c]) < 2e-2
        assert rel_err(p1[c] - p0[c], pr - p0[c]) < 2e-2


def test_bf16_sampler_runs_and_resumes():
    prob = W.small_mlp(n=300, widths=(2, 128, 128, 1), frac=0.2, chains=3, seed=21)
    s = sampler_from(prob, hmc.PREC_BF16)
    q0 = torch.from_numpy(prob.q0)
    S, acc, dH, ql = s.sample(q0, 2e-4, 8, 8, seed=4)
    assert torch.isfinite(dH).all()
    S1, a1, d1, q1 = s.sample(q0, 2e-4, 8, 5, seed=4)
    S2, a2, d2, q2 = s.sample(q1, 2e-4, 8, 3, seed=4, first_traj=5)
    assert torch.equal(torch.cat([S1, S2]), S) and torch.equal(q2, ql)


def test_bf16_metropolis_energy_is_accurate():
    # bf16 activations make energy_grad's U jump by order one between nearby states; the
    # Metropolis test uses the forward pass with hi/lo activations, which follows FP32
    prob = W.small_mlp(n=2000, widths=(2, 256, 256, 256, 1), frac=0.05, chains=4, seed=51)
    s = sampler_from(prob, hmc.PREC_BF16)
    o = oracle.Oracle(prob)
    q = prob.q0
    Um = s.metropolis_energy(torch.from_numpy(q)).cpu().numpy()
    Ub = s.energy_grad(torch.from_numpy(q))[0].cpu().numpy()
    Ur, _ = o.energy_grad_batch(q)
    err_m = np.abs(Um - Ur) / np.abs(Ur)
    err_b = np.abs(Ub - Ur) / np.abs(Ur)
    assert np.all(err_m <= 1e-4), (err_m, err_b)
    # a trajectory's dH follows the FP64 oracle's from the same state and momenta
    eps, L = 2e-4, 10
    _, _, dH, _ = s.sample(torch.from_numpy(q), eps, L, 1, seed=6)
    _, _, dHr, _ = o.sample(q, eps, L, 1, seed=6)
    dH = dH.cpu().numpy()
    assert np.all(np.abs(dH - dHr) <= 0.05 + 0.05 * np.abs(dHr)), (dH, dHr, err_m, err_b)


def test_autotuner_reports_its_choices():
    # the weight-gradient grid (row splits) is timed per shape at handle creation
    prob = W.small_mlp(n=3000, widths=(2, 256, 256, 256, 1), frac=0.05, chains=4, seed=61)
    s = sampler_from(prob, hmc.PREC_BF16)
    t = s.tuning()
    assert t.startswith("problem 0: dw row splits "), t
    # a second handle of the same shape reuses the cached choice
    s2 = sampler_from(prob, hmc.PREC_BF16)
    assert "(cached)" in s2.tuning(), s2.tuning()
    # results do not depend on which handle tuned
    q = torch.from_numpy(prob.q0)
    U1, g1 = s.energy_grad(q)
    U2, g2 = s2.energy_grad(q)
    assert torch.equal(U1, U2) and torch.equal(g1, g2)
