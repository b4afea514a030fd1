"""The tensor-core path with fp16 GEMM operands (HMC_PREC_FP16), through the C ABI.

fp16 keeps 11 significant bits against bf16's 8 at the same bytes and tensor rate.  Its
tolerance against the FP64 oracle, 5e-3 on every gradient (relative 2-norm and relative
infinity-norm) and on U, is ten units of fp16 rounding (2^-11): the deltas of the
adjoint carry r / sigma, so their rounding errors reach the gradient amplified by the
residual-to-noise ratio, a few units on these problems.

* U and grad U against the oracle on small and ragged shapes and at full benchmark size.
* Every gradient along an oracle trajectory, and the endpoint of the library's own
  leapfrog (Sec. 2.2, Algorithm 1), within the tolerance.
* The accurate Metropolis energy (hi/lo activations) within 1e-4 of the oracle.
* Sampling runs, resumes bit-identically, and its acceptance at a fixed step matches
  the FP32 sampler's on paired starts (same states, same momenta): the force error of
  the 16-bit GEMMs does not cost acceptance.
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

SMALL = {
    "one_hidden": lambda: W.small_mlp(n=300, widths=(2, 128, 128, 1), frac=0.2, chains=3, seed=21),
    "ragged": lambda: W.small_mlp(n=517, widths=(3, 256, 256, 256, 1), frac=0.05, chains=2, seed=22),
    "deep64": lambda: W.small_mlp(n=129, widths=(1, 64, 64, 64, 64, 1), frac=0.3, chains=2, seed=23),
    "w192_dx4": lambda: W.small_mlp(n=1000, widths=(4, 192, 192, 1), frac=0.1, chains=2, seed=24),
}


def _eg(s, q):
    U, g = s.energy_grad(torch.from_numpy(q))
    return U.cpu().numpy(), g.cpu().double().numpy()


@pytest.mark.parametrize("case", sorted(SMALL))
def test_fp16_energy_grad_parity_small(case):
    prob = SMALL[case]()
    o = oracle.Oracle(prob)
    U, g = _eg(sampler_from(prob, hmc.PREC_FP16), prob.q0)
    Ur, gr = o.energy_grad_batch(prob.q0)
    for c in range(prob.chains):
        assert abs(U[c] - Ur[c]) <= TOL * abs(Ur[c]), (c, U[c], Ur[c])
        ok, re, rinf = grad_ok_bf16(g[c], gr[c], TOL)
        assert ok, (case, c, re, rinf)


def test_fp16_is_more_accurate_than_bf16():
    prob = W.small_mlp(n=2000, widths=(2, 256, 256, 256, 1), frac=0.05, chains=4, seed=52)
    Ur, gr = oracle.Oracle(prob).energy_grad_batch(prob.q0)
    _, g16 = _eg(sampler_from(prob, hmc.PREC_FP16), prob.q0)
    _, gb = _eg(sampler_from(prob, hmc.PREC_BF16), prob.q0)
    e16 = max(rel_err(g16[c], gr[c]) for c in range(4))
    eb = max(rel_err(gb[c], gr[c]) for c in range(4))
    assert e16 < 0.35 * eb, (e16, eb)


def test_fp16_full_size_wide_mlp_sampled_chains():
    # 2-256-256-256-256-1, N = 8192, 5% subset, 16 chains: the benchmark's configuration
    prob = W.wide_mlp()
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_FP16)
    U, g = _eg(s, prob.q0)
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(g))
    for c in (0, 7, 15):
        Ur, gr = o.energy_grad(prob.q0[c])
        assert abs(U[c] - Ur) <= TOL * abs(Ur), (c, U[c], Ur)
        ok, re, rinf = grad_ok_bf16(g[c], gr, TOL)
        assert ok, (c, re, rinf)
    Um = s.metropolis_energy(torch.from_numpy(prob.q0)).cpu().numpy()
    Ur, _ = o.energy_grad_batch(prob.q0[:2])
    assert np.all(np.abs(Um[:2] - Ur) <= 1e-4 * np.abs(Ur)), (Um[:2], Ur)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_every_gradient_along_an_oracle_trajectory(prec):
    # the oracle integrates L leapfrog steps; at every state it visits the library's
    # gradient is within the precision's tolerance of the oracle's
    tol = TOL if prec == "fp16" else 2e-2
    prob = W.small_mlp(n=400, widths=(2, 128, 128, 128, 1), frac=0.1, chains=2, seed=41)
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_FP16 if prec == "fp16" else hmc.PREC_BF16)
    rng = np.random.default_rng(9)
    p0 = rng.standard_normal(prob.q0.shape).astype(np.float32).astype(np.float64)
    eps, L = 5e-4, 10
    for c in range(2):
        q, p = prob.q0[c].copy(), p0[c].copy()
        states = [q.copy()]
        for _ in range(L):
            q, p, _, _ = o.leapfrog(q, p, eps, 1)
            states.append(q.copy())
        Q = np.stack(states)                           # [L + 1][k] on the oracle's path
        Ur, gr = o.energy_grad_batch(Q)
        for i in range(0, L + 1, 2):                   # chains of the handle: two states at a time
            qq = np.repeat(Q[i:i + 1], prob.chains, axis=0)
            if i + 1 <= L:
                qq[1] = Q[i + 1]
            U, g = _eg(s, qq)
            for j in range(min(2, L + 1 - i)):
                ok, re, rinf = grad_ok_bf16(g[j], gr[i + j], tol)
                assert ok, (prec, c, i + j, re, rinf)
    # and the library's own trajectory ends where the oracle's does, to that tolerance
    q1, p1 = s.leapfrog(torch.from_numpy(prob.q0), torch.from_numpy(p0), eps, L)
    q1, p1 = q1.cpu().double().numpy(), p1.cpu().double().numpy()
    for c in range(2):
        qr, pr, _, _ = o.leapfrog(prob.q0[c], p0[c], eps, L)
        assert rel_err(q1[c] - prob.q0[c], qr - prob.q0[c]) < tol
        assert rel_err(p1[c] - p0[c], pr - p0[c]) < tol


def test_fp16_sampler_runs_and_resumes():
    prob = W.small_mlp(n=300, widths=(2, 128, 128, 1), frac=0.2, chains=3, seed=21)
    s = sampler_from(prob, hmc.PREC_FP16)
    q0 = torch.from_numpy(prob.q0)
    S, acc, dH, ql = s.sample(q0, 2e-4, 8, 8, seed=4)
    assert torch.isfinite(dH).all()
    S1, a1, d1, q1 = s.sample(q0, 2e-4, 8, 5, seed=4)
    S2, a2, d2, q2 = s.sample(q1, 2e-4, 8, 3, seed=4, first_traj=5)
    assert torch.equal(torch.cat([S1, S2]), S) and torch.equal(q2, ql)


def test_fp16_acceptance_matches_fp32_on_paired_starts():
    # a misfit MLP whose residuals are ten times the noise (r / sigma ~ 10, as on the
    # benchmark workload), warmed up by the FP32 sampler; from each visited state both
    # samplers run one trajectory with the same momenta (same seed and index), so the
    # acceptance probabilities min(1, exp(-dH)) are paired
    prob = W.small_mlp(n=2048, widths=(2, 128, 128, 128, 1), frac=0.05, chains=16, seed=77, noise=0.05)
    s32 = sampler_from(prob, hmc.PREC_FP32)
    s16 = sampler_from(prob, hmc.PREC_FP16)
    L = 20
    eps, q = s32.adapt_step_size(torch.from_numpy(prob.q0), L, 1e-3, 60, target_accept=0.8, seed=3)
    S, _, _, _ = s32.sample(q, eps, L, 24, seed=3, first_traj=100)
    a32, a16 = [], []
    for t in range(0, 24, 2):
        start = S[t].contiguous()
        _, _, d32, _ = s32.sample(start, eps, L, 1, seed=11, first_traj=1000 + t, keep_samples=False)
        _, _, d16, _ = s16.sample(start, eps, L, 1, seed=11, first_traj=1000 + t, keep_samples=False)
        a32.append(np.minimum(1.0, np.exp(-d32.cpu().numpy().ravel())))
        a16.append(np.minimum(1.0, np.exp(-d16.cpu().numpy().ravel())))
    a32, a16 = np.concatenate(a32), np.concatenate(a16)
    diff = a16 - a32
    se = diff.std(ddof=1) / np.sqrt(diff.size)
    assert abs(diff.mean()) <= 3.0 * se + 0.01, (a32.mean(), a16.mean(), se)


def test_fp16_engine_tanh_is_accurate_to_1e_6():
    # the fp16 engine's epilogues evaluate tanh from the base-2 exponential and reciprocal;
    # its absolute error must stay under half an fp16 unit of values above 2^-8 (1e-6
    # everywhere), with |tanh| <= 1
    x = torch.cat([torch.linspace(-40, 40, 1 << 20), torch.linspace(-1e-3, 1e-3, 4096),
                   torch.tensor([1e30, -1e30, 9.0, -9.0, 0.0])]).float().cuda()
    y = torch.empty_like(x)
    assert hmc.lib().hmc_diag_tanh16(x.data_ptr(), y.data_ptr(), x.numel()) == 0
    ref = torch.tanh(x.double())
    assert (y.double() - ref).abs().max().item() <= 1e-6
    assert y.abs().max().item() <= 1.0


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("widths", [(2, 40, 40, 1), (3, 100, 100, 100, 1), (4, 200, 200, 1), (6, 100, 100, 1),
                                    (7, 128, 128, 128, 1), (8, 64, 64, 1), (6, 256, 256, 1)])
def test_hidden_widths_padded_with_zero_units(prec, widths):
    # the tensor-core engines pad a hidden width to 128 (or 256 above 128) with zero units
    prob = W.small_mlp(n=300, widths=widths, frac=0.2, chains=2, seed=61)
    tol = TOL if prec == "fp16" else 2e-2
    U, g = _eg(sampler_from(prob, hmc.PREC_FP16 if prec == "fp16" else hmc.PREC_BF16), prob.q0)
    Ur, gr = oracle.Oracle(prob).energy_grad_batch(prob.q0)
    for c in range(prob.chains):
        assert abs(U[c] - Ur[c]) <= tol * abs(Ur[c]), (c, U[c], Ur[c])
        ok, re, rinf = grad_ok_bf16(g[c], gr[c], tol)
        assert ok, (widths, c, re, rinf)
