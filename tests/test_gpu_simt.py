"""GPU parity of the CUDA-core (FP64 / FP32) path against the FP64 oracle, through the C ABI.

Tolerances: FP64 relative 1e-10 (sums in a different order only); FP32 1e-5 on
U and grad U (relative 2-norm and per component against |g| + rms(g)).
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, rel_err, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


def _cases():
    return {
        "small_mlp": W.small_mlp(),
        "sin_1layer": W.small_mlp(widths=(2, 17, 1), acts=[W.ACT_SIN, W.ACT_IDENTITY], frac=0.6, seed=1),
        "mixed_nobias": W.small_mlp(widths=(4, 9, 9, 3), acts=[W.ACT_TANH, W.ACT_SIN, W.ACT_TANH],
                                    bias=[True, False, True], frac=0.5, seed=2),
        "ragged_wide": W.small_mlp(n=517, widths=(3, 130, 67, 1), frac=0.1, seed=5),
        "deeponet": W.small_deeponet(),
        "deeponet_nob0": W.small_deeponet(out_bias=False, frac=0.5, seed=4),
        "deeponet_ragged": W.small_deeponet(n_u=70, n_y=131, du=20, width=65, latent=33, frac=0.2, seed=9),
        "tiny_bnn": W.tiny_bnn(chains=3),
        "k_equals_1": W.small_mlp(frac=0.0007, seed=11),
    }


@pytest.mark.parametrize("name", list(_cases().keys()))
@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_energy_grad_parity(name, prec):
    prob = _cases()[name]
    if prob.k == 0:
        pytest.skip("empty subset")
    o = oracle.Oracle(prob)
    s = sampler_from(prob, prec)
    rng = np.random.default_rng(3)
    q = prob.q0 + 0.02 * rng.standard_normal(prob.q0.shape)
    q = q.astype(np.float32).astype(np.float64)
    U, g = s.energy_grad(torch.from_numpy(q))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    Ur, gr = o.energy_grad_batch(q)
    tol = 1e-10 if prec == hmc.PREC_FP64 else 1e-5
    for c in range(prob.chains):
        assert abs(U[c] - Ur[c]) <= tol * abs(Ur[c]), (c, U[c], Ur[c])
        ok, re, comp = grad_ok(g[c], gr[c], tol)
        assert ok, (c, re, comp)


@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_leapfrog_trajectory_parity(prec):
    prob = W.small_mlp(n=333, widths=(2, 48, 40, 1), frac=0.25, chains=2, seed=12)
    o = oracle.Oracle(prob)
    s = sampler_from(prob, prec)
    rng = np.random.default_rng(4)
    p0 = rng.standard_normal(prob.q0.shape).astype(np.float32).astype(np.float64)
    eps, L = 2e-3, 12
    q1, p1 = s.leapfrog(torch.from_numpy(prob.q0), torch.from_numpy(p0), eps, L)
    q1, p1 = q1.cpu().double().numpy(), p1.cpu().double().numpy()
    tol = 1e-10 if prec == hmc.PREC_FP64 else 1e-5
    for c in range(prob.chains):
        qr, pr, Ur, gr = o.leapfrog(prob.q0[c], p0[c], eps, L)
        assert rel_err(q1[c], qr) <= tol
        assert rel_err(p1[c], pr) <= 10 * tol
        U, _ = s.energy_grad(torch.from_numpy(q1))
        Hg = U.cpu().numpy()[c] + 0.5 * p1[c] @ p1[c]
        Hr = Ur + 0.5 * pr @ pr
        assert abs(Hg - Hr) <= tol * abs(Hr)


def test_leapfrog_zero_steps_is_identity():
    prob = W.small_mlp(chains=2)
    s = sampler_from(prob, hmc.PREC_FP64)
    p0 = np.ones_like(prob.q0)
    q1, p1 = s.leapfrog(torch.from_numpy(prob.q0), torch.from_numpy(p0), 1e-2, 0)
    assert np.array_equal(q1.cpu().numpy(), prob.q0) and np.array_equal(p1.cpu().numpy(), p0)


def _sample_parity(prob, prec, n, eps, L, seed=5, first_traj=0):
    o = oracle.Oracle(prob)
    s = sampler_from(prob, prec)
    S, acc, dH, ql = s.sample(torch.from_numpy(prob.q0), eps, L, n, seed=seed, first_traj=first_traj)
    Sr, accr, dHr, qlr = o.sample(prob.q0, eps, L, n, seed=seed, first_traj=first_traj)
    return (S.cpu().double().numpy(), acc.cpu().numpy(), dH.cpu().numpy(), ql.cpu().double().numpy(),
            Sr, accr, dHr, qlr)


def test_sample_parity_fp64_tiny_bnn():
    # the tiny BNN regression (1-20-20-1 tanh, all 481 parameters) over 25 trajectories
    prob = W.tiny_bnn(chains=2)
    S, acc, dH, ql, Sr, accr, dHr, qlr = _sample_parity(prob, hmc.PREC_FP64, 25, 1e-3, 20)
    band = 1e-8 * (1 + np.abs(dHr))
    lu = np.array([[oracle.log(oracle.mh_uniform(5, c, t)) for c in range(2)] for t in range(25)])
    clear = np.abs(lu + dHr) > band
    assert np.array_equal(acc[clear], accr[clear])
    assert np.allclose(dH, dHr, rtol=1e-6, atol=1e-7)
    assert rel_err(S, Sr) < 1e-9


def test_sample_parity_fp32_deeponet():
    prob = W.small_deeponet(chains=3)
    S, acc, dH, ql, Sr, accr, dHr, qlr = _sample_parity(prob, hmc.PREC_FP32, 10, 1e-3, 6)
    lu = np.array([[oracle.log(oracle.mh_uniform(5, c, t)) for c in range(3)] for t in range(10)])
    clear = np.abs(lu + dHr) > 1e-3 * (1 + np.abs(dHr))
    assert np.array_equal(acc[clear], accr[clear])
    # until the first flag disagreement (none outside the band), the chains track the oracle
    assert rel_err(S, Sr) < 1e-4


def test_gpu_momenta_and_uniforms_bit_exact():
    for seed, chain, traj, k in [(0, 0, 0, 13), (123456789, 7, 99, 1001), (2**63 + 5, 3, 2**40, 8)]:
        got = hmc.diag_momenta(seed, chain, traj, k)
        want = oracle.momenta(seed, chain, traj, k)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (seed, chain, traj)
    lu = hmc.diag_log_uniform(42, 5, 40)
    want = np.array([[oracle.log(oracle.mh_uniform(42, c, t)) for t in range(40)] for c in range(5)])
    assert np.array_equal(lu.view(np.uint64), want.view(np.uint64))
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**63, size=(64, 4), dtype=np.uint64)
    key = rng.integers(0, 2**63, size=(64, 2), dtype=np.uint64)
    got = hmc.diag_philox(ctr, key)
    for i in range(64):
        assert np.array_equal(got[i], oracle.philox4x64_10(ctr[i], key[i]))


def test_sample_momenta_are_the_oracle_momenta():
    # with a prior-only target the first trajectory is a closed-form function of p0
    prob = W.harmonic(k=9, chains=2, eps=0.05, L=3)
    S, acc, dH, ql, Sr, accr, dHr, qlr = _sample_parity(prob, hmc.PREC_FP64, 4, 0.05, 3, seed=77)
    assert np.allclose(S, Sr, rtol=1e-13, atol=1e-14)
    assert np.array_equal(acc, accr)


@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_resume_is_bit_identical(prec):
    prob = W.small_mlp(chains=2)
    s = sampler_from(prob, prec)
    q0 = torch.from_numpy(prob.q0)
    S, acc, dH, ql = s.sample(q0, 2e-3, 4, 10, seed=1)
    S1, a1, d1, q1 = s.sample(q0, 2e-3, 4, 6, seed=1)
    S2, a2, d2, q2 = s.sample(q1, 2e-3, 4, 4, seed=1, first_traj=6)
    assert torch.equal(torch.cat([S1, S2]), S)
    assert torch.equal(torch.cat([d1, d2]), dH)
    assert torch.equal(q2, ql)


def test_host_buffers_match_device_buffers():
    prob = W.small_mlp(chains=2)
    s = sampler_from(prob, hmc.PREC_FP32)
    S, acc, dH, ql = s.sample(torch.from_numpy(prob.q0), 2e-3, 4, 5, seed=3)
    Sh, acch, dHh, qlh = s.sample_host(prob.q0, 2e-3, 4, 5, seed=3)
    assert np.array_equal(S.cpu().numpy(), Sh) and np.array_equal(dH.cpu().numpy(), dHh)
    assert np.array_equal(acc.cpu().numpy(), acch) and np.array_equal(ql.cpu().numpy(), qlh)


def test_autograd_function_uses_the_adjoint():
    prob = W.small_mlp(chains=3)
    s = sampler_from(prob, hmc.PREC_FP64)
    q = torch.from_numpy(prob.q0).cuda().requires_grad_(True)
    U = hmc.energy(q, s)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (U * w).sum().backward()
    _, g = s.energy_grad(q.detach())
    assert torch.allclose(q.grad, w[:, None] * g)


def test_errors_are_reported_not_raised_across_the_abi():
    prob = W.small_mlp()
    with pytest.raises(hmc.HmcError) as e:
        hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, np.zeros(prob.P, np.uint8), prob.frozen, 1)
    assert e.value.status == 1
    with pytest.raises(hmc.HmcError) as e:
        hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, 1, noise_sigma=-1.0)
    assert e.value.status == 1
    with pytest.raises(hmc.HmcError) as e:
        hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, 1, prec=hmc.PREC_TF32)
    assert e.value.status == 6
    s = sampler_from(prob, hmc.PREC_FP32)
    with pytest.raises(hmc.HmcError) as e:
        s.sample(torch.from_numpy(prob.q0), -1.0, 3, 2)
    assert e.value.status == 1


def test_nonfinite_energy_is_flagged_and_rejected():
    prob = W.small_mlp(chains=2)
    s = sampler_from(prob, hmc.PREC_FP32)
    q = np.array(prob.q0)
    q[1, 0] = np.inf
    U = np.zeros(2)
    st = hmc.lib().hmc_energy_grad(s._h, torch.from_numpy(q.astype(np.float32)).cuda().data_ptr(),
                                   U.ctypes.data, None)
    assert st == 4 and np.isfinite(U[0]) and not np.isfinite(U[1])
    # a chain whose proposals blow up rejects them; the other chain is unaffected
    S, acc, dH, ql = s.sample(torch.from_numpy(prob.q0), 50.0, 5, 3, seed=2)
    bad = ~np.isfinite(dH.cpu().numpy())
    assert not acc.cpu().numpy()[bad].any()


@pytest.mark.parametrize("eps0", [2e-1, 1e-3])
def test_step_size_adaptation_reaches_the_target_acceptance(eps0):
    # dual averaging during warm-up (the paper tunes eps to ~80% acceptance): from a step
    # far too large or far too small, the adapted step gives acceptance near the target
    prob = W.bayes_linear(chains=4)
    s = sampler_from(prob, hmc.PREC_FP64)
    L = 10
    eps, q = s.adapt_step_size(torch.from_numpy(prob.q0), L, eps0, 80, target_accept=0.8, seed=12)
    assert np.isfinite(eps) and eps > 0
    S, acc, dH, ql = s.sample(q, eps, L, 60, seed=12, first_traj=80)
    a = float(np.minimum(1.0, np.exp(-dH.cpu().numpy())).mean())
    assert 0.6 <= a <= 0.95, (eps0, eps, a)
