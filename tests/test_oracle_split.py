"""Pins for the oracle's symmetric split integrator over data batches (CPU only).

The split Hamiltonian H = sum_m [U_m + K/M] (U_m: likelihood of data batch m plus
1/M of the prior) is integrated by a forward sweep over the batches and the
mirrored backward sweep (the symmetric split HMC that Sec. 4.2.3 uses for its full-HMC
runs).  What fixes it, independently of its own code:
* the batches partition the data: sum_m U_m = U and sum_m grad U_m = grad U;
* with one batch the step is the leapfrog step (itself pinned by the harmonic
  oscillator's closed form);
* a palindromic composition of exact sub-flows is time reversible;
* it is of second order: |dH| at a fixed trajectory length shrinks 4x when eps halves,
  and its end point converges to the leapfrog end point (the same Hamiltonian flow)
  at the same rate;
* the sampler it drives keeps the closed-form posterior of Bayesian linear
  regression.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_posterior import _check_moments, _linear_closed_form


def _probs():
    return {"small_mlp": W.small_mlp, "deeponet": W.small_deeponet, "tiny_bnn": lambda: W.tiny_bnn(n=64),
            "deeponet_unaligned": W.small_deeponet_unaligned}


@pytest.mark.parametrize("which", ["small_mlp", "deeponet", "deeponet_unaligned"])
@pytest.mark.parametrize("M", [1, 3, 7])
def test_batches_partition_the_data(which, M):
    prob = _probs()[which]()
    o = oracle.Oracle(prob)
    R = o.data_rows()
    bounds = [o.batch_rows(M, m) for m in range(M)]
    assert bounds[0][0] == 0 and bounds[-1][1] == R
    for (a0, a1), (b0, b1) in zip(bounds, bounds[1:]):
        assert a1 == b0
    assert all(r1 - r0 in (R // M, R // M + 1) for r0, r1 in bounds)
    q = prob.q0[1]
    U, g = o.energy_grad(q)
    parts = [o.energy_grad_rows(q, r0, r1, 1.0 / M) for r0, r1 in bounds]
    Us = sum(p[0] for p in parts)
    gs = sum(p[1] for p in parts)
    assert abs(Us - U) <= 1e-12 * abs(U)
    assert np.max(np.abs(gs - g)) <= 1e-11 * np.max(np.abs(g))
    # the prior alone: no rows, whole weight
    U0, g0 = o.energy_grad_rows(q, 0, 0, 1.0)
    assert np.isclose(U0, q @ q / (2 * prob.prior_sigma**2), rtol=1e-14)
    assert np.allclose(g0, q / prob.prior_sigma**2, rtol=1e-14)


@pytest.mark.parametrize("which", ["small_mlp", "deeponet"])
def test_one_batch_is_the_leapfrog(which):
    prob = _probs()[which]()
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(4)
    q0, p0 = prob.q0[0], rng.standard_normal(prob.k)
    q1, p1, _, _ = o.leapfrog(q0, p0, 3e-4, 9)
    q2, p2 = o.split_leapfrog(q0, p0, 3e-4, 9, 1)
    assert np.max(np.abs(q2 - q1)) <= 1e-12 * max(1.0, np.max(np.abs(q1)))
    assert np.max(np.abs(p2 - p1)) <= 1e-10 * max(1.0, np.max(np.abs(p1)))


@pytest.mark.parametrize("which", ["small_mlp", "deeponet", "tiny_bnn"])
def test_split_integrator_is_reversible(which):
    prob = _probs()[which]()
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(5)
    q0, p0 = prob.q0[0], rng.standard_normal(prob.k)
    eps, L, M = 2e-4, 12, 4
    q1, p1 = o.split_leapfrog(q0, p0, eps, L, M)
    q2, p2 = o.split_leapfrog(q1, -p1, eps, L, M)
    assert np.max(np.abs(q2 - q0)) <= 1e-10 * max(1.0, np.max(np.abs(q0)))
    assert np.max(np.abs(-p2 - p0)) <= 1e-10 * max(1.0, np.max(np.abs(p0)))
    assert np.max(np.abs(q1 - q0)) > 1e-6


@pytest.mark.parametrize("which", ["tiny_bnn", "deeponet"])
def test_split_integrator_is_second_order(which):
    prob = _probs()[which]()
    T, eps0 = {"tiny_bnn": (2e-3, 1e-4), "deeponet": (4e-3, 4e-4)}[which]
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(6)
    q, p = prob.q0[0], rng.standard_normal(prob.k)
    H0 = o.energy(q) + 0.5 * p @ p
    dH, gap = [], []
    for m in (1, 2, 4):
        eps = eps0 / m
        L = int(round(T / eps))
        qs, ps = o.split_leapfrog(q, p, eps, L, 3)
        dH.append(abs(o.energy(qs) + 0.5 * ps @ ps - H0))
        ql, pl, _, _ = o.leapfrog(q, p, eps, L)
        gap.append(np.linalg.norm(qs - ql) + np.linalg.norm(ps - pl))
    for e in (dH, gap):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 3.2 < r1 < 4.8, e
        assert 3.2 < r2 < 4.8, e


@pytest.mark.parametrize("M", [2, 5])
def test_split_sampler_keeps_the_linear_posterior(M):
    prob = W.bayes_linear(frac_mask=[1, 1, 0, 1, 1, 1], chains=4)
    m, Cov = _linear_closed_form(prob)
    o = oracle.Oracle(prob)
    S, acc, dH, ql = o.split_sample(prob.q0, eps=0.012, L=12, n=12000, M=M, seed=23, threads=4)
    assert 0.6 < acc.mean() < 1.0
    _check_moments(S, m, Cov)


def test_split_sampler_accept_rule_and_resume():
    prob = W.small_mlp(chains=2)
    o = oracle.Oracle(prob)
    S, acc, dH, ql = o.split_sample(prob.q0, eps=2e-3, L=4, n=8, M=3, seed=9, first_traj=2)
    for i in range(8):
        for c in range(2):
            lu = oracle.log(oracle.mh_uniform(9, c, 2 + i))
            assert acc[i, c] == (lu < -dH[i, c])
    S1, _, d1, q1 = o.split_sample(prob.q0, eps=2e-3, L=4, n=5, M=3, seed=9, first_traj=2)
    S2, _, d2, _ = o.split_sample(q1, eps=2e-3, L=4, n=3, M=3, seed=9, first_traj=7)
    assert np.array_equal(np.concatenate([S1, S2]), S)
    assert np.array_equal(np.concatenate([d1, d2]), dH)
