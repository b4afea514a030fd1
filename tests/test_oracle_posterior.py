"""Whole-sampler pins for the oracle (CPU only).

A model that is linear in its sampled parameters with a Gaussian likelihood and
a Gaussian prior has a Gaussian posterior in closed form (conjugate Bayesian
linear regression):  precision  A = Xs^T Xs / sigma^2 + I / alpha^2,
mean  m = A^{-1} Xs^T (y - X_~s theta_~s) / sigma^2.
The oracle's chains must reproduce m and A^{-1} within Monte Carlo error.  Any
slip in U, grad U, K, the integrator or the accept rule changes the stationary
distribution and fails these tests.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle.ess import ess_chains


def _check_moments(S, m, Cov, burn=200, z_max=4.5, cov_rel=0.08):
    S = S[burn:]
    n, C, k = S.shape
    # HMC chains can be antithetic (ESS > n); never credit more than n*C draws
    ess = np.minimum(ess_chains(S), n * C)
    mean = S.reshape(-1, k).mean(axis=0)
    sd = np.sqrt(np.diag(Cov))
    z = (mean - m) / (sd / np.sqrt(ess))
    assert np.all(np.abs(z) < z_max), (z, ess)
    emp = np.cov(S.reshape(-1, k).T)
    rel = np.linalg.norm(emp - Cov) / np.linalg.norm(Cov)
    assert rel < cov_rel, rel
    return ess


def _linear_closed_form(prob):
    Xa = np.concatenate([prob.x, np.ones((prob.x.shape[0], 1))], axis=1)   # W[0][:], b[0]
    s = prob.mask.astype(bool)
    y_eff = prob.y[:, 0] - Xa[:, ~s] @ prob.frozen[~s]
    Xs = Xa[:, s]
    A = Xs.T @ Xs / prob.noise_sigma**2 + np.eye(s.sum()) / prob.prior_sigma**2
    Cov = np.linalg.inv(A)
    m = Cov @ (Xs.T @ y_eff) / prob.noise_sigma**2
    return m, Cov


@pytest.mark.parametrize("mask", [None, [1, 0, 1, 1, 0, 1]])
def test_bayesian_linear_regression_posterior(mask):
    prob = W.bayes_linear(frac_mask=mask, chains=4)
    m, Cov = _linear_closed_form(prob)
    o = oracle.Oracle(prob)
    S, acc, dH, ql = o.sample(prob.q0, eps=0.012, L=12, n=12000, seed=21, threads=4)
    assert 0.6 < acc.mean() < 1.0
    _check_moments(S, m, Cov)


def test_linear_posterior_is_prior_dominated_with_weak_data():
    # large noise: the posterior approaches the N(0, alpha^2) prior
    prob = W.bayes_linear(noise=50.0, prior=0.8, chains=4)
    m, Cov = _linear_closed_form(prob)
    o = oracle.Oracle(prob)
    S, acc, _, _ = o.sample(prob.q0, eps=0.25, L=6, n=12000, seed=5, threads=4)
    _check_moments(S, m, Cov)
    assert np.allclose(np.diag(Cov), 0.64, rtol=0.05)


def test_deeponet_with_frozen_trunk_is_linear_gaussian():
    # one-layer identity branch and trunk; sampling only branch parameters and the
    # output bias leaves S_ij linear in them: a closed-form Gaussian posterior
    rng = np.random.default_rng(31)
    n_u, n_y, du, dy, p = 9, 7, 3, 2, 2
    branch = W.Net([du, p], [W.ACT_IDENTITY], [True])
    trunk = W.Net([dy, p], [W.ACT_TANH], [True])
    u = W._f32(rng.standard_normal((n_u, du)))
    yq = W._f32(rng.uniform(0, 1, (n_y, dy)))
    t = W._f32(rng.standard_normal((n_u, n_y)))
    Pb, Pt = branch.n_params(), trunk.n_params()
    P = Pb + Pt + 1
    frozen = W._f32(rng.standard_normal(P))
    mask = np.zeros(P, dtype=np.uint8)
    mask[[0, 2, 3, 5, 7, P - 1]] = 1          # some branch weights, a branch bias, b0
    q0 = np.repeat(frozen[mask.astype(bool)][None], 4, axis=0)
    prob = W.Problem("deeponet_linear", W.KIND_DEEPONET, 0.5, 1.5, frozen, mask, q0, eps=0.02, L=10,
                     branch=branch, trunk=trunk, u=u, yq=yq, t=t)
    # design matrix of S with respect to every branch parameter and b0 (trunk fixed)
    Wt = frozen[Pb:Pb + p * dy].reshape(p, dy)
    bt = frozen[Pb + p * dy:Pb + Pt]
    T = np.tanh(yq @ Wt.T + bt)                                    # [n_y][p]
    cols = []
    for c in range(p):
        for a in range(du):
            cols.append((u[:, a][:, None] * T[:, c][None, :]).ravel())
    for c in range(p):
        cols.append(np.repeat(T[:, c][None, :], n_u, axis=0).ravel())
    Xfull = np.stack(cols + [np.ones(n_u * n_y)], axis=1)          # [n_u*n_y][Pb+1]
    cols_idx = list(range(Pb)) + [P - 1]
    s = mask[cols_idx].astype(bool)
    theta_b = frozen[cols_idx]
    y_eff = t.ravel() - Xfull[:, ~s] @ theta_b[~s]
    Xs = Xfull[:, s]
    A = Xs.T @ Xs / 0.25 + np.eye(s.sum()) / 1.5**2
    Cov = np.linalg.inv(A)
    m = Cov @ Xs.T @ y_eff / 0.25
    o = oracle.Oracle(prob)
    S, acc, _, _ = o.sample(q0, eps=0.03, L=10, n=12000, seed=8, threads=4)
    assert acc.mean() > 0.5
    _check_moments(S, m, Cov)


def test_rejection_repeats_the_current_state_and_nan_rejects():
    prob = W.bayes_linear(chains=2)
    o = oracle.Oracle(prob)
    # a huge step makes the integrator unstable: most proposals are rejected
    S, acc, dH, ql = o.sample(prob.q0, eps=3.0, L=30, n=20, seed=3)
    prev = prob.q0
    for i in range(20):
        for c in range(2):
            if not acc[i, c]:
                assert np.array_equal(S[i, c], prev[c])
            else:
                assert not np.array_equal(S[i, c], prev[c])
        prev = S[i]
    assert np.array_equal(ql, S[-1])
    # non-finite energy differences never accept
    bad = ~np.isfinite(dH)
    assert not np.any(acc[bad])


def test_accept_rule_matches_log_uniform_comparison():
    prob = W.small_mlp(chains=3)
    o = oracle.Oracle(prob)
    S, acc, dH, _ = o.sample(prob.q0, eps=2e-3, L=5, n=30, seed=77, first_traj=5)
    for i in range(30):
        for c in range(3):
            lu = oracle.log(oracle.mh_uniform(77, c, 5 + i))
            assert acc[i, c] == (lu < -dH[i, c])


def test_resume_is_bit_identical():
    prob = W.small_mlp(chains=2)
    o = oracle.Oracle(prob)
    S, acc, dH, ql = o.sample(prob.q0, eps=2e-3, L=4, n=10, seed=1)
    S1, a1, d1, q1 = o.sample(prob.q0, eps=2e-3, L=4, n=6, seed=1)
    S2, a2, d2, q2 = o.sample(q1, eps=2e-3, L=4, n=4, seed=1, first_traj=6)
    assert np.array_equal(np.concatenate([S1, S2]), S)
    assert np.array_equal(np.concatenate([d1, d2]), dH)
