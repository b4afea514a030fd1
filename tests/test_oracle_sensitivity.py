"""Pins for the oracle's sensitivities S_i^2 and truncation N-hat (Sec. 3.1), CPU only.

* Closed forms: a linear model (dF/dw_i = x_i) and the Case I sine network, whose
  derivatives the paper itself writes out analytically (Sec. 4.1.1).
* Finite differences of the network output, per parameter, on a ragged
  multi-output MLP and a DeepONet (brute force over every data term).
* The first-order variance the sensitivities come from (Sec. 3.1): drawing
  theta ~ N(mu, diag sd^2) with small sd, the output variance averaged over the data
  equals sum_i S_i^2, and perturbing one parameter alone gives S_i^2.
* The truncation against a brute-force enumeration of N_T, with ties, tau = 0 and 1,
  and an all-zero S2.
* Case I: with the VI means and standard deviations of Table 1, tau = 0.9 keeps the
  four parameters the paper names.
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "case1_table1.json")
NAMES = ["omega1", "omega2", "phi1", "phi2", "a", "b"]   # W1 = (w1, w2), b1 = (p1, p2), W2 = (a, b)


def _case1():
    g = json.load(open(GOLD))
    mu = np.array([g["vi"]["mean"][n] for n in NAMES])
    sd = np.array([g["vi"]["std"][n] for n in NAMES])
    return g, mu, sd


def test_linear_model_closed_form():
    prob = W.bayes_linear(n=50, d=4)
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(1)
    mu = rng.standard_normal(prob.P)
    sd = rng.uniform(0.1, 1.0, prob.P)
    S2 = o.sensitivity(mu, sd)
    x = prob.x
    ref = np.concatenate([sd[:4] ** 2 * np.mean(x ** 2, axis=0), [sd[4] ** 2]])
    assert np.allclose(S2, ref, rtol=1e-13)


def test_case1_sine_network_closed_form():
    g, mu, sd = _case1()
    prob = W.case1_sine(mu)
    S2 = oracle.Oracle(prob).sensitivity(mu, sd)
    x = prob.x[:, 0]
    w1, w2, p1, p2, a, b = mu
    d = [a * x * np.cos(w1 * x + p1), b * x * np.cos(w2 * x + p2), a * np.cos(w1 * x + p1),
         b * np.cos(w2 * x + p2), np.sin(w1 * x + p1), np.sin(w2 * x + p2)]
    ref = sd ** 2 * np.array([np.mean(v ** 2) for v in d])
    assert np.allclose(S2, ref, rtol=1e-12)


def _fd_S2(o, prob, mu, sd, h=1e-6):
    P = mu.size
    acc = np.zeros(P)
    for i in range(P):
        e = np.zeros(P)
        e[i] = h * max(1.0, abs(mu[i]))
        d = (o.forward(mu + e) - o.forward(mu - e)) / (2 * e[i])
        acc[i] = np.sum(d ** 2)
    return sd ** 2 * acc / prob.n_terms()


@pytest.mark.parametrize("which", ["mlp", "deeponet", "deeponet_unaligned"])
def test_finite_differences(which):
    if which == "mlp":
        prob = W.small_mlp(n=25, widths=(3, 7, 5, 2), acts=[W.ACT_TANH, W.ACT_SIN, W.ACT_IDENTITY],
                           bias=[True, False, True], seed=71)
    elif which == "deeponet":
        prob = W.small_deeponet(n_u=6, n_y=5, du=4, width=6, latent=3, seed=72)
    else:
        prob = W.small_deeponet_unaligned(n_u=5, n_q=4, du=3, width=6, latent=3, seed=74)
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(2)
    mu = 0.5 * rng.standard_normal(prob.P)
    sd = rng.uniform(0.05, 0.5, prob.P)
    S2 = o.sensitivity(mu, sd)
    ref = _fd_S2(o, prob, mu, sd)
    assert np.allclose(S2, ref, rtol=1e-6, atol=1e-9 * ref.max())
    assert np.all(S2 >= 0)


def test_first_order_variance_by_monte_carlo():
    # Sec. 3.1: Var[F(x)] ~ sum_i sd_i^2 (dF/dtheta_i)^2 for small sd
    prob = W.small_mlp(n=40, widths=(2, 6, 1), seed=73)
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(3)
    mu = rng.standard_normal(prob.P)
    sd = 1e-4 * rng.uniform(0.5, 1.5, prob.P)
    S2 = o.sensitivity(mu, sd)
    n = 4000
    F = np.stack([o.forward(mu + sd * rng.standard_normal(prob.P)) for _ in range(n)])   # [n][N][1]
    var = F.var(axis=0, ddof=1).mean()
    assert abs(var / S2.sum() - 1) < 4 * np.sqrt(2.0 / n), (var, S2.sum())
    for i in (0, 7, prob.P - 1):
        Fi = np.stack([o.forward(mu + (np.arange(prob.P) == i) * sd[i] * z) for z in rng.standard_normal(n)])
        vi = Fi.var(axis=0, ddof=1).mean()
        assert abs(vi / S2[i] - 1) < 4 * np.sqrt(2.0 / n), (i, vi, S2[i])


def _brute_nhat(S2, tau):
    order = sorted(range(len(S2)), key=lambda i: (-S2[i], i))
    tot = 0.0
    for v in S2:
        tot += v
    best, cum = 0, 0.0
    if tot > 0:
        for r, i in enumerate(order):
            cum += S2[i]
            if cum / tot <= tau:
                best = r + 1
            else:
                break
    return best, order


@pytest.mark.parametrize("seed", range(6))
def test_truncation_brute_force(seed):
    rng = np.random.default_rng(seed)
    P = int(rng.integers(1, 40))
    S2 = rng.exponential(1.0, P) ** 3
    if seed % 2:   # ties: a few repeated values
        S2[rng.integers(0, P, P // 3)] = S2[0]
    for tau in (0.0, 0.1, 0.5, 0.9, 0.999, 1.0):
        nhat, mask, order = oracle.truncate(S2, tau)
        bn, bo = _brute_nhat(list(S2), tau)
        assert nhat == bn
        assert list(order) == bo
        assert mask.sum() == nhat and np.all(mask[bo[:nhat]] == 1)
        # Theta_s holds exactly the parameters ranked above the cut
        if 0 < nhat < P:
            assert S2[mask == 1].min() >= S2[mask == 0].max()


def test_truncation_edges():
    assert oracle.truncate(np.zeros(5), 0.9)[0] == 0
    S2 = np.array([1.0, 1.0, 1.0, 1.0])
    assert oracle.truncate(S2, 0.5)[0] == 2
    assert list(oracle.truncate(S2, 0.5)[1]) == [1, 1, 0, 0]   # ties: lower index first
    assert oracle.truncate(S2, 1.0)[0] == 4
    assert oracle.truncate(np.array([5.0, 1.0]), 0.5)[0] == 0   # the top one alone exceeds tau


def test_case1_selects_the_papers_subset():
    g, mu, sd = _case1()
    prob = W.case1_sine(mu)
    S2 = oracle.Oracle(prob).sensitivity(mu, sd)
    nhat, mask, order = oracle.truncate(S2, g["vi_hmc_subset"]["tau"])
    assert nhat == 4
    assert sorted(NAMES[i] for i in np.flatnonzero(mask)) == sorted(g["vi_hmc_subset"]["sampled"])
    assert sorted(NAMES[i] for i in np.flatnonzero(mask == 0)) == sorted(g["vi_hmc_subset"]["fixed"])
