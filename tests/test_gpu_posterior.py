"""Statistical parity of the GPU samplers: their chains must have the posterior's moments.

HMC with a Metropolis step samples the canonical distribution exp(-U) exactly (Sec. 2.2,
Algorithms 1 and 2), whatever the force's rounding, as long as the energy of the
Metropolis test is the true one.  Checked on the GPU, with means within 4.5 Monte Carlo
standard errors (z over the effective sample size) and covariances within a few percent:

* FP64 and FP32 chains on a Bayesian linear regression (full and partial subsets)
  against its closed-form Gaussian posterior;
* BF16 and FP16 tensor-core chains on a tanh MLP whose sampled parameters are output
  weights and the output bias only: the model is linear in them, so the posterior is
  Gaussian in closed form, with features taken from the oracle's forward pass;
* BF16 and FP16 chains on a subset that reaches into the hidden layers against the
  moments of long FP64 oracle chains of the same problem, stored by
  tests/golden/make_hidden_subset_moments.py (means and variances, both estimates' errors).
"""
import json
import os

import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import sampler_from
from oracle.ess import ess_chains

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


def _ess(S):
    n, C, _ = S.shape
    return np.minimum(ess_chains(S), n * C)     # antithetic chains are never credited more


def _check_moments(S, m, Cov, z_max=4.5, cov_rel=0.08):
    n, C, k = S.shape
    ess = _ess(S)
    mean = S.reshape(-1, k).mean(axis=0)
    sd = np.sqrt(np.diag(Cov))
    z = (mean - m) / (sd / np.sqrt(ess))
    assert np.all(np.abs(z) < z_max), (z, ess)
    emp = np.cov(S.reshape(-1, k).T)
    rel = np.linalg.norm(emp - Cov) / np.linalg.norm(Cov)
    assert rel < cov_rel, (rel, ess.min())


def _gpu_chains(s, q0, eps, Ls, n_per, seed):
    """Chains of blocks of n_per trajectories, block i with L = Ls[i]: a fixed trajectory
    length can sit near a multiple of a half-period of some posterior direction, where HMC
    barely moves; varying it between blocks keeps every block an exact MH kernel."""
    q, out = torch.from_numpy(np.asarray(q0)), []
    for i, L in enumerate(Ls):
        S, _, _, q = s.sample(q, eps, int(L), n_per, seed=seed, first_traj=i * n_per)
        out.append(S.cpu().double().numpy())
    return np.concatenate(out)


def _lengths(L0, blocks, seed):
    return np.random.default_rng(seed).integers(L0 // 2, 3 * L0 // 2 + 1, blocks)


def _linear_closed_form(X, y, mask_cols, frozen_cols, noise, prior):
    """Posterior N(m, Cov) of theta_s for y = X theta + noise, theta_~s fixed."""
    s = mask_cols.astype(bool)
    y_eff = y - X[:, ~s] @ frozen_cols[~s]
    Xs = X[:, s]
    A = Xs.T @ Xs / noise ** 2 + np.eye(s.sum()) / prior ** 2
    Cov = np.linalg.inv(A)
    return Cov @ (Xs.T @ y_eff) / noise ** 2, Cov


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("mask", [None, [1, 0, 1, 1, 0, 1]])
def test_linear_regression_posterior_on_the_gpu(prec, mask):
    prob = W.bayes_linear(frac_mask=mask, chains=32)
    Xa = np.concatenate([prob.x, np.ones((prob.x.shape[0], 1))], axis=1)   # W[0][:], then b[0]
    m, Cov = _linear_closed_form(Xa, prob.y[:, 0], prob.mask, prob.frozen, prob.noise_sigma, prob.prior_sigma)
    s = sampler_from(prob, hmc.PREC_FP64 if prec == "fp64" else hmc.PREC_FP32)
    S = _gpu_chains(s, prob.q0, 0.012, _lengths(12, 30, 1), 50, seed=21)
    _check_moments(S[200:], m, Cov)


def _features(o, prob, woff, width):
    """Output-layer features of the frozen MLP from the oracle's forward pass: with the
    output weights set to a unit vector and the output bias to 0, F(x) is one feature."""
    feats = []
    for j in range(width):
        th = prob.frozen.copy()
        th[woff:woff + width] = 0.0
        th[woff + j] = 1.0
        th[-1] = 0.0
        feats.append(o.forward(th)[:, 0])
    return np.stack(feats, axis=1)


def _output_layer_problem(chains=32, n_out=6):
    """MLP 2-64-64-1 (tanh) sampling n_out output weights and the output bias.  The units
    are picked greedily for a well-conditioned posterior (the ratio of its largest to
    smallest standard deviation stays near 10), so that a modest number of
    trajectories mixes every direction."""
    base = W.mlp_fanin(n=256, widths=(2, 64, 64, 1), chains=chains, noise=0.1, seed=9191)
    P = base.P
    woff = P - 1 - 64                                    # output weights [1][64], then the output bias
    o = oracle.Oracle(W.with_subset(base, np.eye(P, dtype=np.uint8)[P - 1], chains=2))
    X = _features(o, base, woff, 64)
    ones = np.ones((X.shape[0], 1))
    chosen = []
    for _ in range(n_out):
        best = None
        for j in range(64):
            if j in chosen:
                continue
            Xs = np.concatenate([X[:, chosen + [j]], ones], axis=1)
            ev = np.linalg.eigvalsh(Xs.T @ Xs / base.noise_sigma ** 2 + np.eye(len(chosen) + 2))
            if best is None or ev.max() / ev.min() < best[0]:
                best = (ev.max() / ev.min(), j)
        chosen.append(best[1])
    mask = np.zeros(P, dtype=np.uint8)
    mask[[woff + j for j in chosen]] = 1
    mask[P - 1] = 1
    prob = W.with_subset(base, mask, chains=chains)
    cols = np.zeros(65, dtype=np.uint8)
    cols[sorted(chosen)] = 1
    cols[64] = 1
    Xa = np.concatenate([X, ones], axis=1)               # [n][65]: the 64 features, then the bias
    fro = np.concatenate([prob.frozen[woff:woff + 64], prob.frozen[-1:]])
    m, Cov = _linear_closed_form(Xa, prob.y[:, 0], cols, fro, prob.noise_sigma, prob.prior_sigma)
    return prob, m, Cov


def test_output_layer_features_vanish_with_the_output_weights():
    # the feature construction's premise: with zero output weights and bias, F = 0
    prob, _, _ = _output_layer_problem(chains=2)
    th = prob.frozen.copy()
    th[prob.P - 1 - 64:] = 0.0
    assert np.allclose(oracle.Oracle(prob).forward(th), 0.0)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tensor_core_output_layer_posterior_is_the_closed_form(prec):
    prob, m, Cov = _output_layer_problem()
    ev = np.linalg.eigvalsh(Cov)
    sd_min, sd_max = np.sqrt(ev.min()), np.sqrt(ev.max())
    eps = 0.5 * sd_min
    L = int(np.ceil(1.5 * sd_max / eps))
    s = sampler_from(prob, hmc.PREC_BF16 if prec == "bf16" else hmc.PREC_FP16)
    S = _gpu_chains(s, prob.q0, eps, _lengths(L, 25, 2), 40, seed=9)
    _check_moments(S[200:], m, Cov)


def _hidden_subset_problem():
    # the problem of tests/golden/make_hidden_subset_moments.py (which wrote the fixture)
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_hidden_subset_moments", os.path.join(GOLDEN, "make_hidden_subset_moments.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.problem()


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_tensor_core_chains_match_long_oracle_chains(prec):
    # a subset reaching into the hidden layers (four hidden-layer and four output weights):
    # no closed form, so the reference is the moments of long FP64 oracle chains stored in
    # tests/golden/hidden_subset_moments.json; the GPU chains start from the oracle's
    # warmed-up states with its step, and their means and variances agree within both
    # estimates' Monte Carlo error
    with open(os.path.join(GOLDEN, "hidden_subset_moments.json")) as f:
        ref = json.load(f)
    prob = _hidden_subset_problem()
    k = prob.k
    assert k == ref["k"]
    s = sampler_from(prob, hmc.PREC_BF16 if prec == "bf16" else hmc.PREC_FP16)
    Sg = _gpu_chains(s, np.array(ref["warm_states"]), ref["eps"], _lengths(ref["L0"], 30, 4), 100, seed=4)[500:]
    assert np.all(np.isfinite(Sg))
    eg = _ess(Sg)
    mg, vg = Sg.reshape(-1, k).mean(0), Sg.reshape(-1, k).var(0)
    mo, vo = np.array(ref["mean"]), np.array(ref["var"])
    z = (mg - mo) / np.sqrt(np.array(ref["mean_se"]) ** 2 + vg / eg)
    assert np.all(np.abs(z) < 4.5), (z, eg.min())
    # the variance estimate's standard error: var * sqrt(2 / ESS) to first order (Gaussian)
    zv = (vg - vo) / np.sqrt(np.array(ref["var_se"]) ** 2 + 2 * vg ** 2 / eg)
    assert np.all(np.abs(zv) < 4.5), (zv, eg.min())
