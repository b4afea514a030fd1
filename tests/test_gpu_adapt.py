"""Step-size warm-up on the GPU (hmc_adapt_step_size) against the oracle's restatement
of dual averaging (oracle/adapt.py; Hoffman and Gelman 2014, Sec. 3.2, the reading taken
for the paper's tuning to about 80% acceptance, Sec. 4.2.3).

* The device update, fed the same seeded energy errors as the restatement, gives the
  same step sequence to 1e-12.
* A whole FP64 warm-up gives the step sequence of the oracle's own warm-up (its
  trajectories, its updates) to 1e-8 over its first 15 updates (later updates amplify
  rounding differences, see the test).
* The warm-up replays one captured trajectory graph: a new step size captures nothing.
* In a batch every problem adapts its own step from its own chains' acceptance, each
  following the oracle's warm-up of that problem alone; sampling with a step per
  problem (hmc_sample_steps) follows the oracle's chains of each problem at its step.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import sampler_from
from oracle import adapt

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nseg", [1, 16, 300])
def test_device_update_matches_the_restatement(nseg):
    rng = np.random.default_rng(100 + nseg)
    n = 120
    dH = rng.normal(0.3, 1.0, (n, nseg)) * rng.choice([0.01, 1.0, 5.0], (n, 1))
    dH[rng.uniform(size=dH.shape) < 0.02] = np.nan
    dH[rng.uniform(size=dH.shape) < 0.01] = np.inf
    dH[rng.uniform(size=dH.shape) < 0.01] = -np.inf
    for eps0, target in ((1e-3, 0.8), (0.2, 0.65)):
        got = hmc.diag_dual_averaging(dH, eps0, target)
        ref = adapt.dual_averaging_dH(dH, eps0, target)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("case", ["bayes_linear", "small_mlp"])
def test_fp64_warmup_matches_the_oracle_warmup(case):
    prob = {"bayes_linear": lambda: W.bayes_linear(chains=4),
            "small_mlp": lambda: W.small_mlp(n=120, widths=(2, 12, 9, 1), frac=0.6, chains=3, seed=8)}[case]()
    # dual averaging feeds every step back into the next trajectory's acceptance, and early
    # on (large sqrt(m) / gamma) it amplifies a difference several times per update, so two
    # correct implementations agree to rounding only over the first updates: 15 of them here
    L, n, eps0, seed, first = 8, 15, 0.02 if case == "bayes_linear" else 3e-3, 31, 5
    s = sampler_from(prob, hmc.PREC_FP64)
    eps, q = s.adapt_step_size(torch.from_numpy(prob.q0), L, eps0, n, target_accept=0.8, seed=seed,
                               first_traj=first)
    tr = hmc.adapt_trace(s, n)
    tr_o, q_o = adapt.warmup(oracle.Oracle(prob), prob.q0, L, eps0, n, 0.8, seed, first)
    np.testing.assert_allclose(tr, tr_o, rtol=1e-8, atol=0)
    assert eps == pytest.approx(tr_o[-1, 1], rel=1e-8)
    np.testing.assert_allclose(q.cpu().numpy(), q_o, rtol=1e-8, atol=1e-11)


def test_warmup_and_new_step_sizes_capture_no_new_graph():
    prob = W.small_mlp(n=200, widths=(2, 64, 64, 1), frac=0.2, chains=2, seed=3)
    s = sampler_from(prob, hmc.PREC_FP32)
    q0 = torch.from_numpy(prob.q0)
    s.sample(q0, 1e-3, 6, 2, seed=4)
    n0 = hmc.graph_captures(s)
    eps, q = s.adapt_step_size(q0, 6, 1e-3, 25, seed=4, first_traj=10)
    s.sample(q, 0.5 * eps, 6, 2, seed=4, first_traj=35)
    s.sample(q, 2.0 * eps, 6, 2, seed=4, first_traj=37)
    assert hmc.graph_captures(s) == n0
    s.sample(q, eps, 7, 1, seed=4)          # a new L is a new graph
    assert hmc.graph_captures(s) == n0 + 1


def _batch_problems():
    return [W.small_mlp(n=90, widths=(2, 10, 8, 1), frac=0.6, chains=3, seed=41),
            W.small_mlp(n=150, widths=(3, 7, 7, 1), frac=0.5, chains=3, seed=42, noise=0.05),
            W.small_mlp(n=60, widths=(1, 12, 1), frac=0.8, chains=3, seed=43)]


def _batch(probs, prec):
    tup = [(p.net.widths, p.x, p.y, p.mask, p.frozen, p.prior_sigma, p.noise_sigma) for p in probs]
    return hmc.BatchSampler(tup, probs[0].chains, prec)


def test_batch_warmup_adapts_each_problem_on_its_own():
    probs = _batch_problems()
    s = _batch(probs, hmc.PREC_FP64)
    L, n, eps0, seed, first = 8, 15, 3e-3, 17, 2
    q0 = np.concatenate([p.q0.reshape(-1) for p in probs])
    eps, q = s.adapt_step_size(torch.from_numpy(q0), L, eps0, n, target_accept=0.8, seed=seed, first_traj=first)
    tr = hmc.adapt_trace(s, n)
    assert eps.shape == (3,) and tr.shape == (n, 3, 2)
    off = 0
    for i, p in enumerate(probs):
        tr_o, q_o = adapt.warmup(oracle.Oracle(p), p.q0, L, eps0, n, 0.8, seed, first, problem=i)
        np.testing.assert_allclose(tr[:, i, :], tr_o, rtol=1e-8, atol=0)
        assert eps[i] == pytest.approx(tr_o[-1, 1], rel=1e-8)
        size = p.q0.size
        np.testing.assert_allclose(q.cpu().numpy()[off:off + size].reshape(p.q0.shape), q_o, rtol=1e-8, atol=1e-11)
        off += size


def test_batch_sample_with_a_step_per_problem():
    probs = _batch_problems()
    s = _batch(probs, hmc.PREC_FP64)
    eps = np.array([2e-3, 5e-4, 4e-3])
    n, L, seed = 4, 6, 23
    q0 = np.concatenate([p.q0.reshape(-1) for p in probs])
    S, acc, dH, ql = s.sample(torch.from_numpy(q0), eps, L, n, seed=seed, first_traj=3)
    dH = dH.cpu().numpy()
    ql = ql.cpu().numpy()
    C, off = probs[0].chains, 0
    for i, p in enumerate(probs):
        _, accr, dHr, qlr = oracle.Oracle(p).sample(p.q0, eps[i], L, n, seed=seed, first_traj=3, problem=i)
        np.testing.assert_allclose(dH[:, i * C:(i + 1) * C], dHr, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(ql[off:off + p.q0.size].reshape(p.q0.shape), qlr, rtol=1e-8, atol=1e-10)
        off += p.q0.size
    with pytest.raises(ValueError):
        s.sample(torch.from_numpy(q0), eps[:2], L, 1)
    with pytest.raises(hmc.HmcError):
        s.sample(torch.from_numpy(q0), np.array([1e-3, -1.0, 1e-3]), L, 1)
