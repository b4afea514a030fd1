"""Write hidden_subset_moments.json: posterior moments of a subset that reaches into the
hidden layers of a tanh MLP, from long FP64 oracle chains.

The problem has no closed form, so the reference for the GPU samplers' chains is the
oracle's own sampler (Algorithm 1 on the subset, as in Algorithm 2), run long: the step
from the oracle's dual-averaging warm-up, then 16 chains of blocks of 100 trajectories
whose leapfrog lengths vary between blocks (a fixed length can sit near a multiple of a
half-period of some posterior direction).  Only oracle/ and workloads/ are used.
Run from the repository root:  python tests/golden/make_hidden_subset_moments.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
import workloads as W  # noqa: E402
from oracle import adapt  # noqa: E402
from oracle.ess import ess_chains  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hidden_subset_moments.json")


def problem():
    """1-64-64-1 tanh MLP on 128 points; four weights of the hidden 64 x 64 layer and four
    output weights are sampled (the subset is seeded)."""
    base = W.mlp_fanin(n=128, widths=(1, 64, 64, 1), chains=16, noise=0.1, seed=5151)
    rng = np.random.default_rng(1)
    (w1, _), (w2, _) = base.net.layer_slices()[1], base.net.layer_slices()[2]
    mask = np.zeros(base.P, dtype=np.uint8)
    mask[w1 + rng.choice(64 * 64, 4, replace=False)] = 1
    mask[w2 + rng.choice(64, 4, replace=False)] = 1
    return W.with_subset(base, mask, chains=16)


def lengths(L0, blocks, seed):
    return np.random.default_rng(seed).integers(L0 // 2, 3 * L0 // 2 + 1, blocks)


def main():
    prob = problem()
    o = oracle.Oracle(prob)
    L0, per, blocks, burn = 20, 100, 40, 500
    tr, qw = adapt.warmup(o, prob.q0, L0, 1e-3, 150, 0.8, seed=2, first_traj=0)
    eps = float(tr[-1, 1])
    q, S = qw, []
    for i, L in enumerate(lengths(L0, blocks, 11)):
        Si, _, _, q = o.sample(q, eps, int(L), per, seed=3, first_traj=1000 + i * per, threads=os.cpu_count())
        S.append(Si)
    S = np.concatenate(S)[burn:]
    n, C, k = S.shape
    ess = np.minimum(ess_chains(S), n * C)
    flat = S.reshape(-1, k)
    mean, var = flat.mean(0), flat.var(0)
    rec = {"problem": "workloads.mlp_fanin(n=128, widths=(1, 64, 64, 1), noise=0.1, seed=5151), subset as in "
                      "problem() of this script",
           "k": int(k), "eps": eps, "L0": L0, "warm_states": qw.tolist(),
           "draws_per_chain": int(n), "chains": int(C),
           "mean": mean.tolist(), "var": var.tolist(), "ess": ess.tolist(),
           "mean_se": np.sqrt(var / ess).tolist(), "var_se": np.sqrt(2.0 * var ** 2 / ess).tolist(),
           "between_over_within_sd": (S.mean(0).std(0) / np.sqrt(var)).tolist()}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print("wrote", OUT, "ess min", ess.min(), "btw/within max", max(rec["between_over_within_sd"]))


if __name__ == "__main__":
    main()
