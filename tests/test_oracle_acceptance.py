"""The paper's qualitative observation on subset HMC, checked on the oracle (CPU only):
at a fixed step size the acceptance rate does not fall when fewer parameters are
sampled (the cost table of Sec. 4.2.3 and the tau sweep of App. E, where smaller subsets
accept more).  The Sec. 4.2.3 discussion of that table puts this down to the smaller error the leapfrog
accumulates in fewer dimensions; Sec. 3.3 gives only the cost side of the same fact
(drawing an independent sample costs about D^(5/4)).

Nested subsets (5% inside 30% inside all 481 parameters of the tiny BNN) keep the
comparison like for like: the conditional posterior of a sub-block is lower-dimensional,
and for a Gaussian posterior it is no stiffer (a principal submatrix's largest eigenvalue
is bounded by the full Hessian's), so the leapfrog's energy error shrinks with it.  Seeded,
so the rates are fixed numbers; the margins
allow for the Monte Carlo error of 480 post-burn-in trajectories per subset.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W


def _nested(base, frac, order, chains):
    m = np.zeros(base.P, dtype=np.uint8)
    m[order[:int(round(frac * base.P))]] = 1
    q0 = np.repeat(base.frozen[m.astype(bool)][None, :], chains, axis=0)
    return dataclasses.replace(base, mask=m, q0=q0)


@pytest.mark.parametrize("eps", [1.5e-3, 2e-3])
def test_acceptance_does_not_fall_as_the_subset_shrinks(eps):
    chains = 4
    base = W.tiny_bnn(n=256, chains=chains)
    order = np.argsort(np.random.default_rng(5).random(base.P))
    rates = []
    for frac in (1.0, 0.3, 0.05):
        prob = _nested(base, frac, order, chains)
        _, acc, _, _ = oracle.Oracle(prob).sample(prob.q0, eps=eps, L=20, n=150, seed=11, threads=chains)
        rates.append(float(acc[30:].mean()))
    full, part, small = rates
    assert part >= full - 0.03 and small >= part - 0.03, rates
    assert small >= full + 0.05, rates        # the effect itself, not only its sign
    assert small > 0.95, rates
