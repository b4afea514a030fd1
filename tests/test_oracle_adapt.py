"""Pins of the oracle's dual-averaging step-size adaptation (oracle/adapt.py), CPU only.

The recursion (Hoffman and Gelman 2014, Sec. 3.2, the reading taken for the paper's
tuning to about 80% acceptance in Sec. 4.2.3) is checked against what it must do
independently of how it is written: the closed form of its running average under a
constant acceptance statistic, its fixed point when every trajectory meets the target,
the hand-computed statistic of a few energy errors, and convergence of the averaged
step to the root of a monotone acceptance curve.
"""
import math

import numpy as np
import pytest

from oracle import adapt


def test_accept_stat_by_hand():
    dH = [0.0, math.log(2.0), -1.0, float("nan"), float("inf"), float("-inf")]
    # min(1, e^-dH): 1, 1/2, 1, then 0 for each non-finite value
    assert adapt.accept_stat(dH) == pytest.approx(2.5 / 6.0, rel=0, abs=1e-15)


@pytest.mark.parametrize("a", [0.0, 0.3, 0.8, 0.95, 1.0])
def test_constant_statistic_closed_form(a):
    # with a_m = a for all m, (m + t0) Hbar_m = (m - 1 + t0) Hbar_{m-1} + (delta - a), so
    # Hbar_m = m (delta - a) / (m + t0) and log eps_m = mu - sqrt(m) / gamma * Hbar_m
    eps0, delta, n = 3e-4, 0.8, 200
    tr = adapt.dual_averaging([a] * n, eps0, delta)
    mu = math.log(10 * eps0)
    lbar = 0.0
    for m in range(1, n + 1):
        hbar = m * (delta - a) / (m + adapt.T0)
        le = mu - math.sqrt(m) / adapt.GAMMA * hbar
        assert math.log(tr[m - 1, 0]) == pytest.approx(le, rel=1e-12, abs=1e-12)
        eta = m ** -adapt.KAPPA
        lbar = eta * le + (1 - eta) * lbar
        assert math.log(tr[m - 1, 1]) == pytest.approx(lbar, rel=1e-12, abs=1e-12)


def test_target_met_keeps_the_shrinkage_point():
    # a statistic equal to the target leaves Hbar at 0: every step is exp(mu) = 10 eps0
    tr = adapt.dual_averaging([0.65] * 50, 2e-3, 0.65)
    assert np.allclose(tr, 2e-2, rtol=1e-14, atol=0)


@pytest.mark.parametrize("target", [0.6, 0.8, 0.9])
def test_averaged_step_converges_to_the_root(target):
    # a monotone acceptance curve a(eps) = exp(-(eps / s)^2) has the root
    # eps* = s sqrt(ln(1 / target)); the averaged step must approach it
    s = 1e-3
    root = s * math.sqrt(math.log(1.0 / target))
    da = adapt.DualAveraging(1e-4, target)
    eps = 1e-4
    for _ in range(4000):
        eps, ebar = da.update(math.exp(-(eps / s) ** 2))
    assert ebar == pytest.approx(root, rel=0.03)


def test_incremental_and_batch_forms_agree():
    rng = np.random.default_rng(5)
    stats = rng.uniform(0, 1, 300)
    da = adapt.DualAveraging(1e-3, 0.7)
    inc = np.array([da.update(a) for a in stats])
    assert np.array_equal(inc, adapt.dual_averaging(stats, 1e-3, 0.7))
