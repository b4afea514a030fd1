"""Pins for the ESS estimator: i.i.d. draws and AR(1) chains, whose integrated
autocorrelation time (1 + rho) / (1 - rho) is known in closed form."""
import numpy as np

from oracle.ess import ess_geyer, ess_chains


def test_iid_ess_close_to_n():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000)
    assert 0.85 * 20000 < ess_geyer(x) < 1.15 * 20000


def test_ar1_ess_matches_closed_form():
    rng = np.random.default_rng(1)
    for rho in (0.5, 0.9, 0.97):
        n = 200000
        e = rng.standard_normal(n)
        x = np.empty(n)
        x[0] = e[0] / np.sqrt(1 - rho**2)
        for i in range(1, n):
            x[i] = rho * x[i - 1] + e[i]
        want = n * (1 - rho) / (1 + rho)
        got = ess_geyer(x)
        assert 0.8 * want < got < 1.2 * want, (rho, got, want)


def test_ess_sums_over_chains():
    rng = np.random.default_rng(2)
    S = rng.standard_normal((4000, 3, 2))
    e = ess_chains(S)
    assert e.shape == (2,)
    assert np.all(e > 0.8 * 12000) and np.all(e < 1.2 * 12000)
