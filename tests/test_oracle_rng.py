"""Pins for the oracle's counter-based momenta (CPU only).

* Philox4x64-10 against numpy's independent Philox bit generator (library pin).
* The series log and sin/cos against mpmath at 50 digits (closed form).
* The Box-Muller Gaussians against N(0, 1) (moments, KS) and block independence.
"""
import numpy as np
import pytest

import oracle


def test_philox_matches_numpy_bit_generator():
    rng = np.random.default_rng(11)
    cases = [([0, 0, 0, 0], [0, 0]), ([2**64 - 1] * 4, [2**64 - 1] * 2)]
    cases += [(list(rng.integers(0, 2**63, 4)), list(rng.integers(0, 2**63, 2))) for _ in range(20)]
    for ctr, key in cases:
        ctr = [int(c) for c in ctr]
        key = [int(k) for k in key]
        # numpy advances its counter by one before each block
        prev = [(ctr[0] - 1) % 2**64] + ctr[1:]
        carry = ctr[0] == 0
        for i in range(1, 4):
            if not carry:
                break
            prev[i] = (ctr[i] - 1) % 2**64
            carry = ctr[i] == 0
        bg = np.random.Philox(counter=prev, key=key)
        want = bg.random_raw(4).astype(np.uint64)
        got = oracle.philox4x64_10(ctr, key)
        assert np.array_equal(got, want), (ctr, key)


def test_unit_uniform_range():
    assert oracle.unit_uniform(0) == 2.0**-53
    assert oracle.unit_uniform(2**64 - 1) == 1.0
    assert oracle.unit_uniform(1 << 63) == 0.5 + 2.0**-53


def test_series_log_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(5)
    xs = list(rng.uniform(0.0, 1.0, 3000)) + list(10.0 ** rng.uniform(-300, 300, 500))
    xs += [2.0**-53, 1.0, 0.5, 0.70710678118654752, 0.7071067811865476, 2.0, 2.2250738585072014e-308]
    worst = 0.0
    for x in xs:
        ref = mp.log(mp.mpf(x))
        got = oracle.log(x)
        err = abs(mp.mpf(got) - ref)
        scale = max(abs(ref), mp.mpf(1e-300))
        worst = max(worst, float(err / scale))
        # absolute bound near x = 1 where log x -> 0
        assert float(err) <= 4e-16 * max(float(abs(ref)), 1e-300) or float(err) < 2e-17, x
    assert worst < 4e-16


def test_series_sincos_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(6)
    ms = [1, 2**50, 2**51, 2**51 + 2**50, 2**52, 3 * 2**51, 2**53, 2**53 - 1]
    ms += [int(m) for m in rng.integers(1, 2**53 + 1, 3000, dtype=np.uint64)]
    for m in ms:
        ang = 2 * mp.pi * mp.mpf(m) / mp.mpf(2**53)
        s, c = oracle.sincos_2pi(m)
        assert abs(mp.mpf(s) - mp.sin(ang)) < 4e-16, m
        assert abs(mp.mpf(c) - mp.cos(ang)) < 4e-16, m


def test_momenta_are_standard_normal():
    from scipy import stats
    z = np.concatenate([oracle.momenta(seed=3, chain=c, traj=t, k=1000) for c in range(4) for t in range(25)])
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # kurtosis of a Gaussian is 3
    assert abs(np.mean(z**4) - 3.0) < 0.15


def test_momenta_independent_across_components_chains_and_trajectories():
    a = oracle.momenta(seed=9, chain=0, traj=0, k=4000)
    b = oracle.momenta(seed=9, chain=1, traj=0, k=4000)
    c = oracle.momenta(seed=9, chain=0, traj=1, k=4000)
    d = oracle.momenta(seed=10, chain=0, traj=0, k=4000)
    for u, v in [(a, b), (a, c), (a, d), (a[0::2], a[1::2]), (a[0::4], a[2::4])]:
        r = np.corrcoef(u, v)[0, 1]
        assert abs(r) < 5.0 / np.sqrt(u.size)
    # counter-based: the same (seed, chain, traj, j) always gives the same value
    assert np.array_equal(a, oracle.momenta(seed=9, chain=0, traj=0, k=4000))
    # component j of a longer vector equals component j of a shorter one
    assert np.array_equal(a[:7], oracle.momenta(seed=9, chain=0, traj=0, k=7))


def test_mh_uniform_is_uniform():
    from scipy import stats
    u = np.array([oracle.mh_uniform(4, c, t) for c in range(20) for t in range(500)])
    assert u.min() > 0.0 and u.max() <= 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
