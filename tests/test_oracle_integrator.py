"""Pins for the oracle's leapfrog integrator (CPU only).

* Harmonic oscillator (no data, U = |q|^2/(2 alpha^2)): L leapfrog steps equal the
  L-th power of the one-step 2x2 kick-drift-kick matrix.
* Energy error of a fixed-length trajectory shrinks as eps^2.
* Time reversibility: integrate, negate p, integrate, negate p returns the start.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def test_harmonic_oscillator_closed_form():
    for eps, L, alpha in [(0.1, 13, 0.7), (0.37, 5, 1.3), (0.01, 100, 1.0)]:
        prob = W.harmonic(k=6, prior=alpha, eps=eps, L=L)
        o = oracle.Oracle(prob)
        rng = np.random.default_rng(1)
        q = rng.standard_normal(prob.k)
        p = rng.standard_normal(prob.k)
        w2 = 1.0 / alpha**2
        M = np.array([[1 - eps**2 * w2 / 2, eps],
                      [-eps * w2 * (1 - eps**2 * w2 / 4), 1 - eps**2 * w2 / 2]])
        ML = np.linalg.matrix_power(M, L)
        qe = ML[0, 0] * q + ML[0, 1] * p
        pe = ML[1, 0] * q + ML[1, 1] * p
        q1, p1, U1, g1 = o.leapfrog(q, p, eps, L)
        assert np.allclose(q1, qe, rtol=1e-13, atol=1e-13)
        assert np.allclose(p1, pe, rtol=1e-13, atol=1e-13)
        assert np.isclose(U1, 0.5 * w2 * np.sum(q1 * q1), rtol=1e-13)
        assert np.allclose(g1, w2 * q1, rtol=1e-13)


def _dH(o, q, p, eps, L):
    U0, g0 = o.energy_grad(q)
    H0 = U0 + 0.5 * p @ p
    q1, p1, U1, _ = o.leapfrog(q, p, eps, L, U0, g0)
    return (U1 + 0.5 * p1 @ p1) - H0


@pytest.mark.parametrize("which", ["tiny_bnn", "linear", "deeponet"])
def test_energy_error_is_second_order(which):
    if which == "tiny_bnn":
        prob = W.tiny_bnn(n=64)
        T, eps0 = 2e-3, 1e-4
    elif which == "linear":
        prob = W.bayes_linear()
        T, eps0 = 0.2, 0.02
    else:
        prob = W.small_deeponet()
        T, eps0 = 4e-3, 4e-4
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(2)
    q = prob.q0[0]
    p = rng.standard_normal(prob.k)
    errs = []
    for m in (1, 2, 4):
        eps = eps0 / m
        L = int(round(T / eps))
        errs.append(abs(_dH(o, q, p, eps, L)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.2 < r1 < 4.8, errs
    assert 3.2 < r2 < 4.8, errs


@pytest.mark.parametrize("which", ["tiny_bnn", "deeponet", "small_mlp"])
def test_time_reversibility(which):
    prob = {"tiny_bnn": lambda: W.tiny_bnn(n=64), "deeponet": W.small_deeponet,
            "small_mlp": W.small_mlp}[which]()
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(3)
    q0 = prob.q0[0].copy()
    p0 = rng.standard_normal(prob.k)
    eps, L = 2e-4, 15
    q1, p1, U1, g1 = o.leapfrog(q0, p0, eps, L)
    q2, p2, U2, g2 = o.leapfrog(q1, -p1, eps, L, U1, g1)
    p2 = -p2
    assert np.max(np.abs(q2 - q0)) <= 1e-10 * max(1.0, np.max(np.abs(q0)))
    assert np.max(np.abs(p2 - p0)) <= 1e-10 * max(1.0, np.max(np.abs(p0)))
    # and it actually moved
    assert np.max(np.abs(q1 - q0)) > 1e-6
