"""Pins for the oracle's posterior predictive and relative L2 error (Sec. 4.2.1), CPU only.

* One sample: the mean is that sample's forward pass and the spread is zero.
* Two samples: mean (f_a + f_b)/2 and standard deviation |f_a - f_b|/2.
* A model linear in its parameters: the predictive mean is the model at the mean
  sample and the variance is x^T Cov x with Cov the samples' covariance.
* The relative L2 error on hand-computed rows.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def _theta(prob, q):
    th = prob.frozen.copy()
    th[prob.idx] = q
    return th


@pytest.mark.parametrize("which", ["mlp", "deeponet"])
def test_one_and_two_samples(which):
    prob = W.small_mlp(n=40, widths=(3, 9, 2), seed=91) if which == "mlp" else \
        W.small_deeponet(n_u=6, n_y=5, seed=92)
    o = oracle.Oracle(prob)
    qa, qb = prob.q0[0], prob.q0[1]
    fa, fb = o.forward(_theta(prob, qa)), o.forward(_theta(prob, qb))
    m, s = o.predict(qa[None])
    assert np.array_equal(m, fa) and np.all(s == 0)
    m, s = o.predict(np.stack([qa, qb]))
    assert np.allclose(m, 0.5 * (fa + fb), rtol=1e-14, atol=1e-15)
    assert np.allclose(s, 0.5 * np.abs(fa - fb), rtol=1e-12, atol=1e-15)


def test_linear_model_moments():
    prob = W.bayes_linear(n=30, d=4)
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(4)
    Q = rng.standard_normal((200, prob.k))
    m, s = o.predict(Q)
    Xa = np.concatenate([prob.x, np.ones((prob.x.shape[0], 1))], axis=1)
    qbar = Q.mean(axis=0)
    cov = np.cov(Q.T, bias=True)
    assert np.allclose(m[:, 0], Xa @ qbar, rtol=1e-12, atol=1e-12)
    assert np.allclose(s[:, 0] ** 2, np.einsum("ni,ij,nj->n", Xa, cov, Xa), rtol=1e-10)


def test_rel_l2_hand_values():
    Y = np.array([[3.0, 4.0], [1.0, 0.0]])
    Yp = np.array([[3.0, 0.0], [0.0, 0.0]])
    assert oracle.rel_l2(Y, Yp) == pytest.approx(0.9, rel=1e-15)   # rows: 4/5 and 1/1
    assert oracle.rel_l2(Y, Y) == 0.0
    assert oracle.rel_l2(np.array([[2.0, 0.0, 0.0]]), np.array([[0.0, 0.0, 0.0]])) == 1.0
