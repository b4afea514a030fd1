"""Pins for the oracle's U and grad U (CPU only).

* Central finite differences of U along random directions and single coordinates.
* torch.autograd in float64 on the same flat parameter vector (library pin for the
  forward pass, the parameter layout and the reverse pass).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W


def _problems():
    out = [
        W.small_mlp(),
        W.small_mlp(widths=(2, 17, 1), acts=[W.ACT_SIN, W.ACT_IDENTITY], frac=0.6, seed=1),
        W.small_mlp(widths=(4, 9, 9, 3), acts=[W.ACT_TANH, W.ACT_SIN, W.ACT_TANH],
                    bias=[True, False, True], frac=0.5, seed=2),
        W.small_mlp(widths=(1, 8, 8, 1), frac=1.0, seed=3),
        W.small_deeponet(),
        W.small_deeponet(out_bias=False, frac=0.5, seed=4),
        W.tiny_bnn(n=40),
        W.small_deeponet_unaligned(),
        W.small_deeponet_unaligned(out_bias=False, n_q=5, seed=5),
    ]
    return out


def _fd_directional(o, q, v, h):
    return (o.energy(q + h * v) - o.energy(q - h * v)) / (2.0 * h)


@pytest.mark.parametrize("pi", range(9))
def test_gradient_matches_central_differences(pi):
    prob = _problems()[pi]
    o = oracle.Oracle(prob)
    rng = np.random.default_rng(100 + pi)
    q = prob.q0[0] + 0.05 * rng.standard_normal(prob.k)
    U, g = o.energy_grad(q)
    assert np.isfinite(U)
    for _ in range(4):
        v = rng.standard_normal(prob.k)
        v /= np.linalg.norm(v)
        fd = _fd_directional(o, q, v, 1e-5)
        an = float(g @ v)
        assert abs(fd - an) <= 1e-7 * max(1.0, np.linalg.norm(g)), (fd, an)
    for j in rng.choice(prob.k, size=min(prob.k, 25), replace=False):
        e = np.zeros(prob.k)
        e[j] = 1.0
        h = 1e-5 * max(1.0, abs(q[j]))
        fd = _fd_directional(o, q, e, h)
        # truncation O(h^2) plus the rounding of two evaluations of U, over 2h
        tol = 1e-6 * max(1.0, abs(g[j])) + 8.0 * np.finfo(float).eps * abs(U) / h
        assert abs(fd - g[j]) <= tol, (j, fd, g[j])


def _torch_net(nt, theta, x, base=0):
    off = base
    a = x
    for l in range(nt.n_layers):
        wi, wo = nt.widths[l], nt.widths[l + 1]
        Wm = theta[off:off + wo * wi].reshape(wo, wi)
        off += wo * wi
        b = None
        if nt.bias[l]:
            b = theta[off:off + wo]
            off += wo
        z = torch.nn.functional.linear(a, Wm, b)
        act = nt.act[l]
        a = torch.tanh(z) if act == W.ACT_TANH else torch.sin(z) if act == W.ACT_SIN else z
    return a, off


def _torch_energy(prob, q):
    theta = torch.tensor(prob.frozen, dtype=torch.float64)
    qt = torch.tensor(q, dtype=torch.float64, requires_grad=True)
    theta = theta.index_put((torch.tensor(prob.idx),), qt)
    if prob.kind == W.KIND_MLP:
        f, _ = _torch_net(prob.net, theta, torch.tensor(prob.x))
        r = f - torch.tensor(prob.y)
    elif prob.kind == W.KIND_DEEPONET:
        B, off = _torch_net(prob.branch, theta, torch.tensor(prob.u))
        T, off = _torch_net(prob.trunk, theta, torch.tensor(prob.yq), base=off)
        S = B @ T.T
        if prob.out_bias:
            S = S + theta[off]
        r = S - torch.tensor(prob.t)
    else:   # every input function with its own queries
        B, off = _torch_net(prob.branch, theta, torch.tensor(prob.u))
        T, off = _torch_net(prob.trunk, theta, torch.tensor(prob.yq), base=off)   # [n_u][n_q][p]
        S = torch.einsum("ic,ijc->ij", B, T)
        if prob.out_bias:
            S = S + theta[off]
        r = S - torch.tensor(prob.t)
    U = (r * r).sum() / (2 * prob.noise_sigma**2) + (qt * qt).sum() / (2 * prob.prior_sigma**2)
    U.backward()
    return float(U), qt.grad.numpy()


@pytest.mark.parametrize("pi", range(9))
def test_energy_and_gradient_match_torch_autograd(pi):
    prob = _problems()[pi]
    o = oracle.Oracle(prob)
    q = prob.q0[-1]
    U, g = o.energy_grad(q)
    Ut, gt = _torch_energy(prob, q)
    assert abs(U - Ut) <= 1e-11 * abs(Ut)
    assert np.max(np.abs(g - gt)) <= 1e-10 * max(1.0, np.max(np.abs(gt)))


def test_forward_matches_torch_for_full_theta():
    for prob in (W.small_mlp(), W.small_deeponet()):
        o = oracle.Oracle(prob)
        theta = prob.frozen
        f = o.forward(theta)
        th = torch.tensor(theta)
        if prob.kind == W.KIND_MLP:
            ft, _ = _torch_net(prob.net, th, torch.tensor(prob.x))
        else:
            B, off = _torch_net(prob.branch, th, torch.tensor(prob.u))
            T, off = _torch_net(prob.trunk, th, torch.tensor(prob.yq), base=off)
            ft = B @ T.T + (th[off] if prob.out_bias else 0.0)
        assert np.allclose(f, ft.numpy(), rtol=1e-12, atol=1e-12)


def test_prior_only_when_no_data():
    prob = W.harmonic(k=5, prior=0.7)
    o = oracle.Oracle(prob)
    q = prob.q0[0]
    U, g = o.energy_grad(q)
    # with no data terms the energy is the alpha-Gaussian prior alone
    assert np.isclose(U, 0.5 * np.sum(q * q) / 0.49, rtol=1e-14)
    assert np.allclose(g, q / 0.49, rtol=1e-14)


def test_deeponet_without_functions_or_queries_is_the_prior():
    import dataclasses
    base = W.small_deeponet(frac=0.2, chains=1)
    q = base.q0[0]
    prior = 0.5 * np.sum(q * q) / base.prior_sigma**2
    for empty in ({"u": np.zeros((0, base.u.shape[1])), "t": np.zeros((0, base.t.shape[1]))},
                  {"yq": np.zeros((0, base.yq.shape[1])), "t": np.zeros((base.t.shape[0], 0))}):
        o = oracle.Oracle(dataclasses.replace(base, **empty))
        U, g = o.energy_grad(q)
        assert np.isclose(U, prior, rtol=1e-14)
        assert np.allclose(g, q / base.prior_sigma**2, rtol=1e-14)


def test_frozen_parameters_enter_only_through_the_likelihood():
    prob = W.small_mlp(frac=0.3)
    o = oracle.Oracle(prob)
    q = prob.q0[0]
    U1 = o.energy(q)
    # changing a frozen value changes U (it is part of the network) ...
    off = np.flatnonzero(prob.mask == 0)[3]
    prob2 = W.small_mlp(frac=0.3)
    prob2.frozen = prob2.frozen.copy()
    prob2.frozen[off] += 0.5
    U2 = oracle.Oracle(prob2).energy(q)
    assert U1 != U2
    # ... but adds no prior term: with no data, only the subset's prior remains
    h = W.harmonic(k=6)
    h.mask = np.array([1, 0, 1, 0, 1, 1], dtype=np.uint8)
    h.q0 = h.q0[:, h.mask.astype(bool)] if h.q0.shape[1] == 6 else h.q0
    oh = oracle.Oracle(h)
    qh = np.array([0.3, -0.2, 0.5, 1.0])
    assert np.isclose(oh.energy(qh), np.sum(qh**2) / (2 * h.prior_sigma**2), rtol=1e-14)


def test_unaligned_deeponet_with_shared_queries_is_the_aligned_one():
    # every function given the same query set: the per-function layout must give the
    # aligned problem's U exactly and its gradient up to summation order
    pu = W.small_deeponet_unaligned(shared=True)
    pa = W.Problem("aligned", W.KIND_DEEPONET, pu.noise_sigma, pu.prior_sigma, pu.frozen, pu.mask, pu.q0,
                   eps=pu.eps, L=pu.L, branch=pu.branch, trunk=pu.trunk, out_bias=pu.out_bias,
                   u=pu.u, yq=pu.yq[0], t=pu.t)
    ou, oa = oracle.Oracle(pu), oracle.Oracle(pa)
    for q in pu.q0:
        Uu, gu = ou.energy_grad(q)
        Ua, ga = oa.energy_grad(q)
        assert Uu == Ua
        assert np.allclose(gu, ga, rtol=1e-12, atol=1e-12 * np.max(np.abs(ga)))
    assert np.array_equal(ou.forward(pu.frozen), oa.forward(pu.frozen))
