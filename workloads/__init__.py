"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws data: network shapes, training sets, frozen parameter
vectors, subset masks and initial chain states.  It holds none of the sampler's
arithmetic (no energy, no gradient, no integrator, no random momenta), so both
the FP64 oracle and the CUDA path can take their inputs from here without
sharing any part of the method.

The paper's datasets (Burgers solutions, DNS cone wall pressure) and its
trained VI posteriors are not available; every generator below stands in for
them with seeded data of the same shape:

* ``tiny_bnn``        -- MLP 1-20-20-1 tanh, 256 points of y = sin(3x) + noise
                         (Sec. 4.1 style regression, all 481 parameters sampled).
* ``wide_mlp``        -- MLP 2-256-256-256-256-1 tanh, 8192 points of
                         y = sin(pi x1) cos(pi x2) + noise, 5% subset.
* ``deeponet_grf``    -- DeepONet, branch 100-128-128-128-64 on GRF sensor
                         values, trunk 2-128-128-128-64, 500 x 100 pairs, 10%
                         subset (shape of the Burgers operator example, Sec. 4.2.1).
* ``batched_uneven``  -- 64 independent 4-input MLPs of uneven width/depth/N.
* ``cone_deeponet``   -- DeepONet, branch 6-256-256-256-128, trunk
                         2-256-256-256-128, 2000 conditions x 8192 grid points
                         (shape of the cone wall-pressure example, Sec. 4.2.2).
* ``bayes_linear``    -- a linear model (MLP with no hidden layer, identity
                         output) whose posterior is Gaussian in closed form.

All floating-point data, frozen parameters and initial states are rounded to
values exactly representable in float32, so FP32 device code and the FP64
oracle start from bit-identical inputs.

Parameter order (shared convention, not arithmetic): for each Linear layer in
order, W[out][in] row-major, then b[out] if the layer has a bias.  A DeepONet
lists all branch layers, then all trunk layers, then the scalar output bias.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

ACT_IDENTITY, ACT_TANH, ACT_SIN = 0, 1, 2
KIND_MLP, KIND_DEEPONET, KIND_DEEPONET_UNALIGNED = 0, 1, 2


def _f32(a):
    """Round to the nearest float32 value, returned as float64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


@dataclass
class Net:
    """A feed-forward stack of Linear layers: widths[0] inputs ... widths[-1] outputs."""

    widths: List[int]
    act: List[int]
    bias: List[bool]

    @staticmethod
    def mlp(widths, hidden_act=ACT_TANH, last_act=ACT_IDENTITY, bias=True):
        n = len(widths) - 1
        acts = [hidden_act] * (n - 1) + [last_act]
        b = [bias] * n if isinstance(bias, bool) else list(bias)
        return Net(list(widths), acts, b)

    @property
    def n_layers(self):
        return len(self.widths) - 1

    def n_params(self):
        return sum(self.widths[l] * self.widths[l + 1] + (self.widths[l + 1] if self.bias[l] else 0)
                   for l in range(self.n_layers))

    def layer_slices(self, base=0):
        """(weight_offset, bias_offset or -1) per layer, in the shared parameter order."""
        out, off = [], base
        for l in range(self.n_layers):
            wi, wo = self.widths[l], self.widths[l + 1]
            woff = off
            off += wo * wi
            boff = -1
            if self.bias[l]:
                boff = off
                off += wo
            out.append((woff, boff))
        return out


@dataclass
class Problem:
    name: str
    kind: int
    noise_sigma: float
    prior_sigma: float
    frozen: np.ndarray          # [P] float64 (float32-representable)
    mask: np.ndarray            # [P] uint8, 1 = sampled
    q0: np.ndarray              # [C][k] float64
    eps: float
    L: int
    n_samples: int = 100
    seed: int = 0
    net: Optional[Net] = None           # MLP
    branch: Optional[Net] = None        # DeepONet
    trunk: Optional[Net] = None
    out_bias: bool = True
    x: Optional[np.ndarray] = None      # MLP inputs [n][dx]
    y: Optional[np.ndarray] = None      # MLP targets [n][dout]
    u: Optional[np.ndarray] = None      # DeepONet branch inputs [n_u][du]
    yq: Optional[np.ndarray] = None     # DeepONet trunk inputs [n_y][dy] ([n_u][n_y][dy] unaligned)
    t: Optional[np.ndarray] = None      # DeepONet targets [n_u][n_y]
    notes: dict = field(default_factory=dict)

    @property
    def chains(self):
        return self.q0.shape[0]

    @property
    def idx(self):
        return np.flatnonzero(self.mask).astype(np.int64)

    @property
    def k(self):
        return int(self.mask.sum())

    @property
    def P(self):
        return int(self.frozen.shape[0])

    def n_terms(self):
        """Number of data terms in the full-batch likelihood."""
        if self.kind == KIND_MLP:
            return int(self.x.shape[0]) * int(self.y.shape[1])
        return int(self.t.size)

    def with_chains(self, chains, seed=None):
        """Same problem, different number of chains (initial states redrawn)."""
        rng = np.random.default_rng(self.seed + 7919 if seed is None else seed)
        q0 = _initial_states(rng, self.frozen, self.mask, chains)
        p = Problem(**{**self.__dict__})
        p.q0 = q0
        return p


def deeponet_param_count(branch: Net, trunk: Net, out_bias=True):
    return branch.n_params() + trunk.n_params() + (1 if out_bias else 0)


def _subset_mask(rng, P, frac):
    """Top floor(frac*P) entries by a seeded |N(0,1)| score, ties to the lower index."""
    k = int(np.floor(frac * P))
    score = np.abs(rng.standard_normal(P))
    order = np.argsort(-score, kind="stable")
    mask = np.zeros(P, dtype=np.uint8)
    mask[order[:k]] = 1
    return mask


def _initial_states(rng, frozen, mask, chains, jitter=0.01):
    """Chain 0 starts at the frozen values on the subset; others add N(0, jitter^2)."""
    base = frozen[mask.astype(bool)]
    q0 = np.repeat(base[None, :], chains, axis=0)
    if chains > 1:
        q0[1:] += jitter * rng.standard_normal((chains - 1, base.size))
    return _f32(q0)


# --------------------------------------------------------------------------
# The five workloads
# --------------------------------------------------------------------------

def tiny_bnn(n=256, chains=1, n_samples=1000, seed=1001):
    """MLP 1-20-20-1 tanh, 481 parameters, all sampled; y = sin(3x) + N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    net = Net.mlp([1, 20, 20, 1])
    x = _f32(rng.uniform(-1.0, 1.0, size=(n, 1)))
    y = _f32(np.sin(3.0 * x) + 0.1 * rng.standard_normal((n, 1)))
    P = net.n_params()
    frozen = _f32(0.1 * rng.standard_normal(P))
    mask = np.ones(P, dtype=np.uint8)
    q0 = _initial_states(rng, frozen, mask, chains)
    return Problem("tiny_bnn", KIND_MLP, 0.1, 1.0, frozen, mask, q0, eps=1e-3, L=20,
                   n_samples=n_samples, seed=0, net=net, x=x, y=y)


def wide_mlp(n=8192, widths=(2, 256, 256, 256, 256, 1), frac=0.05, chains=16,
             eps=5e-4, L=50, seed=2002):
    """MLP 2-256-256-256-256-1 tanh; y = sin(pi x1) cos(pi x2) + N(0, 0.05^2); 5% subset."""
    rng = np.random.default_rng(seed)
    net = Net.mlp(list(widths))
    x = _f32(rng.uniform(-1.0, 1.0, size=(n, widths[0])))
    y = np.sin(np.pi * x[:, :1]) * np.cos(np.pi * x[:, 1:2]) if widths[0] >= 2 else np.sin(np.pi * x[:, :1])
    y = _f32(np.repeat(y, widths[-1], axis=1) + 0.05 * rng.standard_normal((n, widths[-1])))
    P = net.n_params()
    mask = _subset_mask(rng, P, frac)
    frozen = _f32(0.05 * rng.standard_normal(P))
    q0 = _initial_states(rng, frozen, mask, chains)
    return Problem("wide_mlp", KIND_MLP, 0.05, 1.0, frozen, mask, q0, eps=eps, L=L,
                   n_samples=200, seed=0, net=net, x=x, y=y)


def _grf_rows(rng, n_funcs, n_sensors, length=0.2):
    s = np.linspace(0.0, 1.0, n_sensors)
    K = np.exp(-(s[:, None] - s[None, :]) ** 2 / (2.0 * length ** 2))
    w, V = np.linalg.eigh(K + 1e-10 * np.eye(n_sensors))
    root = V * np.sqrt(np.clip(w, 0.0, None))[None, :]
    return rng.standard_normal((n_funcs, n_sensors)) @ root.T


def deeponet_grf(n_u=500, n_y=100, n_sensors=100, width=128, latent=64, frac=0.10,
                 chains=32, eps=2e-4, L=30, seed=3003):
    """DeepONet on GRF inputs: branch 100-128-128-128-64, trunk 2-128-128-128-64, + b0."""
    rng = np.random.default_rng(seed)
    branch = Net.mlp([n_sensors, width, width, width, latent])
    trunk = Net.mlp([2, width, width, width, latent])
    u = _f32(_grf_rows(rng, n_u, n_sensors))
    yq = _f32(rng.uniform(0.0, 1.0, size=(n_y, 2)))
    M = 8
    c = rng.standard_normal(M)
    g = rng.standard_normal((M, n_sensors))
    kk = rng.integers(1, 4, size=(M, 2))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=M)
    amp = np.tanh(u @ g.T / 10.0) * c[None, :]                       # [n_u][M]
    basis = np.cos(np.pi * (yq @ kk.T) + phi[None, :])               # [n_y][M]
    t = amp @ basis.T
    t = _f32(t / (np.std(t) + 1e-12))
    P = deeponet_param_count(branch, trunk)
    mask = _subset_mask(rng, P, frac)
    frozen = _f32(0.05 * rng.standard_normal(P))
    q0 = _initial_states(rng, frozen, mask, chains)
    return Problem("deeponet_grf", KIND_DEEPONET, 0.05, 1.0, frozen, mask, q0, eps=eps, L=L,
                   n_samples=100, seed=0, branch=branch, trunk=trunk, u=u, yq=yq, t=t)


def cone_deeponet(n_u=2000, grid=(64, 128), width=256, latent=128, frac=0.10, chains=128,
                  eps=1e-5, L=20, seed=5005):
    """DeepONet shaped like the cone wall-pressure surrogate: 6 conditions, 64x128 grid."""
    rng = np.random.default_rng(seed)
    branch = Net.mlp([6, width, width, width, latent])
    trunk = Net.mlp([2, width, width, width, latent])
    u = _f32(rng.uniform(0.0, 1.0, size=(n_u, 6)))
    xi = np.linspace(0.0, 1.0, grid[0])
    ph = np.arange(grid[1]) / grid[1]
    XI, PH = np.meshgrid(xi, ph, indexing="ij")
    yq = _f32(np.stack([XI.ravel(), PH.ravel()], axis=1))
    M = 6
    w = rng.standard_normal((M, 6))
    b = rng.standard_normal(M)
    kk = rng.integers(1, 4, size=(M, 2))
    amp = np.tanh(u @ w.T + b[None, :])                               # [n_u][M]
    basis = np.cos(np.pi * (yq @ kk.T))                               # [n_y][M]
    t = amp @ basis.T
    t = _f32(t / (np.std(t) + 1e-12))
    P = deeponet_param_count(branch, trunk)
    mask = _subset_mask(rng, P, frac)
    frozen = _f32(0.05 * rng.standard_normal(P))
    q0 = _initial_states(rng, frozen, mask, chains)
    return Problem("cone_deeponet", KIND_DEEPONET, 0.05, 1.0, frozen, mask, q0, eps=eps, L=L,
                   n_samples=20, seed=0, branch=branch, trunk=trunk, u=u, yq=yq, t=t)


def batched_uneven(n_problems=64, chains=8, eps=2e-4, L=40, seed=4004, n_range=(128, 4096)):
    """Independent 4-input MLPs with widths {32,64,128,256}, 2-4 hidden layers, uneven N."""
    rng = np.random.default_rng(seed)
    probs = []
    for pi in range(n_problems):
        w = int(rng.choice([32, 64, 128, 256]))
        d = int(rng.integers(2, 5))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        f = float(rng.uniform(0.02, 0.20))
        net = Net.mlp([4] + [w] * d + [1])
        x = _f32(rng.uniform(-1.0, 1.0, size=(n, 4)))
        a = rng.standard_normal(3)
        bb = rng.standard_normal((3, 4))
        cc = rng.uniform(0, 2 * np.pi, 3)
        y = (a[None, :] * np.sin(np.pi * x @ bb.T + cc[None, :])).sum(axis=1, keepdims=True)
        y = _f32(y + 0.05 * rng.standard_normal((n, 1)))
        P = net.n_params()
        mask = _subset_mask(rng, P, f)
        frozen = _f32(0.05 * rng.standard_normal(P))
        q0 = _initial_states(rng, frozen, mask, chains)
        p = Problem(f"batched_{pi}", KIND_MLP, 0.05, 1.0, frozen, mask, q0, eps=eps, L=L,
                    n_samples=50, seed=0, net=net, x=x, y=y)
        p.notes = {"width": w, "hidden_layers": d, "n": n, "frac": f}
        probs.append(p)
    return probs


def bayes_linear(n=64, d=5, frac_mask=None, noise=0.3, prior=1.0, chains=4, eps=0.05, L=20,
                 seed=6006):
    """Linear model y = X beta + b + noise as a one-layer MLP with identity output."""
    rng = np.random.default_rng(seed)
    net = Net.mlp([d, 1], last_act=ACT_IDENTITY)
    x = _f32(rng.standard_normal((n, d)))
    beta = rng.standard_normal(d)
    y = _f32(x @ beta[:, None] + 0.5 + noise * rng.standard_normal((n, 1)))
    P = net.n_params()
    frozen = _f32(0.3 * rng.standard_normal(P))
    if frac_mask is None:
        mask = np.ones(P, dtype=np.uint8)
    else:
        mask = np.asarray(frac_mask, dtype=np.uint8)
    q0 = _initial_states(rng, frozen, mask, chains, jitter=0.1)
    return Problem("bayes_linear", KIND_MLP, noise, prior, frozen, mask, q0, eps=eps, L=L,
                   n_samples=4000, seed=0, net=net, x=x, y=y)


def small_mlp(n=300, widths=(3, 40, 33, 2), acts=None, bias=True, frac=0.3, chains=3, eps=1e-3,
              L=8, noise=0.2, prior=1.0, seed=7007):
    """Small ragged MLP used by parity tests (odd widths, multi-output, ragged tiles)."""
    rng = np.random.default_rng(seed)
    if acts is None:
        net = Net.mlp(list(widths), bias=bias)
    else:
        b = [bias] * (len(widths) - 1) if isinstance(bias, bool) else list(bias)
        net = Net(list(widths), list(acts), b)
    x = _f32(rng.uniform(-1.0, 1.0, size=(n, widths[0])))
    y = _f32(np.sin(2.0 * x.sum(axis=1, keepdims=True)) * np.ones((1, widths[-1]))
             + noise * rng.standard_normal((n, widths[-1])))
    P = net.n_params()
    mask = _subset_mask(rng, P, frac)
    frozen = _f32(0.3 * rng.standard_normal(P))
    q0 = _initial_states(rng, frozen, mask, chains, jitter=0.05)
    return Problem("small_mlp", KIND_MLP, noise, prior, frozen, mask, q0, eps=eps, L=L,
                   n_samples=20, seed=0, net=net, x=x, y=y)


def mlp_fanin(n=256, widths=(2, 64, 64, 1), chains=16, noise=0.1, prior=1.0, scale=1.5, seed=9191):
    """MLP with frozen weights N(0, (scale / sqrt(fan_in))^2) and biases N(0, 0.5^2), so
    the hidden units stay out of saturation and their features differ; targets
    sin(pi x1) cos(pi x2) + N(0, noise^2).  The subset is empty: callers choose it."""
    rng = np.random.default_rng(seed)
    net = Net.mlp(list(widths))
    x = _f32(rng.uniform(-1.0, 1.0, size=(n, widths[0])))
    yb = np.sin(np.pi * x[:, :1]) * (np.cos(np.pi * x[:, 1:2]) if widths[0] >= 2 else 1.0)
    y = _f32(np.repeat(yb, widths[-1], axis=1) + noise * rng.standard_normal((n, widths[-1])))
    P = net.n_params()
    frozen = np.zeros(P)
    for l, (wo, bo) in enumerate(net.layer_slices()):
        wi, wout = net.widths[l], net.widths[l + 1]
        frozen[wo:wo + wi * wout] = scale / np.sqrt(wi) * rng.standard_normal(wi * wout)
        if bo >= 0:
            frozen[bo:bo + wout] = 0.5 * rng.standard_normal(wout)
    frozen = _f32(frozen)
    mask = np.zeros(P, dtype=np.uint8)
    q0 = np.zeros((chains, 0))
    return Problem("mlp_fanin", KIND_MLP, noise, prior, frozen, mask, q0, eps=1e-3, L=10,
                   n_samples=1000, seed=0, net=net, x=x, y=y)


def with_subset(prob, mask, chains=None, jitter=0.01, seed=None):
    """The same problem sampling the parameters of `mask`; chains start at the frozen
    values (chain 0) plus seeded N(0, jitter^2) (the others)."""
    rng = np.random.default_rng(prob.seed + 4242 if seed is None else seed)
    p = Problem(**{**prob.__dict__})
    p.mask = np.asarray(mask, dtype=np.uint8)
    p.q0 = _initial_states(rng, p.frozen, p.mask, prob.chains if chains is None else chains, jitter=jitter)
    return p


def small_deeponet(n_u=37, n_y=29, du=12, dy=2, width=24, latent=10, frac=0.3, chains=3,
                   eps=1e-3, L=6, noise=0.2, seed=8008, out_bias=True):
    """Small ragged DeepONet used by parity and finite-difference tests."""
    rng = np.random.default_rng(seed)
    branch = Net.mlp([du, width, width, latent])
    trunk = Net.mlp([dy, width, latent])
    u = _f32(rng.standard_normal((n_u, du)))
    yq = _f32(rng.uniform(0.0, 1.0, size=(n_y, dy)))
    t = _f32(np.tanh(u[:, :1]) @ np.cos(np.pi * yq[:, :1]).T + 0.1 * rng.standard_normal((n_u, n_y)))
    P = deeponet_param_count(branch, trunk, out_bias)
    mask = _subset_mask(rng, P, frac)
    frozen = _f32(0.3 * rng.standard_normal(P))
    q0 = _initial_states(rng, frozen, mask, chains, jitter=0.05)
    return Problem("small_deeponet", KIND_DEEPONET, noise, 1.0, frozen, mask, q0, eps=eps, L=L,
                   n_samples=20, seed=0, branch=branch, trunk=trunk, out_bias=out_bias,
                   u=u, yq=yq, t=t)


def case1_sine(theta, mask=None, chains=1, eps=1e-5, L=724, noise=1e-3, prior=1.0,
               true=(4.0, -3.0, 0.0, 1.57, 0.4, 0.5), seed=1111):
    """Case I of the BNN example (Sec. 4.1.1): y = a sin(w1 x + p1) + b sin(w2 x + p2) + noise
    on 20 points, ten equispaced on each of [-1, -0.2] and [0.2, 1].  The network is
    1-2-1 with sine hidden units, a hidden bias and no output bias; its parameters
    (W1 = (w1, w2), b1 = (p1, p2), W2 = (a, b)) are `theta`, which also gives the frozen
    values.  `true` = (w1, w2, p1, p2, a, b) generates the data.  Default eps and L are
    the paper's (App. C: step 1e-5, L = pi * 0.0679^2 / (2 * 1e-5))."""
    rng = np.random.default_rng(seed)
    net = Net([1, 2, 1], [ACT_SIN, ACT_IDENTITY], [True, False])
    x = _f32(np.concatenate([np.linspace(-1.0, -0.2, 10), np.linspace(0.2, 1.0, 10)])[:, None])
    w1, w2, p1, p2, a, b = true
    y = _f32(a * np.sin(w1 * x + p1) + b * np.sin(w2 * x + p2) + noise * rng.standard_normal(x.shape))
    frozen = _f32(theta)
    mask = np.ones(6, dtype=np.uint8) if mask is None else np.asarray(mask, dtype=np.uint8)
    q0 = np.repeat(frozen[mask.astype(bool)][None, :], chains, axis=0)
    return Problem("case1_sine", KIND_MLP, noise, prior, frozen, mask, q0, eps=eps, L=L, n_samples=5000,
                   seed=0, net=net, x=x, y=y)


def small_deeponet_unaligned(n_u=23, n_q=11, du=6, dy=2, width=16, latent=8, frac=0.4, chains=3,
                             eps=1e-3, L=6, noise=0.2, seed=8108, out_bias=True, shared=False):
    """A DeepONet whose input functions each come with their own n_q query points
    (yq [n_u][n_q][dy], t [n_u][n_q]).  shared=True repeats one query set for every
    function, which makes it the aligned problem in the unaligned layout."""
    rng = np.random.default_rng(seed)
    branch = Net.mlp([du, width, width, latent])
    trunk = Net.mlp([dy, width, latent])
    u = _f32(rng.standard_normal((n_u, du)))
    if shared:
        yq = np.repeat(_f32(rng.uniform(0.0, 1.0, size=(1, n_q, dy))), n_u, axis=0)
    else:
        yq = _f32(rng.uniform(0.0, 1.0, size=(n_u, n_q, dy)))
    t = _f32(np.tanh(u[:, :1]) * np.cos(np.pi * yq[:, :, 0]) + 0.1 * rng.standard_normal((n_u, n_q)))
    P = deeponet_param_count(branch, trunk, out_bias)
    mask = _subset_mask(rng, P, frac)
    frozen = _f32(0.3 * rng.standard_normal(P))
    q0 = _initial_states(rng, frozen, mask, chains, jitter=0.05)
    return Problem("small_deeponet_unaligned", KIND_DEEPONET_UNALIGNED, noise, 1.0, frozen, mask, q0, eps=eps,
                   L=L, n_samples=20, seed=0, branch=branch, trunk=trunk, out_bias=out_bias, u=u, yq=yq, t=t)


def harmonic(k=7, prior=0.7, chains=1, eps=0.1, L=13, seed=9009):
    """No data at all: U(q) = |q|^2 / (2 alpha^2), a harmonic oscillator."""
    rng = np.random.default_rng(seed)
    net = Net.mlp([k, 1], last_act=ACT_IDENTITY, bias=False)
    x = np.zeros((0, k))
    y = np.zeros((0, 1))
    P = net.n_params()
    frozen = _f32(rng.standard_normal(P))
    mask = np.ones(P, dtype=np.uint8)
    q0 = _initial_states(rng, frozen, mask, chains, jitter=0.3)
    return Problem("harmonic", KIND_MLP, 1.0, prior, frozen, mask, q0, eps=eps, L=L,
                   n_samples=10, seed=0, net=net, x=x, y=y)


CONFIGS = {
    "tiny_bnn": tiny_bnn,
    "wide_mlp": wide_mlp,
    "deeponet_grf": deeponet_grf,
    "batched_uneven": batched_uneven,
    "cone_deeponet": cone_deeponet,
}
