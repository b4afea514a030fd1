"""FP64 CPU oracle of the subset-HMC hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.

The arithmetic lives in ``hmc_oracle.c`` (plain C, FP64, one data term at a
time); this module only marshals numpy arrays into it.  ``ess.py`` holds the
effective-sample-size estimator used to score chains.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

_MAXL = 16
_lib = None


class _Net(ct.Structure):
    _fields_ = [("n_layers", ct.c_int), ("width", ct.c_int * (_MAXL + 1)),
                ("act", ct.c_int * _MAXL), ("bias", ct.c_int * _MAXL)]


class _Problem(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("out_bias", ct.c_int),
                ("net", _Net), ("branch", _Net), ("trunk", _Net),
                ("n", ct.c_long), ("dx", ct.c_int), ("x", ct.c_void_p), ("y", ct.c_void_p),
                ("n_u", ct.c_long), ("du", ct.c_int), ("u", ct.c_void_p),
                ("n_y", ct.c_long), ("dy", ct.c_int), ("yq", ct.c_void_p),
                ("t", ct.c_void_p),
                ("noise_sigma", ct.c_double), ("prior_sigma", ct.c_double),
                ("frozen", ct.c_void_p), ("P", ct.c_long),
                ("idx", ct.c_void_p), ("k", ct.c_long)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        d, vp, u64, lg, i = ct.c_double, ct.c_void_p, ct.c_uint64, ct.c_long, ct.c_int
        L.or_param_count.restype = lg
        L.or_param_count.argtypes = [vp]
        L.or_energy_grad.restype = d
        L.or_energy_grad.argtypes = [vp, vp, vp]
        L.or_energy_grad_batch.restype = None
        L.or_energy_grad_batch.argtypes = [vp, i, vp, vp, vp, i]
        L.or_forward.restype = None
        L.or_forward.argtypes = [vp, vp, vp]
        L.or_philox4x64_10.restype = None
        L.or_philox4x64_10.argtypes = [vp, vp, vp]
        L.or_unit_uniform.restype = d
        L.or_unit_uniform.argtypes = [u64]
        L.or_log.restype = d
        L.or_log.argtypes = [d]
        L.or_sincos_2pi.restype = None
        L.or_sincos_2pi.argtypes = [u64, vp, vp]
        L.or_momentum.restype = d
        L.or_momentum.argtypes = [u64, u64, u64, u64, u64]
        L.or_mh_uniform.restype = d
        L.or_mh_uniform.argtypes = [u64, u64, u64, u64]
        L.or_leapfrog.restype = None
        L.or_leapfrog.argtypes = [vp, vp, vp, d, i, vp, vp]
        L.or_sample.restype = None
        L.or_sample.argtypes = [vp, vp, i, d, i, lg, u64, u64, lg, vp, vp, vp, vp, i]
        L.or_data_rows.restype = lg
        L.or_data_rows.argtypes = [vp]
        L.or_energy_grad_rows.restype = d
        L.or_energy_grad_rows.argtypes = [vp, vp, vp, lg, lg, d]
        L.or_batch_rows.restype = None
        L.or_batch_rows.argtypes = [vp, i, i, vp, vp]
        L.or_split_leapfrog.restype = None
        L.or_split_leapfrog.argtypes = [vp, i, vp, vp, d, i]
        L.or_split_sample.restype = None
        L.or_split_sample.argtypes = [vp, i, vp, i, d, i, lg, u64, u64, lg, vp, vp, vp, vp, i]
        L.or_sensitivity.restype = None
        L.or_sensitivity.argtypes = [vp, vp, vp, vp]
        L.or_truncate.restype = lg
        L.or_truncate.argtypes = [vp, lg, d, vp, vp]
        L.or_predict.restype = None
        L.or_predict.argtypes = [vp, vp, lg, vp, vp]
        L.or_rel_l2.restype = d
        L.or_rel_l2.argtypes = [vp, vp, lg, lg]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ct.c_void_p) if a is not None else None


def _net(nt):
    s = _Net()
    if nt is None:
        return s
    s.n_layers = nt.n_layers
    for l, w in enumerate(nt.widths):
        s.width[l] = int(w)
    for l in range(nt.n_layers):
        s.act[l] = int(nt.act[l])
        s.bias[l] = 1 if nt.bias[l] else 0
    return s


class Oracle:
    """Wraps one workloads.Problem for the C oracle.  All arrays are float64."""

    def __init__(self, prob):
        self.prob = prob
        self._keep = []
        s = _Problem()
        s.kind = prob.kind
        s.out_bias = 1 if prob.out_bias else 0

        def keep(a, dtype=np.float64):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dtype)
            self._keep.append(a)
            return a

        if prob.kind == 0:
            s.net = _net(prob.net)
            x, y = keep(prob.x), keep(prob.y)
            s.n, s.dx, s.x, s.y = x.shape[0], x.shape[1], _ptr(x), _ptr(y)
        else:
            s.branch, s.trunk = _net(prob.branch), _net(prob.trunk)
            u, yq, t = keep(prob.u), keep(prob.yq), keep(prob.t)
            s.n_u, s.du, s.u = u.shape[0], u.shape[1], _ptr(u)
            if prob.kind == 2:   # every input function with its own queries: yq [n_u][n_y][dy]
                s.n_y, s.dy, s.yq = yq.shape[1], yq.shape[2], _ptr(yq)
            else:
                s.n_y, s.dy, s.yq = yq.shape[0], yq.shape[1], _ptr(yq)
            s.t = _ptr(t)
        s.noise_sigma, s.prior_sigma = float(prob.noise_sigma), float(prob.prior_sigma)
        fr = keep(prob.frozen)
        idx = keep(prob.idx, np.int64)
        s.frozen, s.P = _ptr(fr), fr.shape[0]
        s.idx, s.k = _ptr(idx), idx.shape[0]
        self._s = s
        self._sp = ct.cast(ct.pointer(s), ct.c_void_p)
        self.k = int(idx.shape[0])
        self.P = int(fr.shape[0])

    def param_count(self):
        return int(lib().or_param_count(self._sp))

    def forward(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        p = self.prob
        if p.kind == 0:
            f = np.zeros((p.x.shape[0], p.net.widths[-1]))
        else:
            f = np.zeros(p.t.shape)
        lib().or_forward(self._sp, _ptr(theta), _ptr(f))
        return f

    def energy_grad(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        g = np.zeros(self.k)
        U = lib().or_energy_grad(self._sp, _ptr(q), _ptr(g))
        return U, g

    def energy(self, q):
        q = np.ascontiguousarray(q, dtype=np.float64)
        return lib().or_energy_grad(self._sp, _ptr(q), None)

    def energy_grad_batch(self, Q, threads=0):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        C = Q.shape[0]
        U = np.zeros(C)
        G = np.zeros((C, self.k))
        lib().or_energy_grad_batch(self._sp, C, _ptr(Q), _ptr(U), _ptr(G), int(threads))
        return U, G

    def data_rows(self):
        return int(lib().or_data_rows(self._sp))

    def batch_rows(self, M, m):
        r0, r1 = ct.c_long(), ct.c_long()
        lib().or_batch_rows(self._sp, int(M), int(m), ct.byref(r0), ct.byref(r1))
        return r0.value, r1.value

    def energy_grad_rows(self, q, r0, r1, w=1.0):
        """Likelihood of data rows [r0, r1) plus the fraction w of the prior, and its gradient."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        g = np.zeros(self.k)
        U = lib().or_energy_grad_rows(self._sp, _ptr(q), _ptr(g), int(r0), int(r1), float(w))
        return U, g

    def split_leapfrog(self, q, p, eps, L, M):
        """L steps of the symmetric split integrator over M data batches."""
        q = np.array(q, dtype=np.float64)
        p = np.array(p, dtype=np.float64)
        lib().or_split_leapfrog(self._sp, int(M), _ptr(q), _ptr(p), float(eps), int(L))
        return q, p

    def split_sample(self, q0, eps, L, n, M, seed=0, first_traj=0, problem=0, threads=0):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        C = q0.shape[0]
        S = np.zeros((n, C, self.k))
        acc = np.zeros((n, C), dtype=np.uint8)
        dH = np.zeros((n, C))
        ql = np.zeros((C, self.k))
        lib().or_split_sample(self._sp, int(M), _ptr(q0), C, float(eps), int(L), int(n), int(seed), int(problem),
                              int(first_traj), _ptr(S), _ptr(acc), _ptr(dH), _ptr(ql), int(threads))
        return S, acc, dH, ql

    def sensitivity(self, mu, sd):
        """S_i^2 of Sec. 3.1 for every parameter: the network at the VI means mu [P]
        with VI standard deviations sd [P]."""
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        sd = np.ascontiguousarray(sd, dtype=np.float64)
        S2 = np.zeros(self.P)
        lib().or_sensitivity(self._sp, _ptr(mu), _ptr(sd), _ptr(S2))
        return S2

    def predict(self, samples):
        """Mean and standard deviation over posterior samples [S][k] of the network's
        outputs on this problem's inputs (Sec. 4.2.1)."""
        Q = np.ascontiguousarray(samples, dtype=np.float64).reshape(-1, self.k)
        p = self.prob
        shape = (p.x.shape[0], p.net.widths[-1]) if p.kind == 0 else p.t.shape
        mean, sd = np.zeros(shape), np.zeros(shape)
        lib().or_predict(self._sp, _ptr(Q), Q.shape[0], _ptr(mean), _ptr(sd))
        return mean, sd

    def leapfrog(self, q, p, eps, L, U=None, g=None):
        q = np.array(q, dtype=np.float64)
        p = np.array(p, dtype=np.float64)
        if U is None or g is None:
            U, g = self.energy_grad(q)
        g = np.array(g, dtype=np.float64)
        Ub = np.array([U], dtype=np.float64)
        lib().or_leapfrog(self._sp, _ptr(q), _ptr(p), float(eps), int(L), _ptr(Ub), _ptr(g))
        return q, p, float(Ub[0]), g

    def sample(self, q0, eps, L, n, seed=0, first_traj=0, problem=0, threads=0):
        q0 = np.ascontiguousarray(q0, dtype=np.float64)
        C = q0.shape[0]
        S = np.zeros((n, C, self.k))
        acc = np.zeros((n, C), dtype=np.uint8)
        dH = np.zeros((n, C))
        ql = np.zeros((C, self.k))
        lib().or_sample(self._sp, _ptr(q0), C, float(eps), int(L), int(n), int(seed), int(problem),
                        int(first_traj), _ptr(S), _ptr(acc), _ptr(dH), _ptr(ql), int(threads))
        return S, acc, dH, ql


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def unit_uniform(w):
    return lib().or_unit_uniform(int(w))


def log(x):
    return lib().or_log(float(x))


def sincos_2pi(m):
    s, c = ct.c_double(), ct.c_double()
    lib().or_sincos_2pi(int(m), ct.byref(s), ct.byref(c))
    return s.value, c.value


def momenta(seed, chain, traj, k, problem=0):
    L = lib()
    return np.array([L.or_momentum(int(seed), int(problem), int(chain), int(traj), j) for j in range(k)])


def mh_uniform(seed, chain, traj, problem=0):
    return lib().or_mh_uniform(int(seed), int(problem), int(chain), int(traj))


def truncate(S2, tau):
    """N-hat of Sec. 3.1 and the subset mask [P] (uint8), plus the ranking [P]."""
    S2 = np.ascontiguousarray(S2, dtype=np.float64)
    P = S2.shape[0]
    mask = np.zeros(P, dtype=np.uint8)
    order = np.zeros(P, dtype=np.int64)
    nhat = lib().or_truncate(_ptr(S2), P, float(tau), _ptr(mask), _ptr(order))
    return int(nhat), mask, order


def rel_l2(Y, Yp):
    """(1/N) sum_i ||Y_i - Yp_i|| / ||Y_i|| over the rows of Y [N][m] (Sec. 4.2.1)."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    Yp = np.ascontiguousarray(Yp, dtype=np.float64)
    Y2, P2 = Y.reshape(Y.shape[0], -1), Yp.reshape(Y.shape[0], -1)
    return float(lib().or_rel_l2(_ptr(Y2), _ptr(P2), Y2.shape[0], Y2.shape[1]))
