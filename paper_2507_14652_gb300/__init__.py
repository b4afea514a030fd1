"""Python binding of libhmc.so -- the GB300 subset-HMC library.

Argument marshalling only: every step of U, grad U, the leapfrog integrator and
the Metropolis step runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the compiled library is missing
the import of :func:`lib` raises.

Typical use::

    import paper_2507_14652_gb300 as hmc
    s = hmc.Sampler.mlp([2, 256, 256, 1], x, y, mask, frozen, chains=16,
                        prior_sigma=1.0, noise_sigma=0.05, prec=hmc.PREC_BF16)
    U, g = s.energy_grad(q)                      # torch CUDA tensors
    S, acc, dH, q_last = s.sample(q0, eps=5e-4, L=50, n=100, seed=0)
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhmc.so")
MAXL = 16

ACT_IDENTITY, ACT_TANH, ACT_SIN = 0, 1, 2
PREC_FP64, PREC_FP32, PREC_TF32, PREC_BF16, PREC_FP16 = 0, 1, 2, 3, 4
NET_MLP, NET_DEEPONET, NET_DEEPONET_UNALIGNED = 0, 1, 2
STATUS = {0: "HMC_OK", 1: "HMC_ERR_ARG", 2: "HMC_ERR_CUDA", 3: "HMC_ERR_OOM", 4: "HMC_ERR_NONFINITE",
          5: "HMC_ERR_TIMEOUT", 6: "HMC_ERR_UNSUPPORTED"}

# every symbol the C ABI (include/hmc.h, include/hmc_diag.h) declares
EXPORTS = ["hmc_create", "hmc_create_batch", "hmc_create_split", "hmc_create_chunked", "hmc_num_passes",
           "hmc_sensitivity", "hmc_select_subset",
           "hmc_predict", "hmc_subset_size", "hmc_param_count", "hmc_num_chains", "hmc_diag_umma_gemm",
           "hmc_energy_grad", "hmc_leapfrog", "hmc_sample", "hmc_sample_steps", "hmc_adapt_step_size", "hmc_check",
           "hmc_destroy",
           "hmc_last_error",
           "hmc_energy_grad_noalloc",
           "hmc_diag_philox", "hmc_diag_momenta", "hmc_diag_log_uniform", "hmc_diag_graph_kernels",
           "hmc_diag_profile_energy_grad", "hmc_diag_metropolis_energy", "hmc_diag_tuning",
           "hmc_diag_expire_wait", "hmc_diag_graph_captures", "hmc_diag_adapt_trace", "hmc_diag_dual_averaging",
           "hmc_diag_device_bytes", "hmc_diag_set_memory_cap", "hmc_diag_tanh16", "hmc_diag_set_grouping",
           "hmc_diag_groups"]


class HmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MlpSpec(ct.Structure):
    _fields_ = [("n_layers", ct.c_int), ("widths", ct.c_int * (MAXL + 1)),
                ("act", ct.c_int * MAXL), ("has_bias", ct.c_int * MAXL)]


class NetSpec(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("net", MlpSpec), ("branch", MlpSpec), ("trunk", MlpSpec),
                ("deeponet_out_bias", ct.c_int), ("prec", ct.c_int)]


class Data(ct.Structure):
    _fields_ = [("x", ct.c_void_p), ("n", ct.c_long), ("dx", ct.c_int), ("y", ct.c_void_p),
                ("u", ct.c_void_p), ("n_u", ct.c_long), ("du", ct.c_int),
                ("yq", ct.c_void_p), ("n_y", ct.c_long), ("dy", ct.c_int), ("t", ct.c_void_p),
                ("dtype", ct.c_int)]


DATA_F64, DATA_F32 = 0, 1


_lib = None


def build(force=False, verbose=False):
    from . import _build
    return _build.build(force=force, verbose=verbose)


def lib():
    """Load libhmc.so.  Raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2507_14652_gb300.build() first")
        L = ct.CDLL(LIB_PATH)
        vp, d, i, lg, u64 = ct.c_void_p, ct.c_double, ct.c_int, ct.c_long, ct.c_ulonglong
        L.hmc_create.argtypes = [ct.POINTER(vp), ct.POINTER(NetSpec), ct.POINTER(Data), d, d, vp, vp, i, vp]
        L.hmc_create_batch.argtypes = [ct.POINTER(vp), i, ct.POINTER(NetSpec), ct.POINTER(Data),
                                       ct.POINTER(d), ct.POINTER(d), ct.POINTER(vp), ct.POINTER(vp), i, vp]
        L.hmc_predict.argtypes = [vp, vp, lg, ct.POINTER(Data), vp, vp, ct.POINTER(d)]
        L.hmc_sensitivity.argtypes = [ct.POINTER(NetSpec), ct.POINTER(Data), vp, vp, vp, vp]
        L.hmc_select_subset.argtypes = [vp, lg, d, vp, ct.POINTER(lg), vp, vp]
        L.hmc_create_split.argtypes = [ct.POINTER(vp), ct.POINTER(NetSpec), ct.POINTER(Data), d, d, vp, vp, i, i, vp]
        L.hmc_create_chunked.argtypes = [ct.POINTER(vp), ct.POINTER(NetSpec), ct.POINTER(Data), d, d, vp, vp, i, lg,
                                         vp]
        L.hmc_num_passes.argtypes = [vp]
        L.hmc_num_passes.restype = i
        L.hmc_diag_device_bytes.argtypes = []
        L.hmc_diag_device_bytes.restype = lg
        L.hmc_diag_set_memory_cap.argtypes = [lg]
        L.hmc_diag_tanh16.argtypes = [vp, vp, lg]
        L.hmc_diag_set_memory_cap.restype = None
        L.hmc_diag_set_grouping.argtypes = [i]
        L.hmc_diag_set_grouping.restype = None
        L.hmc_diag_groups.argtypes = [vp, ct.c_char_p, lg]
        L.hmc_diag_groups.restype = lg
        L.hmc_subset_size.argtypes = [vp]
        L.hmc_subset_size.restype = lg
        L.hmc_param_count.argtypes = [vp]
        L.hmc_param_count.restype = lg
        L.hmc_num_chains.argtypes = [vp]
        L.hmc_num_chains.restype = i
        L.hmc_energy_grad.argtypes = [vp, vp, vp, vp]
        L.hmc_leapfrog.argtypes = [vp, vp, vp, d, i]
        L.hmc_sample.argtypes = [vp, vp, d, i, lg, u64, lg, vp, vp, vp, vp]
        L.hmc_sample_steps.argtypes = [vp, vp, vp, i, lg, u64, lg, vp, vp, vp, vp]
        L.hmc_adapt_step_size.argtypes = [vp, vp, i, d, lg, d, u64, lg, vp]
        L.hmc_check.argtypes = [vp]
        L.hmc_diag_expire_wait.argtypes = [vp, lg]
        L.hmc_destroy.argtypes = [vp]
        L.hmc_last_error.restype = ct.c_char_p
        L.hmc_diag_philox.argtypes = [vp, vp, lg, vp]
        L.hmc_diag_momenta.argtypes = [u64, u64, u64, u64, lg, vp]
        L.hmc_diag_log_uniform.argtypes = [u64, u64, lg, lg, vp]
        L.hmc_energy_grad_noalloc.argtypes = [ct.POINTER(MlpSpec), vp, vp, lg, vp, vp, lg, d, d, i, vp, vp, vp,
                                              vp]
        L.hmc_diag_graph_kernels.argtypes = [vp]
        L.hmc_diag_graph_kernels.restype = lg
        L.hmc_diag_graph_captures.argtypes = [vp]
        L.hmc_diag_graph_captures.restype = lg
        L.hmc_diag_adapt_trace.argtypes = [vp, vp, lg]
        L.hmc_diag_dual_averaging.argtypes = [vp, lg, i, d, d, vp]
        L.hmc_diag_profile_energy_grad.argtypes = [vp, vp, i, vp, i]
        L.hmc_diag_umma_gemm.argtypes = [i] * 6 + [vp] * 3
        L.hmc_diag_metropolis_energy.argtypes = [vp, vp, vp]
        L.hmc_diag_tuning.argtypes = [vp, ct.c_char_p, lg]
        L.hmc_diag_tuning.restype = lg
        for f in EXPORTS:
            if f not in ("hmc_subset_size", "hmc_param_count", "hmc_num_chains", "hmc_last_error", "hmc_num_passes",
                         "hmc_diag_device_bytes", "hmc_diag_set_memory_cap", "hmc_diag_set_grouping",
                         "hmc_diag_groups", "hmc_diag_graph_kernels", "hmc_diag_graph_captures", "hmc_diag_tuning"):
                getattr(L, f).restype = ct.c_int
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise HmcError(st, lib().hmc_last_error().decode())


def mlp_spec(widths, act=None, bias=True):
    """MlpSpec from widths; default act: tanh hidden layers, identity output."""
    s = MlpSpec()
    n = len(widths) - 1
    assert 1 <= n <= MAXL
    if act is None:
        act = [ACT_TANH] * (n - 1) + [ACT_IDENTITY]
    if isinstance(bias, bool):
        bias = [bias] * n
    s.n_layers = n
    for l, w in enumerate(widths):
        s.widths[l] = int(w)
    for l in range(n):
        s.act[l] = int(act[l])
        s.has_bias[l] = 1 if bias[l] else 0
    return s


def _ptr(a):
    """Raw pointer of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _f64(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    import torch
    return a.detach().to(torch.float64).contiguous()


def _is_f32(a):
    return str(getattr(a, "dtype", "")) in ("float32", "torch.float32")


def _training_arrays(*arrays):
    """The training set as passed to the library: float32 when every array is float32
    (numpy or torch, handed over without a copy to float64), else float64."""
    if all(_is_f32(a) for a in arrays):
        out = []
        for a in arrays:
            out.append(np.ascontiguousarray(a) if isinstance(a, np.ndarray) else a.detach().contiguous())
        return out, DATA_F32
    return [_f64(a) for a in arrays], DATA_F64


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Sampler:
    """One libhmc handle: a problem (or a batch of problems) with C chains."""

    def __init__(self, spec, data, arrays, prior_sigma, noise_sigma, mask, frozen, chains, stream=None,
                 n_splits=1, rows_per_pass=0):
        import torch
        self.prec = spec.prec
        self.dtype = torch.float64 if spec.prec == PREC_FP64 else torch.float32
        self._keep = list(arrays)
        m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8))
        f = _f64(np.asarray(frozen)) if not hasattr(frozen, "data_ptr") else _f64(frozen)
        self._keep += [m, f]
        h = ct.c_void_p()
        if rows_per_pass:   # evaluate the data in passes of rows_per_pass rows (hmc_create_chunked)
            assert n_splits == 1, "a handle is either chunked or split"
            _check(lib().hmc_create_chunked(ct.byref(h), ct.byref(spec), ct.byref(data), float(prior_sigma),
                                            float(noise_sigma), _ptr(m), _ptr(f), int(chains), int(rows_per_pass),
                                            _stream_ptr(stream)))
        elif n_splits == 1:
            _check(lib().hmc_create(ct.byref(h), ct.byref(spec), ct.byref(data), float(prior_sigma),
                                    float(noise_sigma), _ptr(m), _ptr(f), int(chains), _stream_ptr(stream)))
        else:   # symmetric split integrator over n_splits data batches
            _check(lib().hmc_create_split(ct.byref(h), ct.byref(spec), ct.byref(data), float(prior_sigma),
                                          float(noise_sigma), _ptr(m), _ptr(f), int(chains), int(n_splits),
                                          _stream_ptr(stream)))
        self._h = h
        self.n_splits = int(n_splits)
        self.dout = spec.net.widths[spec.net.n_layers] if spec.kind == NET_MLP else 1
        self.chains = int(chains)
        self.k = int(lib().hmc_subset_size(h))
        self.P = int(lib().hmc_param_count(h))
        self.n_problems = 1
        self.passes = int(lib().hmc_num_passes(h))

    @classmethod
    def mlp(cls, widths, x, y, mask, frozen, chains, prior_sigma=1.0, noise_sigma=1.0, prec=PREC_FP32,
            act=None, bias=True, stream=None, n_splits=1, rows_per_pass=0):
        spec = NetSpec()
        spec.kind = NET_MLP
        spec.net = mlp_spec(widths, act, bias)
        spec.prec = prec
        (x, y), dt = _training_arrays(x, y)
        d = Data()
        d.x, d.n, d.dx, d.y, d.dtype = _ptr(x), x.shape[0], x.shape[1], _ptr(y), dt
        return cls(spec, d, [x, y], prior_sigma, noise_sigma, mask, frozen, chains, stream, n_splits, rows_per_pass)

    @classmethod
    def deeponet(cls, branch, trunk, u, yq, t, mask, frozen, chains, prior_sigma=1.0, noise_sigma=1.0,
                 prec=PREC_FP32, out_bias=True, branch_act=None, trunk_act=None, branch_bias=True,
                 trunk_bias=True, stream=None, n_splits=1, rows_per_pass=0):
        """A DeepONet; yq [n_y][dy] holds query points shared by every input function, or
        yq [n_u][n_y][dy] each function's own (HMC_NET_DEEPONET_UNALIGNED)."""
        spec = NetSpec()
        spec.kind = NET_DEEPONET if np.ndim(yq) == 2 else NET_DEEPONET_UNALIGNED
        spec.branch = mlp_spec(branch, branch_act, branch_bias)
        spec.trunk = mlp_spec(trunk, trunk_act, trunk_bias)
        spec.deeponet_out_bias = 1 if out_bias else 0
        spec.prec = prec
        (u, yq, t), dt = _training_arrays(u, yq, t)
        d = Data()
        d.dtype = dt
        d.u, d.n_u, d.du = _ptr(u), u.shape[0], u.shape[1]
        d.yq, d.n_y, d.dy = _ptr(yq), yq.shape[-2], yq.shape[-1]
        d.t = _ptr(t)
        return cls(spec, d, [u, yq, t], prior_sigma, noise_sigma, mask, frozen, chains, stream, n_splits,
                   rows_per_pass)

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().hmc_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _state(self, q):
        import torch
        if isinstance(q, np.ndarray):
            q = torch.from_numpy(q)
        return q.to(device="cuda", dtype=self.dtype).contiguous()

    def energy_grad(self, q, want_grad=True):
        """U [C] (float64) and grad U [C][k] for states q [C][k] (CUDA tensors)."""
        import torch
        q = self._state(q)
        U = torch.empty(self.n_problems * self.chains, dtype=torch.float64, device="cuda")
        g = torch.empty_like(q) if want_grad else None
        _check(lib().hmc_energy_grad(self._h, _ptr(q), _ptr(U), _ptr(g)))
        return U, g

    def leapfrog(self, q, p, eps, L):
        q = self._state(q).clone()
        p = self._state(p).clone()
        _check(lib().hmc_leapfrog(self._h, _ptr(q), _ptr(p), float(eps), int(L)))
        return q, p

    def sample(self, q0, eps, L, n, seed=0, first_traj=0, keep_samples=True):
        """n trajectories per chain; returns (samples [n][C][k], accepted [n][C], dH [n][C], q_last [C][k]).
        eps: one step for every problem, or a sequence of one per problem (hmc_sample_steps)."""
        import torch
        q0 = self._state(q0)
        nseg = self.n_problems * self.chains
        S = torch.empty((n,) + tuple(q0.shape), dtype=self.dtype, device="cuda") if keep_samples else None
        acc = torch.empty((n, nseg), dtype=torch.uint8, device="cuda")
        dH = torch.empty((n, nseg), dtype=torch.float64, device="cuda")
        ql = torch.empty_like(q0)
        if np.ndim(eps) == 0:
            _check(lib().hmc_sample(self._h, _ptr(q0), float(eps), int(L), int(n), int(seed), int(first_traj),
                                    _ptr(S), _ptr(acc), _ptr(dH), _ptr(ql)))
        else:
            e = np.ascontiguousarray(eps, dtype=np.float64)
            if e.shape != (self.n_problems,):
                raise ValueError(f"need one step per problem ({self.n_problems}), got shape {e.shape}")
            _check(lib().hmc_sample_steps(self._h, _ptr(q0), _ptr(e), int(L), int(n), int(seed), int(first_traj),
                                          _ptr(S), _ptr(acc), _ptr(dH), _ptr(ql)))
        return S, acc, dH, ql

    def adapt_step_size(self, q0, L, eps0, n_warmup, target_accept=0.8, seed=0, first_traj=0):
        """Dual-averaging warm-up (hmc_adapt_step_size): returns (eps, q after the warm-up),
        eps a float for one problem, else an array of one step per problem."""
        q = self._state(q0).clone()
        eps = np.zeros(self.n_problems)
        _check(lib().hmc_adapt_step_size(self._h, _ptr(q), int(L), float(eps0), int(n_warmup), float(target_accept),
                                         int(seed), int(first_traj), _ptr(eps)))
        return (float(eps[0]) if self.n_problems == 1 else eps), q

    def check(self):
        """hmc_check: wait for the handle's work; raises HmcError (HMC_ERR_TIMEOUT) when a
        bounded device-side wait gave up since the last check."""
        _check(lib().hmc_check(self._h))

    def tuning(self):
        """What the engines autotuned at creation (hmc_diag_tuning)."""
        n = lib().hmc_diag_tuning(self._h, None, 0)
        buf = ct.create_string_buffer(int(n) + 1)
        lib().hmc_diag_tuning(self._h, buf, int(n) + 1)
        return buf.value.decode()

    def predict(self, samples, x=None, y=None, u=None, yq=None, t=None):
        """Posterior predictive on new inputs (hmc_predict): mean and std ([n][d_out] for
        an MLP, [n_u][n_y] for a DeepONet) as float64 CUDA tensors, and the mean relative
        L2 error of the mean when targets (y or t) are given (else None)."""
        import torch
        S = samples.reshape(-1, self.k).to(device="cuda", dtype=self.dtype).contiguous()
        d = Data()
        keep = []
        if x is not None:
            x = _f64(x)
            d.x, d.n, d.dx = _ptr(x), x.shape[0], x.shape[1]
            keep.append(x)
            shape = (x.shape[0], self.dout)
            tg = y
        else:
            u, yq = _f64(u), _f64(yq)
            d.u, d.n_u, d.du = _ptr(u), u.shape[0], u.shape[1]
            d.yq, d.n_y, d.dy = _ptr(yq), yq.shape[0], yq.shape[1]
            keep += [u, yq]
            shape = (u.shape[0], yq.shape[0])
            tg = t
        rel = None
        if tg is not None:
            tg = _f64(tg)
            keep.append(tg)
            if x is not None:
                d.y = _ptr(tg)
            else:
                d.t = _ptr(tg)
            rel = ct.c_double()
        mean = torch.empty(shape, dtype=torch.float64, device="cuda")
        std = torch.empty_like(mean)
        _check(lib().hmc_predict(self._h, _ptr(S), S.shape[0], ct.byref(d), _ptr(mean), _ptr(std),
                                 ct.byref(rel) if rel is not None else None))
        return mean, std, (rel.value if rel is not None else None)

    def metropolis_energy(self, q):
        """U [C] used by the Metropolis test (hmc_diag_metropolis_energy)."""
        import torch
        q = self._state(q)
        U = torch.empty(self.n_problems * self.chains, dtype=torch.float64, device="cuda")
        _check(lib().hmc_diag_metropolis_energy(self._h, _ptr(q), _ptr(U)))
        return U

    def sample_host(self, q0, eps, L, n, seed=0, first_traj=0):
        """Same as sample() with numpy (host) buffers: the library stages the copies."""
        dt = np.float64 if self.prec == PREC_FP64 else np.float32
        q0 = np.ascontiguousarray(q0, dtype=dt)
        nseg = self.n_problems * self.chains
        S = np.empty((n,) + q0.shape, dtype=dt)
        acc = np.empty((n, nseg), dtype=np.uint8)
        dH = np.empty((n, nseg), dtype=np.float64)
        ql = np.empty_like(q0)
        _check(lib().hmc_sample(self._h, _ptr(q0), float(eps), int(L), int(n), int(seed), int(first_traj),
                                _ptr(S), _ptr(acc), _ptr(dH), _ptr(ql)))
        return S, acc, dH, ql


def _sens(spec, d, keep, mu, sd):
    import torch
    P = int(np.asarray(mu).shape[0]) if not hasattr(mu, "data_ptr") else int(mu.shape[0])
    m = mu.to(device="cuda", dtype=torch.float64).contiguous() if hasattr(mu, "data_ptr") else \
        torch.from_numpy(np.ascontiguousarray(mu, dtype=np.float64)).cuda()
    v = sd.to(device="cuda", dtype=torch.float64).contiguous() if hasattr(sd, "data_ptr") else \
        torch.from_numpy(np.ascontiguousarray(sd, dtype=np.float64)).cuda()
    S2 = torch.empty(P, dtype=torch.float64, device="cuda")
    _check(lib().hmc_sensitivity(ct.byref(spec), ct.byref(d), _ptr(m), _ptr(v), _ptr(S2), _stream_ptr(None)))
    return S2


def sensitivity_mlp(widths, x, mu, sd, prec=PREC_FP32, act=None, bias=True):
    """S_i^2 (Sec. 3.1) of every parameter of an MLP at the VI means mu with VI standard
    deviations sd (hmc_sensitivity); a float64 CUDA tensor [P]."""
    spec = NetSpec()
    spec.kind = NET_MLP
    spec.net = mlp_spec(widths, act, bias)
    spec.prec = prec
    x = _f64(x)
    d = Data()
    d.x, d.n, d.dx = _ptr(x), x.shape[0], x.shape[1]
    return _sens(spec, d, [x], mu, sd)


def sensitivity_deeponet(branch, trunk, u, yq, mu, sd, prec=PREC_FP32, out_bias=True, branch_act=None,
                         trunk_act=None, branch_bias=True, trunk_bias=True):
    """S_i^2 (Sec. 3.1) of every DeepONet parameter over all (input function, query) pairs."""
    spec = NetSpec()
    spec.kind = NET_DEEPONET
    spec.branch = mlp_spec(branch, branch_act, branch_bias)
    spec.trunk = mlp_spec(trunk, trunk_act, trunk_bias)
    spec.deeponet_out_bias = 1 if out_bias else 0
    spec.prec = prec
    u, yq = _f64(u), _f64(yq)
    d = Data()
    d.u, d.n_u, d.du = _ptr(u), u.shape[0], u.shape[1]
    d.yq, d.n_y, d.dy = _ptr(yq), yq.shape[0], yq.shape[1]
    return _sens(spec, d, [u, yq], mu, sd)


def select_subset(S2, tau):
    """N-hat of Sec. 3.1 and the subset (hmc_select_subset): (n_hat, mask [P] uint8,
    ranking [P] int64), all from the GPU."""
    import torch
    S2 = S2.to(device="cuda", dtype=torch.float64).contiguous() if hasattr(S2, "data_ptr") else \
        torch.from_numpy(np.ascontiguousarray(S2, dtype=np.float64)).cuda()
    P = int(S2.shape[0])
    mask = torch.empty(P, dtype=torch.uint8, device="cuda")
    order = torch.empty(P, dtype=torch.int64, device="cuda")
    n = ct.c_long()
    _check(lib().hmc_select_subset(_ptr(S2), P, float(tau), _ptr(mask), ct.byref(n), _ptr(order),
                                   _stream_ptr(None)))
    return int(n.value), mask, order


class KernelTime(ct.Structure):
    _fields_ = [("name", ct.c_char * 48), ("ms_total", ct.c_double), ("launches", ct.c_long)]


def profile_energy_grad(sampler, q, reps=5):
    """{kernel kind: (mean ms per launch, launches per evaluation)} from CUDA events
    recorded around every launch on the library's stream."""
    import torch
    q = sampler._state(q)
    buf = (KernelTime * 64)()
    n = lib().hmc_diag_profile_energy_grad(sampler._h, _ptr(q), int(reps), buf, 64)
    if n < 0:
        _check(-n)
    return {buf[i].name.decode(): (buf[i].ms_total / buf[i].launches, buf[i].launches / reps) for i in range(n)}


def graph_kernels(sampler):
    """Kernel launches in one captured trajectory of the last sample() call."""
    return int(lib().hmc_diag_graph_kernels(sampler._h))


def graph_captures(sampler):
    """Trajectory graphs the handle has captured so far (hmc_diag_graph_captures)."""
    return int(lib().hmc_diag_graph_captures(sampler._h))


def adapt_trace(sampler, n):
    """Step sizes of the last adapt_step_size() call: [n][2] = (step of trajectory m + 1,
    averaged step after update m) for m = 1..n (hmc_diag_adapt_trace); [n][problems][2]
    for a batch."""
    out = np.zeros((n, sampler.n_problems, 2))
    _check(lib().hmc_diag_adapt_trace(sampler._h, _ptr(out), int(n)))
    return out[:, 0, :] if sampler.n_problems == 1 else out


def diag_dual_averaging(dH, eps0, target):
    """The library's device dual-averaging update run on given dH[n][nseg] rows
    (hmc_diag_dual_averaging); returns [n][2] as adapt_trace()."""
    d = np.ascontiguousarray(dH, dtype=np.float64)
    out = np.zeros((d.shape[0], 2))
    _check(lib().hmc_diag_dual_averaging(_ptr(d), d.shape[0], d.shape[1], float(eps0), float(target), _ptr(out)))
    return out


class BatchSampler(Sampler):
    """Several independent problems behind one handle (hmc_create_batch)."""

    def __init__(self, problems, chains, prec, stream=None, grouped=True):
        """problems: one tuple per problem, (widths, x, y, mask, frozen, prior_sigma,
        noise_sigma) for an MLP, or ("deeponet", branch_widths, trunk_widths, u, yq, t, mask,
        frozen, prior_sigma, noise_sigma, out_bias) for a DeepONet whose n_y query points
        are shared by its input functions.  grouped: problems of one tensor-core kernel
        shape share launches (the default); False launches every problem's kernels on
        their own (for comparison)."""
        n = len(problems)
        specs = (NetSpec * n)()
        datas = (Data * n)()
        alphas = (ct.c_double * n)()
        sigmas = (ct.c_double * n)()
        masks = (ct.c_void_p * n)()
        frozens = (ct.c_void_p * n)()
        keep = []
        for i, pr in enumerate(problems):
            specs[i].prec = prec
            if isinstance(pr[0], str):
                kind, branch, trunk, u, yq, t, mask, frozen, alpha, sigma, out_bias = pr
                if kind != "deeponet":
                    raise ValueError("unknown problem kind %r" % (kind,))
                specs[i].kind = NET_DEEPONET
                specs[i].branch, specs[i].trunk = mlp_spec(branch), mlp_spec(trunk)
                specs[i].deeponet_out_bias = 1 if out_bias else 0
                u, yq, t = _f64(u), _f64(yq), _f64(t)
                keep += [u, yq, t]
                d = datas[i]
                d.u, d.n_u, d.du = _ptr(u), u.shape[0], u.shape[1]
                d.yq, d.n_y, d.dy = _ptr(yq), yq.shape[0], yq.shape[1]
                d.t = _ptr(t)
            else:
                widths, x, y, mask, frozen, alpha, sigma = pr
                specs[i].kind = NET_MLP
                specs[i].net = mlp_spec(widths)
                x, y = _f64(x), _f64(y)
                keep += [x, y]
                datas[i].x, datas[i].n, datas[i].dx, datas[i].y = _ptr(x), x.shape[0], x.shape[1], _ptr(y)
            m = np.ascontiguousarray(mask, dtype=np.uint8)
            f = _f64(np.asarray(frozen))
            keep += [m, f]
            alphas[i], sigmas[i] = alpha, sigma
            masks[i], frozens[i] = _ptr(m), _ptr(f)
        import torch
        self.prec = prec
        self.dtype = torch.float64 if prec == PREC_FP64 else torch.float32
        self._keep = keep
        h = ct.c_void_p()
        lib().hmc_diag_set_grouping(1 if grouped else 0)
        try:
            _check(lib().hmc_create_batch(ct.byref(h), n, specs, datas, alphas, sigmas, masks, frozens, int(chains),
                                          _stream_ptr(stream)))
        finally:
            lib().hmc_diag_set_grouping(1)
        self._h = h
        self.chains = int(chains)
        self.n_problems = n
        self.k = int(lib().hmc_subset_size(h))
        self.P = int(lib().hmc_param_count(h))

    def groups(self):
        """The handle's launch groups, one description per group."""
        buf = ct.create_string_buffer(8192)
        n = lib().hmc_diag_groups(self._h, buf, len(buf))
        return [ln for ln in buf.value.decode().splitlines() if ln][:max(n, 0)]


def _energy_grad_fn():
    import torch

    class EnergyGrad(torch.autograd.Function):
        """U(q) per chain with the library's hand-written adjoint as its backward.

        forward(q [C][k], sampler) -> U [C] (float64); backward multiplies the stored
        grad U by the upstream gradient of each chain's U.
        """

        @staticmethod
        def forward(ctx, q, sampler):
            U, g = sampler.energy_grad(q.detach())
            ctx.save_for_backward(g)
            return U

        @staticmethod
        def backward(ctx, gU):
            (g,) = ctx.saved_tensors
            return (gU.to(g.dtype)[:, None] * g), None

    return EnergyGrad


_EG = None


def energy(q, sampler):
    """Differentiable U(q): torch.autograd sees the library's adjoint kernel as the gradient."""
    global _EG
    if _EG is None:
        _EG = _energy_grad_fn()
    return _EG.apply(q, sampler)


def diag_philox(ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint64).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint64).reshape(-1, 2)
    out = np.zeros_like(ctr)
    _check(lib().hmc_diag_philox(_ptr(ctr), _ptr(key), ctr.shape[0], _ptr(out)))
    return out


def diag_momenta(seed, chain, traj, k, problem=0):
    out = np.zeros(k)
    _check(lib().hmc_diag_momenta(int(seed), int(problem), int(chain), int(traj), int(k), _ptr(out)))
    return out


def diag_log_uniform(seed, n_chain, n_traj, problem=0):
    out = np.zeros((n_chain, n_traj))
    _check(lib().hmc_diag_log_uniform(int(seed), int(problem), int(n_chain), int(n_traj), _ptr(out)))
    return out
