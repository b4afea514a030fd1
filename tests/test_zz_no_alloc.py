"""hmc_energy_grad_noalloc: U and grad U of an FP32 MLP without any device allocation.

It is meant for callers that cannot call cudaMalloc: a plug-in whose host
framework's memory pool owns the device, or a loop that may not block in the
allocator.  Its intermediates live in one fixed array inside the library, shared
by every call.  The tests check, on two calls in a row that reuse that array, its
results against the FP64 oracle at the FP32 tolerance of the other tests (1e-5)
and against hmc_energy_grad on an FP32 handle; that problems beyond the array are
refused; and that an index list out of range or out of order gives NaN instead of
being used as an address.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


def _noalloc(prob, q, idx=None):
    L = hmc.lib()
    net = hmc.mlp_spec(prob.net.widths, prob.net.act, prob.net.bias)
    x = torch.from_numpy(prob.x).float().cuda().contiguous()
    y = torch.from_numpy(prob.y).float().cuda().contiguous()
    fr = torch.from_numpy(prob.frozen).float().cuda()
    idx = torch.from_numpy((prob.idx if idx is None else idx).astype(np.int32)).cuda()
    qd = torch.from_numpy(q).float().cuda().contiguous()
    C = q.shape[0]
    U = torch.full((C,), 12345.0, dtype=torch.float64, device="cuda")
    g = torch.full((C, prob.k), 12345.0, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    st = L.hmc_energy_grad_noalloc(ctypes.byref(net), x.data_ptr(), y.data_ptr(), x.shape[0], fr.data_ptr(),
                                   idx.data_ptr(), prob.k, prob.prior_sigma, prob.noise_sigma, C, qd.data_ptr(),
                                   U.data_ptr(), g.data_ptr(), stream.cuda_stream)
    assert st == 0, L.hmc_last_error()
    torch.cuda.synchronize()
    return U.cpu().numpy(), g.cpu().double().numpy()


CASES = {
    "tanh": lambda: W.small_mlp(n=517, widths=(3, 130, 67, 1), frac=0.1, chains=3, seed=5),
    "sin_nobias": lambda: W.small_mlp(widths=(4, 9, 9, 3), acts=[W.ACT_TANH, W.ACT_SIN, W.ACT_TANH],
                                      bias=[True, False, True], frac=0.5, chains=2, seed=2),
    "tiny_bnn": lambda: W.tiny_bnn(chains=2),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_oracle_and_handle_on_two_consecutive_calls(case):
    prob = CASES[case]()
    o = oracle.Oracle(prob)
    s = sampler_from(prob, hmc.PREC_FP32)
    rng = np.random.default_rng(17)
    for call in range(2):
        q = (prob.q0 + 0.03 * rng.standard_normal(prob.q0.shape)).astype(np.float32).astype(np.float64)
        Ur, gr = o.energy_grad_batch(q)
        U0, g0 = s.energy_grad(torch.from_numpy(q))
        U0, g0 = U0.cpu().numpy(), g0.cpu().double().numpy()
        U1, g1 = _noalloc(prob, q)
        for c in range(prob.chains):
            assert abs(U1[c] - Ur[c]) <= 1e-5 * abs(Ur[c]), (call, c, U1[c], Ur[c])
            ok, re, comp = grad_ok(g1[c], gr[c], 1e-5)
            assert ok, (call, c, re, comp)
            assert abs(U1[c] - U0[c]) <= 1e-5 * abs(U0[c]), (call, c, U1[c], U0[c])
            ok, re, comp = grad_ok(g1[c], g0[c], 1e-5)
            assert ok, (call, c, re, comp)


@pytest.mark.parametrize("bad", ["negative", "beyond_P", "not_ascending"])
def test_noalloc_index_list_is_checked_on_the_device(bad):
    prob = CASES["tanh"]()
    idx = prob.idx.copy()
    if bad == "negative":
        idx[3] = -7
    elif bad == "beyond_P":
        idx[-1] = prob.P + 1000
    else:
        idx[[4, 5]] = idx[[5, 4]]
    U, g = _noalloc(prob, prob.q0, idx=idx)
    assert np.all(np.isnan(U)) and np.all(np.isnan(g))
    # the next call with a valid list is unaffected by the flag of the one before
    U2, g2 = _noalloc(prob, prob.q0)
    Ur, _ = oracle.Oracle(prob).energy_grad_batch(prob.q0)
    assert np.all(np.abs(U2 - Ur) <= 1e-5 * np.abs(Ur))


def test_noalloc_rejects_problems_beyond_its_fixed_scratch():
    L = hmc.lib()
    prob = W.wide_mlp(n=8192, chains=16)        # needs far more than 16 MiB of intermediates
    net = hmc.mlp_spec(prob.net.widths)
    dummy = torch.zeros(16, device="cuda")
    U = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = L.hmc_energy_grad_noalloc(ctypes.byref(net), dummy.data_ptr(), dummy.data_ptr(), 8192, dummy.data_ptr(),
                                   dummy.data_ptr(), prob.k, 1.0, 0.05, 16, dummy.data_ptr(), U.data_ptr(), None,
                                   None)
    assert st == 1
    assert b"16 MiB" in L.hmc_last_error()
    # a row count whose byte size would wrap around 64 bits is refused the same way
    st = L.hmc_energy_grad_noalloc(ctypes.byref(net), dummy.data_ptr(), dummy.data_ptr(), 1 << 61,
                                   dummy.data_ptr(), dummy.data_ptr(), prob.k, 1.0, 0.05, 16, dummy.data_ptr(),
                                   U.data_ptr(), None, None)
    assert st == 1
    assert b"16 MiB" in L.hmc_last_error()
