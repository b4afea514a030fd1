"""Evaluation in passes over the data rows (hmc_create_chunked), through the C ABI.

U and grad U are sums over the data terms (Sec. 2.2; the full-batch potential of
Sec. 3.3), so a handle that evaluates the rows a pass at a time, with one pass's
activations on the device, must give the oracle's U and grad U at each precision's
tolerance, ragged last pass included, and sample the same chains.  hmc_create falls back
to passes when the whole batch does not fit; a cap on the library's device memory drives
that fallback here without filling the GPU.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, grad_ok_bf16, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "fp16": 5e-3, "bf16": 2e-2}
PREC = {"fp64": hmc.PREC_FP64, "fp32": hmc.PREC_FP32, "fp16": hmc.PREC_FP16, "bf16": hmc.PREC_BF16}


def _check(prob, prec, rows_per_pass, passes):
    s = sampler_from(prob, PREC[prec], rows_per_pass=rows_per_pass)
    assert s.passes == passes
    U, g = s.energy_grad(torch.from_numpy(prob.q0))
    U, g = U.cpu().numpy(), g.cpu().double().numpy()
    Ur, gr = oracle.Oracle(prob).energy_grad_batch(prob.q0)
    tol = TOL[prec]
    for c in range(prob.chains):
        assert abs(U[c] - Ur[c]) <= tol * abs(Ur[c]), (prec, c, U[c], Ur[c])
        ok = grad_ok(g[c], gr[c], tol)[0] if prec in ("fp64", "fp32") else grad_ok_bf16(g[c], gr[c], tol)[0]
        assert ok, (prec, c)
    return s


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chunked_mlp_cuda_cores(prec):
    prob = W.small_mlp(n=517, widths=(3, 40, 33, 2), frac=0.3, chains=3, seed=71)
    _check(prob, prec, 128, 5)          # 517 rows in passes of at most 128: 5 passes, ragged


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_chunked_mlp_tensor_cores(prec):
    prob = W.small_mlp(n=1500, widths=(2, 128, 128, 128, 1), frac=0.1, chains=4, seed=72)
    _check(prob, prec, 400, 4)          # four passes of 375 rows: tiles cut mid-pass


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_chunked_deeponet(prec):
    prob = W.small_deeponet(n_u=37, n_y=29, chains=3, seed=73) if prec != "bf16" else \
        W.small_deeponet(n_u=70, n_y=130, du=12, dy=2, width=64, latent=64, frac=0.2, chains=2, seed=74)
    _check(prob, prec, 10 if prec != "bf16" else 30, 4 if prec != "bf16" else 3)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_chunked_wide_deeponet_on_the_pair_kernels(prec):
    # width 256 and latent 128: the branch's hidden and last layers run on the CTA-pair
    # kernels (forward, reverse with bias sums, the 256 -> 128 layer both ways), the trunk
    # on its second stream, every pass drawing its row buffers from the shared arena
    prob = W.small_deeponet(n_u=300, n_y=260, du=3, dy=2, width=256, latent=128, frac=0.1, chains=2, seed=77)
    _check(prob, prec, 100, 3)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chunked_deeponet_with_own_queries(prec):
    prob = W.small_deeponet_unaligned(chains=3)
    _check(prob, prec, 6, -(-prob.u.shape[0] // 6))


def test_chunked_chains_follow_the_oracle():
    # FP64: the same trajectories as the oracle's (dH to 1e-8, identical accept decisions)
    prob = W.small_mlp(n=300, widths=(2, 16, 16, 1), frac=0.4, chains=3, seed=75)
    s = sampler_from(prob, hmc.PREC_FP64, rows_per_pass=70)
    assert s.passes == 5
    S, acc, dH, ql = s.sample(torch.from_numpy(prob.q0), 2e-3, 8, 6, seed=12)
    Sr, accr, dHr, qlr = oracle.Oracle(prob).sample(prob.q0, 2e-3, 8, 6, seed=12)
    assert np.array_equal(acc.cpu().numpy(), accr)
    assert np.allclose(dH.cpu().numpy(), dHr, rtol=1e-8, atol=1e-10)
    assert np.allclose(ql.cpu().numpy(), qlr, rtol=1e-9, atol=1e-12)


def test_passes_hold_less_device_memory():
    prob = W.small_mlp(n=32768, widths=(2, 256, 256, 256, 1), frac=0.02, chains=4, seed=76)
    b0 = hmc.lib().hmc_diag_device_bytes()
    full = sampler_from(prob, hmc.PREC_BF16)
    b_full = hmc.lib().hmc_diag_device_bytes() - b0
    full.close()
    b0 = hmc.lib().hmc_diag_device_bytes()
    ch = sampler_from(prob, hmc.PREC_BF16, rows_per_pass=4096)
    b_ch = hmc.lib().hmc_diag_device_bytes() - b0
    assert ch.passes == 8
    assert b_ch < 0.35 * b_full, (b_ch, b_full)
    ch.close()


def test_create_falls_back_to_passes_when_memory_runs_short():
    prob = W.small_mlp(n=32768, widths=(2, 256, 256, 256, 1), frac=0.02, chains=4, seed=76)
    b0 = hmc.lib().hmc_diag_device_bytes()
    full = sampler_from(prob, hmc.PREC_FP32)
    need = hmc.lib().hmc_diag_device_bytes() - b0
    U_full, g_full = full.energy_grad(torch.from_numpy(prob.q0))
    full.close()
    try:
        hmc.lib().hmc_diag_set_memory_cap(hmc.lib().hmc_diag_device_bytes() + need // 2)
        s = sampler_from(prob, hmc.PREC_FP32)          # plain hmc_create
        assert s.passes >= 2, s.passes
        U, g = s.energy_grad(torch.from_numpy(prob.q0))
    finally:
        hmc.lib().hmc_diag_set_memory_cap(0)
    # the passes give the whole batch's U and grad U (each checked against the oracle above)
    assert torch.allclose(U, U_full, rtol=1e-6, atol=0)
    for c in range(prob.chains):
        assert grad_ok(g[c].cpu().double().numpy(), g_full[c].cpu().double().numpy(), 1e-5)[0]
