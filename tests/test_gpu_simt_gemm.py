"""The FP32 CUDA-core engine at the benchmark's size, through the C ABI.

Its weight gradients reduce over all 8192 data rows on a 256 x 256 output, which the
engine splits over K (split-K partials added in a fixed order).  U and grad U must match
the FP64 oracle to the FP32 tolerance (1e-5), and since the split depends on the shape
only, a chain gives bit-identical results whether it runs alone or beside others.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


def test_fp32_wide_mlp_one_chain_and_batched():
    prob = W.wide_mlp(chains=3)
    s1 = sampler_from(prob, hmc.PREC_FP32, chains=1)
    s3 = sampler_from(prob, hmc.PREC_FP32)
    U1, g1 = s1.energy_grad(torch.from_numpy(prob.q0[:1]))
    U3, g3 = s3.energy_grad(torch.from_numpy(prob.q0))
    assert torch.equal(U1[0], U3[0]) and torch.equal(g1[0], g3[0])
    Ur, gr = oracle.Oracle(prob).energy_grad(prob.q0[0])
    assert abs(U1[0].item() - Ur) <= 1e-5 * abs(Ur)
    ok, re, comp = grad_ok(g1[0].cpu().double().numpy(), gr, 1e-5)
    assert ok, (re, comp)
