"""Grouped launches of a batch's tensor-core problems (hmc_create_batch), through the C ABI.

A batch handle puts its BF16/FP16 MLP problems of one kernel shape (padded hidden width,
input width, kernel family) into a group whose gradient takes one launch per kernel and
layer slot for all of them.  Each launch runs every problem's own kernel body on its own
buffers, so U and grad U must equal the per-problem launches bit for bit, and so must
whole trajectories; against the FP64 oracle the tolerances are the single problems'.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok_bf16

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu

PREC = {"bf16": hmc.PREC_BF16, "fp16": hmc.PREC_FP16}
TOL = {"bf16": 2e-2, "fp16": 5e-3}


def _tuples(probs):
    return [(p.net.widths, p.x, p.y, p.mask, p.frozen, p.prior_sigma, p.noise_sigma) for p in probs]


def _mixed(chains=3, seed=5):
    """Widths 32..256 (up to 128 padded to 128, 200 to 256), one to three hidden w x w
    layers, ragged N, subsets from 2% to 30%, two problems with six inputs at width 256
    (the tile kernel: the pair kernel keeps the first layer's sums for up to four), and
    one problem whose subset holds only output-layer weights (no reverse pass below the
    top layer)."""
    rng = np.random.default_rng(seed)
    probs = []
    for i, (dx, w, d) in enumerate([(4, 32, 2), (4, 64, 4), (4, 64, 3), (4, 32, 3), (4, 128, 2), (4, 100, 4),
                                    (4, 128, 3), (4, 128, 4), (4, 256, 2), (4, 256, 4), (4, 200, 3), (4, 256, 2),
                                    (6, 256, 3), (6, 200, 2)]):
        n = int(rng.integers(100, 700))
        frac = float(rng.uniform(0.02, 0.3))
        probs.append(W.small_mlp(n=n, widths=(dx,) + (w,) * d + (1,), frac=frac, chains=chains, seed=100 + i))
    top = W.small_mlp(n=333, widths=(4, 256, 256, 1), frac=0.1, chains=chains, seed=99)
    P = top.P
    mask = np.zeros(P, dtype=np.uint8)
    mask[P - 1 - 256:P - 1:7] = 1                       # a few output weights
    probs.append(W.with_subset(top, mask, chains=chains))
    return probs


def _states(probs, seed=7):
    rng = np.random.default_rng(seed)
    return np.concatenate([(p.q0 + 0.02 * rng.standard_normal(p.q0.shape)).reshape(-1) for p in probs])


def _split(flat, probs):
    out, off = [], 0
    for p in probs:
        C, k = p.q0.shape
        out.append(flat[off:off + C * k].reshape(C, k))
        off += C * k
    return out


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_grouped_gradient_is_bitwise_the_per_problem_one(prec):
    probs = _mixed()
    q = torch.from_numpy(_states(probs).astype(np.float32))
    sg = hmc.BatchSampler(_tuples(probs), probs[0].chains, PREC[prec])
    su = hmc.BatchSampler(_tuples(probs), probs[0].chains, PREC[prec], grouped=False)
    assert su.groups() == []
    groups = sg.groups()
    assert len(groups) == 3, groups                     # 128 and 256 (pair kernel), 256 with dx 6 (tile kernel)
    Ug, gg = sg.energy_grad(q)
    Uu, gu = su.energy_grad(q)
    assert torch.equal(Ug, Uu) and torch.equal(gg, gu)
    # and against the oracle, problem by problem
    C = probs[0].chains
    qs = _split(q.double().numpy(), probs)
    gs = _split(gg.cpu().double().numpy(), probs)
    Ug = Ug.cpu().numpy()
    for i, p in enumerate(probs):
        Ur, gr = oracle.Oracle(p).energy_grad_batch(qs[i])
        for c in range(C):
            assert abs(Ug[i * C + c] - Ur[c]) <= TOL[prec] * abs(Ur[c]), (i, c)
            ok, r2, rinf = grad_ok_bf16(gs[i][c], gr[c], TOL[prec])
            assert ok, (i, p.net.widths, c, r2, rinf)
    sg.close()
    su.close()


def test_grouped_trajectories_are_bitwise_the_per_problem_ones():
    probs = _mixed(chains=2, seed=8)
    q0 = torch.from_numpy(np.concatenate([p.q0.reshape(-1) for p in probs]).astype(np.float32))
    out = []
    for grouped in (True, False):
        s = hmc.BatchSampler(_tuples(probs), 2, hmc.PREC_BF16, grouped=grouped)
        out.append(s.sample(q0, 2e-4, 12, 4, seed=3))
        s.close()
    for a, b in zip(*out):
        assert torch.equal(a, b)
    acc = out[0][1].float().mean().item()
    assert 0.0 < acc <= 1.0


def test_grouped_full_size_batched_workload():
    # the 64-problem workload (widths 32..256, 2-4 hidden layers, N 128..4096, 8 chains):
    # grouped equals per-problem bit for bit; three problems checked against the oracle
    probs = W.batched_uneven()
    q = torch.from_numpy(_states(probs).astype(np.float32))
    sg = hmc.BatchSampler(_tuples(probs), 8, hmc.PREC_BF16)
    su = hmc.BatchSampler(_tuples(probs), 8, hmc.PREC_BF16, grouped=False)
    assert len(sg.groups()) == 2                        # widths up to 128, and 256
    Ug, gg = sg.energy_grad(q)
    Uu, gu = su.energy_grad(q)
    assert torch.equal(Ug, Uu) and torch.equal(gg, gu)
    qs = _split(q.double().numpy(), probs)
    gs = _split(gg.cpu().double().numpy(), probs)
    for i in (0, 31, 63):
        Ur, gr = oracle.Oracle(probs[i]).energy_grad(qs[i][5])
        assert abs(Ug[i * 8 + 5].item() - Ur) <= 2e-2 * abs(Ur)
        assert grad_ok_bf16(gs[i][5], gr)[0], i
    sg.close()
    su.close()


def test_one_problem_per_shape_is_not_grouped():
    probs = [W.small_mlp(n=200, widths=(dx, w, w, 1), frac=0.1, chains=2, seed=s)
             for s, dx, w in ((1, 4, 64), (2, 6, 256), (3, 4, 256))]
    s = hmc.BatchSampler(_tuples(probs), 2, hmc.PREC_BF16)
    assert s.groups() == []
    s.close()
