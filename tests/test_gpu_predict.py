"""GPU parity of the posterior predictive (hmc_predict, Sec. 4.2.1) against the FP64
oracle, through the C ABI.

The GPU runs samples in batches (a batched forward pass) and reduces them with an
FP64 Welford update; the oracle takes one forward pass per sample and two passes
over the samples.  FP64: 1e-12 on the mean and 1e-9 on the standard deviation
(relative to the output scale); FP32: the forward pass's float rounding, 2e-5 of
the output scale on both.  Full-size workloads (several sample batches) are checked
on sampled inputs, which the predictive treats independently.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import sampler_from

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


def _samples(prob, S, seed, spread=0.05):
    rng = np.random.default_rng(seed)
    q = prob.q0[0] + spread * rng.standard_normal((S, prob.k))
    return q.astype(np.float32).astype(np.float64)


def _check(m, s, mr, sr, tol_m, tol_s):
    scale = max(np.max(np.abs(mr)), 1e-300)
    assert np.max(np.abs(m - mr)) <= tol_m * scale, np.max(np.abs(m - mr)) / scale
    assert np.max(np.abs(s - sr)) <= tol_s * scale, np.max(np.abs(s - sr)) / scale


@pytest.mark.parametrize("which", ["mlp", "deeponet"])
@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_predict_parity(which, prec):
    if which == "mlp":
        prob = W.small_mlp(n=200, widths=(3, 40, 33, 2), chains=1, seed=95)
        new = W.small_mlp(n=123, widths=(3, 40, 33, 2), chains=1, seed=96)   # new inputs and targets
        new.net, new.frozen, new.mask = prob.net, prob.frozen, prob.mask
        kw = dict(x=new.x, y=new.y)
        targets = new.y.reshape(1, -1)    # an MLP's outputs form one row
    else:
        prob = W.small_deeponet(n_u=37, n_y=29, chains=1, seed=97)
        new = W.small_deeponet(n_u=21, n_y=17, chains=1, seed=98)
        new.branch, new.trunk, new.frozen, new.mask = prob.branch, prob.trunk, prob.frozen, prob.mask
        kw = dict(u=new.u, yq=new.yq, t=new.t)
        targets = new.t
    Q = _samples(prob, 37, 1)
    s = sampler_from(prob, prec, chains=1)
    m, sd, rel = s.predict(torch.from_numpy(Q), **kw)
    m, sd = m.cpu().numpy(), sd.cpu().numpy()
    o = oracle.Oracle(new)
    mr, sr = o.predict(Q)
    if prec == hmc.PREC_FP64:
        _check(m, sd, mr, sr, 1e-12, 1e-9)
        assert rel == pytest.approx(oracle.rel_l2(targets, mr.reshape(targets.shape)), rel=1e-12)
    else:
        _check(m, sd, mr, sr, 2e-5, 2e-5)
        assert rel == pytest.approx(oracle.rel_l2(targets, mr.reshape(targets.shape)), rel=1e-4)


def test_predict_one_sample_has_no_spread():
    prob = W.small_mlp(n=50, chains=1, seed=99)
    s = sampler_from(prob, hmc.PREC_FP64, chains=1)
    m, sd, rel = s.predict(torch.from_numpy(prob.q0), x=prob.x)
    assert rel is None
    assert torch.all(sd == 0)
    th = prob.frozen.copy()
    th[prob.idx] = prob.q0[0]
    assert np.allclose(m.cpu().numpy(), oracle.Oracle(prob).forward(th), rtol=1e-13, atol=1e-14)


def test_predict_full_size_wide_mlp_several_batches():
    # 70 samples of the 2-256-256-256-256-1 MLP on 8192 points: about 31 samples per batch
    prob = W.wide_mlp(chains=1)
    Q = _samples(prob, 70, 2, spread=0.02)
    s = sampler_from(prob, hmc.PREC_FP32, chains=1)
    m, sd, rel = s.predict(torch.from_numpy(Q), x=prob.x, y=prob.y)
    rows = np.random.default_rng(3).choice(prob.x.shape[0], 48, replace=False)
    sub = W.wide_mlp(chains=1)
    sub.x, sub.y = prob.x[rows], prob.y[rows]
    mr, sr = oracle.Oracle(sub).predict(Q)
    _check(m.cpu().numpy()[rows], sd.cpu().numpy()[rows], mr, sr, 2e-5, 2e-5)
    assert 0 < rel < 10


def test_predict_full_size_cone_deeponet_several_batches():
    # 25 samples of the 6-256-256-256-128 / 2-256-256-256-128 DeepONet on 2000 x 8192 outputs
    prob = W.cone_deeponet(chains=1)
    Q = _samples(prob, 25, 4, spread=0.01)
    s = sampler_from(prob, hmc.PREC_FP32, chains=1)
    m, sd, rel = s.predict(torch.from_numpy(Q), u=prob.u, yq=prob.yq, t=prob.t)
    rng = np.random.default_rng(5)
    iu, iy = rng.choice(prob.u.shape[0], 6, replace=False), rng.choice(prob.yq.shape[0], 40, replace=False)
    sub = W.cone_deeponet(n_u=6, grid=(4, 10), chains=1)
    sub.u, sub.yq = prob.u[iu], prob.yq[iy]
    sub.frozen, sub.mask = prob.frozen, prob.mask
    mr, sr = oracle.Oracle(sub).predict(Q)
    _check(m.cpu().numpy()[np.ix_(iu, iy)], sd.cpu().numpy()[np.ix_(iu, iy)], mr, sr, 2e-5, 2e-5)
    assert np.isfinite(rel)


@pytest.mark.parametrize("prec", [hmc.PREC_BF16, hmc.PREC_FP16])
@pytest.mark.parametrize("which", ["mlp", "deeponet"])
def test_predict_of_a_16bit_handle_is_the_fp32_one(which, prec):
    # a BF16 or FP16 handle predicts in float from its network, frozen vector and subset,
    # as an FP32 handle of the same problem does: the same numbers, bit for bit
    if which == "mlp":
        prob = W.small_mlp(n=300, widths=(2, 128, 128, 1), frac=0.1, chains=1, seed=93)
        kw = dict(x=prob.x[:111], y=prob.y[:111])
    else:
        prob = W.small_deeponet(n_u=40, n_y=130, du=8, width=64, latent=64, frac=0.1, chains=1, seed=94)
        kw = dict(u=prob.u[:13], yq=prob.yq[:50], t=prob.t[:13, :50])
    Q = torch.from_numpy(_samples(prob, 9, 6))
    m16, s16, r16 = sampler_from(prob, prec, chains=1).predict(Q, **kw)
    m32, s32, r32 = sampler_from(prob, hmc.PREC_FP32, chains=1).predict(Q, **kw)
    assert torch.equal(m16, m32) and torch.equal(s16, s32) and r16 == r32
