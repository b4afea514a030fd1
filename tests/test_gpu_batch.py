"""GPU parity of independent problems behind one handle (hmc_create_batch) against the
FP64 oracle, one problem at a time.

The problems mix hidden widths 32..256, 2..4 hidden layers and ragged data sizes, the
shape of the batched small-MLP workload (64 problems x 8 chains) scaled down so the
oracle finishes in seconds.  The state is the problems' [C][k_p] blocks back to back;
U is [problem][chain].  Tolerances are those of the single-problem tests.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _adapt import grad_ok, grad_ok_bf16

torch = pytest.importorskip("torch")
hmc = pytest.importorskip("paper_2507_14652_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    hmc.lib()


def _problems(widths=None, n=16, chains=2):
    probs = W.batched_uneven(n_problems=n, chains=chains, n_range=(100, 900))
    if widths is not None:
        probs = [p for p in probs if p.notes["width"] in widths]
    return probs


def _batch(probs, prec):
    tup = [(p.net.widths, p.x, p.y, p.mask, p.frozen, p.prior_sigma, p.noise_sigma) for p in probs]
    return hmc.BatchSampler(tup, probs[0].chains, prec)


def _states(probs, seed=7):
    rng = np.random.default_rng(seed)
    return [(p.q0 + 0.02 * rng.standard_normal(p.q0.shape)).astype(np.float32).astype(np.float64) for p in probs]


def _split(flat, probs):
    out, off = [], 0
    for p in probs:
        C, k = p.q0.shape
        out.append(flat[off:off + C * k].reshape(C, k))
        off += C * k
    assert off == flat.size
    return out


def _energy_grad(probs, prec):
    s = _batch(probs, prec)
    qs = _states(probs)
    U, g = s.energy_grad(torch.from_numpy(np.concatenate([q.reshape(-1) for q in qs])))
    return qs, U.cpu().numpy(), _split(g.cpu().double().numpy(), probs), s


@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32])
def test_batch_energy_grad_parity(prec):
    probs = _problems()
    qs, U, gs, s = _energy_grad(probs, prec)
    assert s.n_problems == len(probs) and s.k == sum(p.q0.shape[1] for p in probs)
    tol = 1e-10 if prec == hmc.PREC_FP64 else 1e-5
    C = probs[0].chains
    for i, (p, q, g) in enumerate(zip(probs, qs, gs)):
        Ur, gr = oracle.Oracle(p).energy_grad_batch(q)
        for c in range(C):
            assert abs(U[i * C + c] - Ur[c]) <= tol * abs(Ur[c]), (i, c, U[i * C + c], Ur[c])
            ok, re, comp = grad_ok(g[c], gr[c], tol)
            assert ok, (i, p.notes, c, re, comp)


def test_batch_bf16_energy_grad_parity():
    # widths 64 (padded to 128), 128 and 256 on the persistent pair kernels
    probs = _problems(widths=(64, 128, 256))
    assert {p.notes["width"] for p in probs} == {64, 128, 256}
    qs, U, gs, _ = _energy_grad(probs, hmc.PREC_BF16)
    C = probs[0].chains
    for i, (p, q, g) in enumerate(zip(probs, qs, gs)):
        Ur, gr = oracle.Oracle(p).energy_grad_batch(q)
        for c in range(C):
            assert abs(U[i * C + c] - Ur[c]) <= 2e-2 * abs(Ur[c]), (i, c, U[i * C + c], Ur[c])
            ok, r2, rinf = grad_ok_bf16(g[c], gr[c])
            assert ok, (i, p.notes, c, r2, rinf)


def test_batch_bf16_pads_width_32_onto_the_tensor_cores():
    # hidden widths below 128 run on the tensor cores padded to 128 with units
    # whose weights are zero (they change neither U nor the real parameters' gradient)
    probs = _problems(widths=(32, 128))
    assert {p.notes["width"] for p in probs} == {32, 128}
    qs, U, gs, _ = _energy_grad(probs, hmc.PREC_BF16)
    C = probs[0].chains
    for i, (p, q, g) in enumerate(zip(probs, qs, gs)):
        Ur, gr = oracle.Oracle(p).energy_grad_batch(q)
        for c in range(C):
            assert abs(U[i * C + c] - Ur[c]) <= 2e-2 * abs(Ur[c]), (i, c, U[i * C + c], Ur[c])
            ok, r2, rinf = grad_ok_bf16(g[c], gr[c])
            assert ok, (i, p.notes, c, r2, rinf)
    # a single-problem tensor-core handle takes width 32 as well, and still refuses a width
    # beyond 256
    p = probs[[q.notes["width"] for q in probs].index(32)]
    hmc.Sampler.mlp(p.net.widths, p.x, p.y, p.mask, p.frozen, p.chains, prec=hmc.PREC_BF16).close()
    wide = W.small_mlp(n=200, widths=(4, 300, 300, 1), frac=0.05, chains=2, seed=3)
    with pytest.raises(hmc.HmcError):
        hmc.Sampler.mlp(wide.net.widths, wide.x, wide.y, wide.mask, wide.frozen, 2, prec=hmc.PREC_BF16)


def test_batch_sample_parity_fp64():
    # each problem draws its momenta and uniforms from its own Philox stream (problem index)
    probs = [p for p in _problems() if p.q0.shape[1] < 1200][:3]
    assert len(probs) == 3
    s = _batch(probs, hmc.PREC_FP64)
    n, eps, L, seed = 4, 2e-4, 5, 11
    q0 = np.concatenate([p.q0.reshape(-1) for p in probs])
    S, acc, dH, ql = s.sample(torch.from_numpy(q0), eps, L, n, seed=seed)
    S, acc, dH = S.cpu().numpy(), acc.cpu().numpy(), dH.cpu().numpy()
    C = probs[0].chains
    for i, p in enumerate(probs):
        Sr, accr, dHr, qlr = oracle.Oracle(p).sample(p.q0, eps, L, n, seed=seed, problem=i)
        lu = np.array([[oracle.log(oracle.mh_uniform(seed, c, t, problem=i)) for c in range(C)] for t in range(n)])
        band = 1e-8 * (1 + np.abs(dHr))
        clear = np.abs(lu + dHr) > band
        assert np.array_equal(acc[:, i * C:(i + 1) * C][clear], accr[clear]), i
        assert np.allclose(dH[:, i * C:(i + 1) * C], dHr, rtol=1e-6, atol=1e-7), i
        Si = np.stack([_split(S[t], probs)[i] for t in range(n)])
        assert np.max(np.abs(Si - Sr)) <= 1e-9 * max(1.0, np.max(np.abs(Sr))), i


def _mixed_kinds(chains=2):
    """Two MLPs and two DeepONets (branch and trunk widths 64 and 128, ragged sizes)."""
    return [W.small_mlp(n=333, widths=(4, 64, 64, 1), frac=0.2, chains=chains, seed=61),
            W.small_deeponet(n_u=40, n_y=130, du=8, width=64, latent=64, frac=0.1, chains=chains, seed=62),
            W.small_mlp(n=517, widths=(3, 128, 128, 128, 1), frac=0.1, chains=chains, seed=63),
            W.small_deeponet(n_u=150, n_y=90, du=5, width=128, latent=64, frac=0.2, chains=chains, seed=64,
                             out_bias=False)]


def _tuple(p):
    if p.branch is not None:
        return ("deeponet", p.branch.widths, p.trunk.widths, p.u, p.yq, p.t, p.mask, p.frozen, p.prior_sigma,
                p.noise_sigma, p.out_bias)
    return (p.net.widths, p.x, p.y, p.mask, p.frozen, p.prior_sigma, p.noise_sigma)


@pytest.mark.parametrize("prec", [hmc.PREC_FP64, hmc.PREC_FP32, hmc.PREC_BF16, hmc.PREC_FP16])
def test_batch_mixes_mlps_and_deeponets(prec):
    # a batch may hold DeepONets beside MLPs: each problem's U and grad U are its own
    probs = _mixed_kinds()
    s = hmc.BatchSampler([_tuple(p) for p in probs], 2, prec)
    assert s.n_problems == 4 and s.k == sum(p.q0.shape[1] for p in probs)
    qs = _states(probs)
    U, g = s.energy_grad(torch.from_numpy(np.concatenate([q.reshape(-1) for q in qs])))
    U, gs = U.cpu().numpy(), _split(g.cpu().double().numpy(), probs)
    tol = {hmc.PREC_FP64: 1e-10, hmc.PREC_FP32: 1e-5, hmc.PREC_BF16: 2e-2, hmc.PREC_FP16: 5e-3}[prec]
    for i, (p, q) in enumerate(zip(probs, qs)):
        Ur, gr = oracle.Oracle(p).energy_grad_batch(q)
        for c in range(2):
            assert abs(U[i * 2 + c] - Ur[c]) <= tol * abs(Ur[c]), (i, c, U[i * 2 + c], Ur[c])
            if prec in (hmc.PREC_FP64, hmc.PREC_FP32):
                ok, re, comp = grad_ok(gs[i][c], gr[c], tol)
            else:
                ok, re, comp = grad_ok_bf16(gs[i][c], gr[c], tol)
            assert ok, (i, c, re, comp)
    s.close()


def test_batch_with_deeponets_sample_parity_fp64():
    # problem i draws from Philox stream i, DeepONet or MLP
    probs = _mixed_kinds()
    s = hmc.BatchSampler([_tuple(p) for p in probs], 2, hmc.PREC_FP64)
    n, eps, L, seed = 3, 2e-4, 4, 13
    q0 = np.concatenate([p.q0.reshape(-1) for p in probs])
    S, acc, dH, _ = s.sample(torch.from_numpy(q0), eps, L, n, seed=seed)
    S, acc, dH = S.cpu().numpy(), acc.cpu().numpy(), dH.cpu().numpy()
    for i, p in enumerate(probs):
        Sr, accr, dHr, _ = oracle.Oracle(p).sample(p.q0, eps, L, n, seed=seed, problem=i)
        lu = np.array([[oracle.log(oracle.mh_uniform(seed, c, t, problem=i)) for c in range(2)] for t in range(n)])
        clear = np.abs(lu + dHr) > 1e-8 * (1 + np.abs(dHr))
        assert np.array_equal(acc[:, 2 * i:2 * i + 2][clear], accr[clear]), i
        assert np.allclose(dH[:, 2 * i:2 * i + 2], dHr, rtol=1e-6, atol=1e-7), i
        Si = np.stack([_split(S[t], probs)[i] for t in range(n)])
        assert np.max(np.abs(Si - Sr)) <= 1e-9 * max(1.0, np.max(np.abs(Sr))), i
    s.close()
