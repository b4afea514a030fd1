"""Network-convention pins from the parameter counts the paper prints, and the
shapes of the five synthetic workloads (CPU only)."""
import json
import os

import numpy as np

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "param_counts.json")


def _net(widths, bias=None):
    n = len(widths) - 1
    return W.Net(list(widths), [W.ACT_TANH] * (n - 1) + [W.ACT_IDENTITY],
                 [True] * n if bias is None else list(bias))


def test_paper_parameter_counts():
    gold = json.load(open(GOLD))
    for name, e in gold.items():
        if name.startswith("_"):
            continue
        if e["kind"] == "mlp":
            nt = _net(e["widths"], e["bias"])
            count = nt.n_params()
            prob = W.Problem(name, W.KIND_MLP, 1.0, 1.0, np.zeros(count), np.zeros(count, np.uint8),
                             np.zeros((1, 0)), 1e-3, 1, net=nt, x=np.zeros((0, e["widths"][0])),
                             y=np.zeros((0, e["widths"][-1])))
        else:
            b, t = _net(e["branch"]), _net(e["trunk"])
            count = W.deeponet_param_count(b, t)
            prob = W.Problem(name, W.KIND_DEEPONET, 1.0, 1.0, np.zeros(count), np.zeros(count, np.uint8),
                             np.zeros((1, 0)), 1e-3, 1, branch=b, trunk=t,
                             u=np.zeros((0, e["branch"][0])), yq=np.zeros((0, e["trunk"][0])),
                             t=np.zeros((0, 0)))
        assert count == e["count"], name
        assert oracle.Oracle(prob).param_count() == e["count"], name


def test_workload_shapes():
    p = W.tiny_bnn()
    assert (p.P, p.k, p.x.shape, p.chains, p.L, p.eps) == (481, 481, (256, 1), 1, 20, 1e-3)
    p = W.wide_mlp()
    assert (p.P, p.k, p.x.shape, p.chains, p.L) == (198401, 9920, (8192, 2), 16, 50)
    p = W.deeponet_grf()
    assert (p.P, p.k, p.u.shape, p.yq.shape, p.t.shape, p.chains, p.L) == \
        (95873, 9587, (500, 100), (100, 2), (500, 100), 32, 30)
    p = W.cone_deeponet(n_u=16, chains=2)
    assert (p.P, p.k, p.yq.shape) == (331521, 33152, (8192, 2))
    probs = W.batched_uneven()
    assert len(probs) == 64
    for q in probs:
        assert q.notes["width"] in (32, 64, 128, 256) and 2 <= q.notes["hidden_layers"] <= 4
        assert 128 <= q.x.shape[0] <= 4096 and q.chains == 8 and q.L == 40
        assert q.k == int(np.floor(q.notes["frac"] * q.P))


def test_inputs_are_float32_representable_and_seeded():
    a, b = W.wide_mlp(n=512, chains=2), W.wide_mlp(n=512, chains=2)
    for x in (a.x, a.y, a.frozen, a.q0):
        assert np.array_equal(x, x.astype(np.float32).astype(np.float64))
    assert np.array_equal(a.q0, b.q0) and np.array_equal(a.mask, b.mask)
    assert np.array_equal(a.q0[0], a.frozen[a.mask.astype(bool)])
