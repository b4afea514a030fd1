"""CPU tests of bench.py's measurement helpers (no GPU).

* The algorithmic FLOPs and bytes per launch behind the roofline fractions, against hand
  counts for the wide-MLP workload (N = 8192 points, width 256, 16 chains, bf16 arrays).
* The nvidia-smi clock record: median SM clock, maximum, and the throttle reasons that
  decide whether a run is rejected.
* The recorded ncu DRAM traffic is returned only while the kernel's source text is the
  one that was profiled.
"""
import hashlib
import json
import os

import pytest

import bench
import workloads as W


def test_algorithmic_counts_of_the_wide_mlp():
    prob = W.wide_mlp()
    alg = bench.algorithmic(prob, 16)
    N, w, C = 8192, 256, 16
    act = 2 * N * w * C                      # one bf16 activation array of all chains: 64 MiB
    assert act == 67_108_864
    gemm = 2 * N * w * w * C                 # one hidden layer's product: 17.2 GFLOP
    w_hilo = 2 * 2 * w * w * C               # bf16 hi and lo weights of all chains
    assert alg["layer_fwd_tanh"] == (gemm, 2 * act + w_hilo)
    assert alg["layer_fwd_out"] == (gemm, 2 * act + w_hilo + 4 * N)
    assert alg["layer_bwd_tanh"] == (gemm, 3 * act + w_hilo / 2)
    assert alg["layer_bwd_first"] == (gemm, 2 * act + w_hilo / 2)
    k_layer = prob.k / 5                     # the sampled entries spread over five layers
    assert alg["dw2"] == (gemm, 2 * act + 4 * k_layer * C)
    assert alg["first_fwd"] == (2 * N * w * 2 * C, act)


def test_clock_summary_flags_throttling():
    # index, clocks.sm, clocks.max.sm, power.draw, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2070, 2070, 900.0 W, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 950.0 W, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 960.0 W, 0x0, Not Active, Not Active, Not Active, Not Active",
             "index, clocks.sm [MHz], ..."]
    c = bench._summarise_clocks(lines, 0)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    c = bench._summarise_clocks(["0, 1200, 2070, 1 W, 0x8, Active, Not Active, Not Active, Not Active"], 0)
    assert c["reasons"] == ["hw_slowdown"] and c["sm_mhz"] == 1200.0
    assert bench._summarise_clocks([], 0) is None


def test_traffic_is_dropped_once_the_kernel_changes(tmp_path, monkeypatch):
    src = "head\n__global__ void k_x(int a)\n{\n    body;\n}\ntail\n"
    (tmp_path / "k.cu").write_text(src)
    start, end = "__global__ void k_x(", "\n}\n"
    i = src.index(start)
    j = src.index(end, i + len(start))
    rec = {"k": {"kernel": "k_x", "dram_bytes_per_launch": 1234, "source": "k.cu", "region_start": start,
                 "region_end": end, "region_sha256": hashlib.sha256(src[i:j].encode()).hexdigest()}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("k") == 1234.0
    assert bench._traffic("other") is None
    (tmp_path / "k.cu").write_text(src.replace("body;", "body2;"))
    assert bench._traffic("k") is None


def test_committed_traffic_records_name_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)
    for name, rec in recs.items():
        if name.startswith("_"):
            continue
        text = open(os.path.join(bench.ROOT, rec["source"]), encoding="utf-8").read()
        assert rec["region_start"] in text, name
        assert os.path.exists(os.path.join(bench.ROOT, rec["capture"])), name
        assert rec["dram_bytes_per_launch"] > 0
