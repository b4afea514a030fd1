#!/usr/bin/env python
"""Throughput of full-batch subset HMC on one GB300 (or N replicas on N GPUs).

Workload: the wide-MLP subset-HMC configuration -- MLP 2-256-256-256-256-1 with
tanh, 198,401 parameters, 8192 synthetic points (x ~ U[-1,1]^2,
y = sin(pi x1) cos(pi x2) + N(0, 0.05^2)), a 5% subset (9,920 parameters) chosen
by a seeded |N(0,1)| score, the rest frozen at seeded N(0, 0.05^2) values, prior
N(0, 1), noise sigma 0.05, 16 chains, L = 50 leapfrog steps of eps = 5e-4.

One step = one HMC trajectory for all chains: momentum draw, L x (drift with
the subset scatter, forward pass, energy, adjoint, gather, kick), kinetic
energy and the Metropolis step -- every row of the hot path.  The metric is
gradient evaluations per second (one grad-eval = U and grad U for one chain), so
value = chains * L * steps / time, summed over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload: one gradient evaluation per chain per step).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "grad-evals/s"
WORKLOAD = "wide_mlp: MLP 2-256-256-256-256-1 tanh, N=8192, 5% subset (k=9920), 16 chains, L=50, eps=5e-4"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _clock_sampler(stop, out):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return
    dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]

    def reader():
        for line in p.stdout:
            out.append(line.strip())

    t = threading.Thread(target=reader, daemon=True)
    t.start()
    stop.wait()
    p.terminate()
    try:
        p.wait(timeout=2)
    except subprocess.TimeoutExpired:
        p.kill()
    t.join(timeout=1)


def _summarise_clocks(lines, gpu_index):
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() in ("active", "1", "yes"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def cpu_baseline(prob, threads=None, chains=None):
    """The FP64 oracle as it stands: one gradient evaluation per chain, chains in parallel."""
    import oracle
    cores = threads or os.cpu_count() or 1
    C = chains or min(cores, prob.chains)
    o = oracle.Oracle(prob)
    Q = np.repeat(prob.q0[:1], C, axis=0) if C > prob.chains else prob.q0[:C]
    t0 = time.perf_counter()
    o.energy_grad_batch(Q, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": C / dt, "unit": METRIC, "cores": min(cores, C), "kind": "oracle",
            "sample": f"{C} gradient evaluations (one per chain) of the full workload, {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    prob = W.wide_mlp()
    secs, evals, cb = [], 0, None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_baseline(prob)
        if i >= args.warmup:
            secs.append(time.perf_counter() - t0)
            evals += int(cb["sample"].split()[0])
    value = evals / float(np.sum(secs))
    line = {"metric": METRIC, "value": value, "unit": METRIC, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD + " (oracle: one gradient evaluation per chain per step)"},
            "cpu_baseline": {**cb, "value": value},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _traffic(kernel):
    """DRAM bytes per launch of a bench kernel from the committed ncu capture, or None
    when there is none or the kernel's source text changed since it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
        if not rec:
            return None
        with open(os.path.join(ROOT, rec["source"]), encoding="utf-8") as f:
            text = f.read()
        i = text.index(rec["region_start"])           # the kernel's own source text
        j = text.index(rec["region_end"], i + len(rec["region_start"]))
        if hashlib.sha256(text[i:j].encode("utf-8")).hexdigest() != rec["region_sha256"]:
            return None
        return float(rec["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def algorithmic(prob, C):
    """Per-launch algorithmic FLOPs and DRAM bytes of each tensor-core kernel kind."""
    N, w = prob.x.shape[0], prob.net.widths[1]
    gemm = 2.0 * N * w * w * C
    act = 2.0 * N * w * C                     # one bf16 activation array, all chains
    wts = 2.0 * 2.0 * w * w * C               # bf16 hi + lo weights
    k_layer = prob.k / max(1, prob.net.n_layers)
    fwd = (gemm, act + act + wts)                              # read A_i, write A_{i+1}
    out = (gemm, act + act + wts + 4.0 * N)                    # read A_i, write delta, read y
    bwd = (gemm, 3 * act + wts / 2)                            # read delta, A_i; write delta_i (bf16 W)
    first = (gemm, 2 * act + wts / 2)                          # read delta, A_1
    dw = (gemm, 2 * act + 4.0 * k_layer * C)                   # read delta, A_i; sampled entries out
    return {
        "umma_fwd_tanh": fwd, "layer_fwd_tanh": fwd, "umma_fwd_out": out, "layer_fwd_out": out,
        "umma_bwd_tanh": bwd, "solo_bwd_tanh": bwd, "layer_bwd_tanh": bwd,
        "umma_bwd_first": first, "solo_bwd_first": first, "layer_bwd_first": first,
        "umma_dw": dw, "dw2": dw,
        "first_fwd": (2.0 * N * w * prob.x.shape[1] * C, act),
    }


def other_workloads(hmc, torch, steps=3):
    """The other synthetic workloads, timed the same way (one trajectory to capture the
    graph, one to size the timed run, then at least `steps` trajectories and about 0.3 s of
    them between CUDA events): grad-evals/s and acceptance."""
    from oracle.ess import ess_chains
    out = {}

    def timed(name, sp, q0, eps, L, chains_total, prec_name, ess_traj=0, ess_fn=None):
        q0 = torch.from_numpy(q0) if isinstance(q0, np.ndarray) else q0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sp.sample(q0, eps, L, 1, seed=5, keep_samples=False)   # captures the trajectory graph
        torch.cuda.synchronize()
        a.record()
        sp.sample(q0, eps, L, 1, seed=5, keep_samples=False)
        b.record()
        torch.cuda.synchronize()
        # at least `steps` trajectories and about 0.3 s of them, so that short trajectories
        # are not timed over a few milliseconds only
        n = int(min(50, max(steps, 300.0 / max(a.elapsed_time(b), 1e-3))))
        a.record()
        _, acc, dH, ql = sp.sample(q0, eps, L, n, seed=5, first_traj=1, keep_samples=False)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n
        eps_rec = float(eps) if np.ndim(eps) == 0 else {
            "per_problem": len(eps), "min": float(np.min(eps)), "median": float(np.median(eps)), "max": float(np.max(eps))}
        rec = {"dtype": prec_name, "chains": chains_total, "L": L, "eps": eps_rec, "ms_per_trajectory": ms,
               "timed_trajectories": n,
               "grad_evals_per_s": chains_total * L / (ms / 1000.0),
               "accept_rate": float(acc.float().mean().item()),
               "abs_dH_median": float(np.nanmedian(np.abs(dH.cpu().numpy())))}
        # kernels in one captured trajectory, and the time per kernel they average to (a
        # few microseconds apiece marks a workload bound by launches rather than bytes)
        kern = int(hmc.graph_kernels(sp))
        if kern > 0:
            rec.update({"kernels_per_trajectory": kern, "us_per_kernel": 1000.0 * ms / kern})
        if ess_traj:
            torch.cuda.synchronize()
            a.record()
            S, acc2, _, _ = sp.sample(ql, eps, L, ess_traj, seed=6, first_traj=100)
            b.record()
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1000.0
            Sn = S.cpu().double().numpy()[ess_traj // 5:]
            e = ess_fn(Sn) if ess_fn else ess_chains(Sn if Sn.ndim == 3 else Sn[:, None, :])
            rec.update({"ess_trajectories": ess_traj, "ess_min": float(e.min()), "ess_min_per_s": float(e.min()) / sec,
                        "ess_median_per_s": float(np.median(e)) / sec,
                        "ess_accept_rate": float(acc2.float().mean().item()),
                        "chains_never_accepting": int((acc2.cpu().numpy().sum(axis=0) == 0).sum())})
        out[name] = rec
        sp.close()

    p = W.tiny_bnn()
    timed("tiny_bnn_fp64", hmc.Sampler.mlp(p.net.widths, p.x, p.y, p.mask, p.frozen, 1, prior_sigma=p.prior_sigma,
                                           noise_sigma=p.noise_sigma, prec=hmc.PREC_FP64),
          p.q0, p.eps, p.L, 1, "f64", ess_traj=200)
    # The DeepONets run at their workloads' fixed steps: their chains start at random frozen
    # weights, far from any fit (U about 1e7 for the GRF one, 3e9 for the cone), where a
    # dual-averaging warm-up drives the step toward zero; their throughput does not depend
    # on the step
    p = W.deeponet_grf()
    for nm, pr in (("bf16", hmc.PREC_BF16), ("fp16", hmc.PREC_FP16)):
        sp = hmc.Sampler.deeponet(p.branch.widths, p.trunk.widths, p.u, p.yq, p.t, p.mask, p.frozen, p.chains,
                                  prior_sigma=p.prior_sigma, noise_sigma=p.noise_sigma, prec=pr)
        timed("deeponet_grf_" + nm, sp, p.q0, p.eps, p.L, p.chains, nm)
    probs = W.batched_uneven()
    tup = [(q.net.widths, q.x, q.y, q.mask, q.frozen, q.prior_sigma, q.noise_sigma) for q in probs]
    q0 = np.concatenate([q.q0.reshape(-1) for q in probs])   # packed [problem][chain][k_problem]
    # grouped launches (the default), then every problem launching its own kernels on the
    # batch's concurrent lanes, for comparison; each problem's step adapted first (the
    # problems differ too much for one common step), the warm-up untimed
    bs = hmc.BatchSampler(tup, probs[0].chains, hmc.PREC_BF16)
    groups = bs.groups()
    n_warm = 100
    eps_b, q_b = bs.adapt_step_size(torch.from_numpy(q0.astype(np.float32)), probs[0].L, probs[0].eps, n_warm,
                                    target_accept=0.8, seed=71)
    C = probs[0].chains

    def ess_per_problem(Sn):   # each problem's 8 chains together, every coordinate; packed [n][problem][C][k]
        out_e, off = [], 0
        for q in probs:
            out_e.append(ess_chains(Sn[:, off:off + C * q.k].reshape(Sn.shape[0], C, q.k)))
            off += C * q.k
        return np.concatenate(out_e)

    timed("batched_uneven_bf16", bs, q_b, eps_b, probs[0].L, len(probs) * C, "bf16", ess_traj=100,
          ess_fn=ess_per_problem)
    out["batched_uneven_bf16"]["groups"] = groups
    out["batched_uneven_bf16"]["warmup_trajectories"] = n_warm
    timed("batched_uneven_bf16_per_problem_launches", hmc.BatchSampler(tup, probs[0].chains, hmc.PREC_BF16,
                                                                       grouped=False),
          q_b, eps_b, probs[0].L, len(probs) * probs[0].chains, "bf16")
    p = W.cone_deeponet()
    sp = hmc.Sampler.deeponet(p.branch.widths, p.trunk.widths, p.u, p.yq, p.t, p.mask, p.frozen, p.chains,
                              prior_sigma=p.prior_sigma, noise_sigma=p.noise_sigma, prec=hmc.PREC_BF16)
    timed("cone_deeponet_bf16", sp, p.q0, p.eps, p.L, p.chains, "bf16")
    return out


def gradients_only(name, n, chains=0):
    """U and grad U of the named workload n times (BF16), for profiling; `chains` > 0
    replaces a single-problem workload's chain count (a smaller capture)."""
    import torch
    import paper_2507_14652_gb300 as hmc
    if name == "wide_mlp":
        p = W.wide_mlp()
        if chains:
            p.q0 = np.ascontiguousarray(p.q0[:chains])
        s = hmc.Sampler.mlp(p.net.widths, p.x, p.y, p.mask, p.frozen, p.chains, prior_sigma=p.prior_sigma,
                            noise_sigma=p.noise_sigma, prec=hmc.PREC_BF16)
        q = torch.from_numpy(p.q0).float().cuda()
    elif name == "batched_uneven":
        probs = W.batched_uneven()
        s = hmc.BatchSampler([(p.net.widths, p.x, p.y, p.mask, p.frozen, p.prior_sigma, p.noise_sigma)
                              for p in probs], probs[0].chains, hmc.PREC_BF16)
        q = torch.from_numpy(np.concatenate([p.q0.reshape(-1) for p in probs]).astype(np.float32)).cuda()
    else:
        p = W.deeponet_grf() if name == "deeponet_grf" else W.cone_deeponet()
        if chains:
            p.q0 = np.ascontiguousarray(p.q0[:chains])
        s = hmc.Sampler.deeponet(p.branch.widths, p.trunk.widths, p.u, p.yq, p.t, p.mask, p.frozen, p.chains,
                                 prior_sigma=p.prior_sigma, noise_sigma=p.noise_sigma, prec=hmc.PREC_BF16)
        q = torch.from_numpy(p.q0).float().cuda()
    for _ in range(n):
        s.energy_grad(q)
    torch.cuda.synchronize()
    s.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ess-traj", type=int, default=200, help="trajectories for the ESS/s comparison (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--split", type=int, default=4, help="data batches of the split-integrator run (0 = skip)")
    ap.add_argument("--no-around", action="store_true", help="skip the sensitivity/truncation/predictive timings")
    ap.add_argument("--no-other", action="store_true", help="skip the other workloads (tiny BNN, DeepONets, batch)")
    ap.add_argument("--gradients-only", choices=["wide_mlp", "batched_uneven", "deeponet_grf", "cone_deeponet"],
                    help="build the workload's handle, run --steps gradient evaluations and exit (a short "
                         "program for ncu launch lists and captures; prints no bench line)")
    ap.add_argument("--chains", type=int, default=0, help="with --gradients-only: chains (0 = the workload's)")
    args = ap.parse_args()
    assert args.warmup >= 3, "timing rules need at least 3 warm-up steps"
    if args.impl == "reference":
        return run_reference(args)
    if args.gradients_only:
        return gradients_only(args.gradients_only, args.steps, args.chains)

    import torch
    import paper_2507_14652_gb300 as hmc
    from paper_2507_14652_gb300.replicas import job_rate, reduce_max, replica_seed

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hmc.lib()

    prob = W.wide_mlp()
    C, L, eps = prob.chains, prob.L, prob.eps
    seed = replica_seed(rank)               # replicas: independent chains per rank
    s = hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, C, prior_sigma=prob.prior_sigma,
                        noise_sigma=prob.noise_sigma, prec=hmc.PREC_BF16)
    q0 = torch.from_numpy(prob.q0).float().cuda()

    # warm-up (captures the trajectory graph)
    _, acc_w, dH_w, q = s.sample(q0, eps, L, args.warmup, seed=seed)
    torch.cuda.synchronize()

    # timed region: exactly `steps` trajectories
    clock_lines, stop = [], threading.Event()
    th = threading.Thread(target=_clock_sampler, args=(stop, clock_lines), daemon=True)
    th.start()
    time.sleep(0.5)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    S, acc, dH, q_last = s.sample(q, eps, L, args.steps, seed=seed, first_traj=args.warmup)
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stop.set()
    th.join(timeout=5)
    ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    value = job_rate(ws, C * L * args.steps, ms / 1000.0)
    graph_k = hmc.graph_kernels(s)
    acc_np, dH_np = acc.cpu().numpy(), dH.cpu().numpy()

    # live per-kernel times on the library's stream (roofline of the dominant kernel)
    prof = hmc.profile_energy_grad(s, q_last, reps=5)
    per_eval_launches = int(round(sum(v[1] for v in prof.values())))
    gpu_launches = args.steps * graph_k + per_eval_launches + 1
    peaks, peak_src = _peaks()
    alg = algorithmic(prob, C)
    dom = max(prof, key=lambda k: prof[k][0] * prof[k][1])
    roof = None
    if dom in alg:
        fl, by = alg[dom]
        t_ms = prof[dom][0]
        t_hbm = by / (peaks["hbm_gbs"] * 1e9)
        t_tc = fl / (peaks["bf16_tflops_sustained"] * 1e12)
        if t_hbm >= t_tc:
            ach = by / (t_ms / 1e3) / 1e9
            roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"], "traffic": _traffic(dom),
                    "peak_source": peak_src + " (hbm_gbs)"}
        else:
            ach = fl / (t_ms / 1e3) / 1e12
            roof = {"kernel": dom, "bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops_sustained"],
                    "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops_sustained"], "traffic": None,
                    "peak_source": peak_src + " (bf16_tflops_sustained)"}
        roof["kernel_ms"] = t_ms
    # the same arithmetic for every kernel kind of the evaluation (context for the dominant one)
    roof_all = {}
    for name, (t_k, _n) in prof.items():
        if name not in alg:
            continue
        fl, by = alg[name]
        t_hbm = by / (peaks["hbm_gbs"] * 1e9)
        t_tc = fl / (peaks["bf16_tflops_sustained"] * 1e12)
        frac = max(t_hbm, t_tc) / (t_k / 1e3)
        roof_all[name] = {"bound": "hbm" if t_hbm >= t_tc else "tensor", "kernel_ms": t_k,
                          "floor_ms": 1e3 * max(t_hbm, t_tc), "frac": frac, "traffic": _traffic(name)}

    # end to end through the public C ABI with pinned host buffers: every step copies
    # the chain state in and the step's sample, accept flags and dH out
    qh = torch.empty((C, prob.k), dtype=torch.float32, pin_memory=True)
    qh.copy_(q_last.cpu())
    Sh = torch.empty((1, C, prob.k), dtype=torch.float32, pin_memory=True)
    ah = torch.empty((1, C), dtype=torch.uint8, pin_memory=True)
    dh = torch.empty((1, C), dtype=torch.float64, pin_memory=True)
    L_ = hmc.lib()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        st = L_.hmc_sample(s._h, qh.data_ptr(), float(eps), int(L), 1, int(seed), int(args.warmup + args.steps + i),
                           Sh.data_ptr(), ah.data_ptr(), dh.data_ptr(), qh.data_ptr())
        if st != 0:
            raise hmc.HmcError(st, L_.hmc_last_error().decode())
    t_e2e = reduce_max(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": job_rate(ws, C * L * args.steps, t_e2e), "unit": METRIC, "h2d_bytes_per_step": 4 * C * prob.k,
           "d2h_bytes_per_step": 4 * C * prob.k + C + 8 * C + 4 * C * prob.k}

    # The same timed trajectories with the fp16 tensor-core engine (same kernels and
    # bytes, 11 significant bits against bf16's 8): its throughput and acceptance
    s16 = hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, C, prior_sigma=prob.prior_sigma,
                          noise_sigma=prob.noise_sigma, prec=hmc.PREC_FP16)
    s16.sample(q0, eps, L, args.warmup, seed=seed)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    _, acc16, dH16, _ = s16.sample(q, eps, L, args.steps, seed=seed, first_traj=args.warmup)
    b.record()
    torch.cuda.synchronize()
    ms16 = a.elapsed_time(b)
    fp16 = {"value": job_rate(1, C * L * args.steps, ms16 / 1000.0), "ms_per_step": ms16 / args.steps,
            "accept_rate": float(acc16.float().mean().item()),
            "abs_dH_median": float(np.nanmedian(np.abs(dH16.cpu().numpy())))}

    # ESS/s and acceptance at one step size: the step is adapted by dual averaging to ~80%
    # acceptance on the batched fp16 sampler during a warm-up (a fixed eps that suits the
    # start of the chains rejects nearly everything once they reach the sharper posterior
    # mode).  Then, at that step:
    # * acceptance on paired starts: states visited by the fp16 chains, and from each, one
    #   trajectory per precision with the same momenta and uniforms (same seed and index),
    #   so the mean acceptance probabilities min(1, exp(-dH)) differ only by the forces;
    # * ESS/s of chains from the warmed-up states (same seed and indices): batched fp16 and
    #   bf16, the batched FP32 CUDA-core sampler and the plain one-chain FP32 sampler (on
    #   the chain whose paired FP32 acceptance is the median one).
    ess = None
    if args.ess_traj > 0 and rank == 0:
        from oracle.ess import ess_chains
        n_adapt = max(20, args.ess_traj // 4)
        eps_ad, q_ad = s16.adapt_step_size(q_last, L, eps, n_adapt, target_accept=0.8, seed=seed + 77,
                                           first_traj=10 ** 6)
        ess = {"eps_adapted": eps_ad, "adapted_on": "fp16_batched", "adapt_trajectories": n_adapt,
               "target_accept": 0.8}
        s32 = hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, C,
                              prior_sigma=prob.prior_sigma, noise_sigma=prob.noise_sigma, prec=hmc.PREC_FP32)

        def acc_prob(d):
            d = d.cpu().numpy().ravel()
            return np.where(np.isfinite(d), np.minimum(1.0, np.exp(-np.nan_to_num(d, nan=0.0, posinf=0.0))), 0.0)

        n_start = 12
        Sst, _, _, _ = s16.sample(q_ad, eps_ad, L, 3 * n_start, seed=seed + 55, first_traj=3 * 10 ** 6)
        paired = {"starts": n_start, "trajectories_per_start": 1}
        ap = {}
        for name, sp in (("fp16", s16), ("bf16", s), ("fp32", s32)):
            a, dd = [], []
            for t in range(n_start):
                _, _, d, _ = sp.sample(Sst[3 * t + 2].contiguous(), eps_ad, L, 1, seed=seed + 99,
                                       first_traj=4 * 10 ** 6 + t, keep_samples=False)
                a.append(acc_prob(d))
                dd.append(np.abs(d.cpu().numpy().ravel()))
            ap[name] = np.stack(a)                                    # [start][chain]
            paired[name] = {"mean_accept_prob": float(ap[name].mean()),
                            "abs_dH_median": float(np.nanmedian(np.concatenate(dd)))}
        for name in ("fp16", "bf16"):
            diff = (ap[name] - ap["fp32"]).ravel()
            paired[name]["minus_fp32"] = float(diff.mean())
            paired[name]["minus_fp32_se"] = float(diff.std(ddof=1) / np.sqrt(diff.size))
        ess["paired_acceptance"] = paired
        c1 = int(np.argsort(ap["fp32"].mean(axis=0))[C // 2])      # the median chain
        ess["plain_chain"] = c1
        arms = (("fp16_batched", s16, None, args.ess_traj), ("bf16_batched", s, None, args.ess_traj),
                ("fp32_batched", s32, None, max(10, args.ess_traj // 5)),
                ("fp32_plain_1chain", None, c1, max(10, args.ess_traj // 2)))
        for name, sp, one, ntraj in arms:
            if sp is None:
                sp = hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, 1,
                                     prior_sigma=prob.prior_sigma, noise_sigma=prob.noise_sigma, prec=hmc.PREC_FP32)
            qs = (q_ad if one is None else q_ad[one:one + 1]).contiguous()
            chains = qs.shape[0]
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            Se, ae, de, _ = sp.sample(qs, eps_ad, L, ntraj, seed=seed + 77, first_traj=10 ** 6 + n_adapt)
            b.record()
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) / 1000.0
            e = ess_chains(Se.cpu().double().numpy()[ntraj // 5:])
            ess[name] = {"chains": chains, "trajectories": ntraj, "seconds": sec,
                         "ess_min": float(e.min()), "ess_median": float(np.median(e)),
                         "ess_min_per_s": float(e.min()) / sec, "ess_median_per_s": float(np.median(e)) / sec,
                         "accept_rate": float(ae.float().mean().item()),
                         "mean_accept_prob": float(acc_prob(de).mean()),
                         "abs_dH_median": float(np.nanmedian(np.abs(de.cpu().numpy()))),
                         "grad_evals_per_s": chains * L * ntraj / sec}
        # executed work of the FP32 CUDA-core engine per chain-evaluation: the forward GEMMs,
        # the input adjoints and the dense weight gradients (every weight's entry, then the
        # sampled ones are gathered), 2 flops per multiply-add; its peak is the CUDA cores'
        # FP32 rate from unit counts and clock: 152 SMs x 128 lanes x 2 flops x max clock
        w = prob.net.widths
        fl = 2.0 * prob.x.shape[0] * sum(w[l] * w[l + 1] for l in range(len(w) - 1))
        fl_exec = fl + fl + (fl - 2.0 * prob.x.shape[0] * w[0] * w[1])
        clk = (peaks.get("sm_max_mhz") or 2070.0) * 1e6
        fp32_peak = 152 * 128 * 2 * clk / 1e12
        for name in ("fp32_batched", "fp32_plain_1chain"):
            tf = ess[name]["grad_evals_per_s"] * fl_exec / 1e12
            ess[name].update({"executed_tflops": tf, "fp32_cuda_core_peak_tflops": fp32_peak,
                              "fp32_peak_frac": tf / fp32_peak})
        s32.close()

    # the symmetric split integrator over data batches on the same workload and step:
    # trajectories of the same L, each step 2M - 1 batch gradients of N/M points
    split = None
    if args.split > 1 and rank == 0:
        M = args.split
        ss = hmc.Sampler.mlp(prob.net.widths, prob.x, prob.y, prob.mask, prob.frozen, C,
                             prior_sigma=prob.prior_sigma, noise_sigma=prob.noise_sigma, prec=hmc.PREC_BF16,
                             n_splits=M)
        # the same start state, momenta and uniforms as the timed leapfrog run, so the
        # acceptance rates compare the two integrators on the same trajectories' starts
        ss.sample(q, eps, L, 1, seed=seed, first_traj=10 ** 7, keep_samples=False)   # graph capture
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, acs, dhs, _ = ss.sample(q, eps, L, args.steps, seed=seed, first_traj=args.warmup, keep_samples=False)
        b.record()
        torch.cuda.synchronize()
        sms = a.elapsed_time(b) / args.steps
        split = {"n_splits": M, "ms_per_trajectory": sms, "leapfrog_ms_per_trajectory": ms / args.steps,
                 "batch_gradients_per_step": 2 * M - 1, "points_per_batch": int(prob.x.shape[0]) // M,
                 "accept_rate": float(acs.float().mean().item()), "leapfrog_accept_rate": float(acc_np.mean()),
                 "abs_dH_median": float(np.nanmedian(np.abs(dhs.cpu().numpy()))),
                 "full_gradient_equivalents_per_s": C * L * (2 * M - 1) / M / (sms / 1000.0)}
        ss.close()

    # the steps around the sampler on the same workload: sensitivities of all P
    # parameters at the frozen values (FP32), the tau = 0.9 truncation, and the
    # posterior predictive of 256 samples on the 8192 training inputs
    around = None
    if rank == 0 and not args.no_around:
        mu = torch.from_numpy(prob.frozen).cuda()
        sd = torch.full_like(mu, 0.05)
        hmc.sensitivity_mlp(prob.net.widths, prob.x, mu, sd)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S2 = hmc.sensitivity_mlp(prob.net.widths, prob.x, mu, sd)
        torch.cuda.synchronize()
        t_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        nhat, _, _ = hmc.select_subset(S2, 0.9)
        torch.cuda.synchronize()
        t_sel = time.perf_counter() - t0
        Sp = q.repeat(16, 1)                                       # 256 samples
        s.predict(Sp[:16], x=prob.x)                               # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, rel = s.predict(Sp, x=prob.x, y=prob.y)
        torch.cuda.synchronize()
        t_p = time.perf_counter() - t0
        around = {"sensitivity": {"params": prob.P, "points": int(prob.x.shape[0]), "dtype": "f32", "ms": 1e3 * t_s},
                  "select_subset": {"params": prob.P, "tau": 0.9, "n_hat": nhat, "ms": 1e3 * t_sel},
                  "predict": {"samples": int(Sp.shape[0]), "points": int(prob.x.shape[0]), "dtype": "f32",
                              "ms": 1e3 * t_p, "samples_per_s": Sp.shape[0] / t_p, "rel_l2": rel}}

    other = None
    if rank == 0 and not args.no_other:
        other = other_workloads(hmc, torch)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob)

    clocks = _summarise_clocks(clock_lines, local)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": {"workload": WORKLOAD, "chains": C, "leapfrog_steps": L, "eps": eps,
                           "subset_k": prob.k, "params": prob.P, "points": int(prob.x.shape[0]),
                           "step": "one HMC trajectory for all chains (L gradient evaluations each)",
                           "l2": "inputs larger than L2: 0.4 GB of bf16 activations and deltas per gradient evaluation",
                           "samples": "every trajectory's samples are written to device memory in the timed region",
                           "parallelism": f"replicas x{ws}"},
                "accept_rate": float(acc_np.mean()), "abs_dH_mean": float(np.nanmean(np.abs(dH_np))),
                "abs_dH_median": float(np.nanmedian(np.abs(dH_np))),
                "gpu_launches": gpu_launches, "kernels_per_trajectory": graph_k,
                "roofline": roof, "roofline_by_kernel": roof_all, "kernel_ms": {k: v[0] for k, v in prof.items()},
                "tuning": s.tuning().strip(),
                "kernel_launches_per_eval": {k: v[1] for k, v in prof.items()},
                "e2e": e2e, "cpu_baseline": cpu, "fp16": fp16, "ess": ess, "split_hmc": split,
                "around_the_sampler": around, "other_workloads": other,
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
