#!/usr/bin/env python
"""Benchmark: population-wide SR fitness (forward + MSE) on one GB300.

One step = one pass of the fitness hot path over one population: validate
and compile the trees, evaluate every tree on every data point, reduce the
squared residuals to a per-tree MSE.  Workload (default): 5,000 random trees
of length <= 255 (depth <= 8), 16 float32 features N(0,1), 100,000 points,
targets from a length-31 ground-truth tree plus N(0, 0.01^2) noise.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is node-point evaluations per second
(GPops/s with one generation, Sec. V-C) over the whole job with inputs
resident in HBM; `e2e` is the same metric through the C ABI from pinned host
buffers with the copies inside the timed region; `roofline` relates the
evaluation kernel to the FP32/SFU issue and HBM roofline; `cpu_baseline` is
the FP64 oracle on the host cores on a bounded sample of the same workload.
`--impl reference` times that oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "node·point evals/sec and % roofline for population MSE fitness; fwd+bwd time"
UNIT = "node·point evals/s"
L2_FLUSH_BYTES = 256 << 20

# Algorithmic instruction counts per node-point (one lane-op each) and SFU
# cost in SM cycles per lane-op: sin, cos, lg2 and rcp issue at 16 lanes per
# SM per clock on GB300, ex2 (ftz) at 32 (measured).  Leaves cost nothing.
FP32_OPS = {0: 1, 1: 1, 2: 1, 3: 2, 4: 1, 5: 1, 6: 1, 7: 2, 8: 2, 9: 2}
SFU_CYC = {3: 1 / 16, 5: 1 / 16, 6: 1 / 16, 7: 1 / 16, 8: 1 / 32, 9: 3 / 16}
MSE_FP32_PER_POINT = 2
# Extra algorithmic work of the reverse sweep per function node-point: the
# local derivatives and adjoint products (add/sub pass the adjoint through;
# pdiv reuses the reciprocal of the forward; sin/cos need the other of the
# pair; plog one reciprocal; tan 1 + t^2), one accumulate per constant or
# feature leaf, and the seed 2 g (o - y) / D per point and output.
ADJ_FP32_OPS = {0: 0, 1: 0, 2: 2, 3: 4, 4: 1, 5: 1, 6: 1, 7: 1, 8: 1, 9: 2}
ADJ_SFU_CYC = {5: 1 / 16, 6: 1 / 16, 7: 1 / 16}
ADJ_LEAF_FP32 = 1
ADJ_SEED_FP32_PER_POINT = 2


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sr_scale", choices=["sr_scale"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pop", type=int, default=5000, help="trees (smaller cases for profiling)")
    ap.add_argument("--points", type=int, default=100_000, help="data points")
    ap.add_argument("--no-parts", action="store_true",
                    help="skip the metric's other parts in the default line (forward + adjoint on "
                         "the differentiation workload, the autotuned uneven batch, the Modi "
                         "workload)")
    ap.add_argument("--suite", action="store_true",
                    help="also time the other workloads (one JSON line each, after the main line)")
    ap.add_argument("--case", default=None,
                    choices=["adjoint", "modi", "batched", "genetic", "sweep", "e1"],
                    help="time only one case for profiling: the fused forward + adjoint on the "
                         "differentiation workload or the Modi forward (--pop/--points), the "
                         "8-problem uneven batch (one batched call, then one call per problem), "
                         "the genetic operators (crossover, selection, one generation), or the "
                         "fitness throughput over the paper's population x data set grid")
    return ap.parse_args()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def _workload_desc(prob):
    return (f"{prob.name}: {prob.pop.pop} random trees, length<=255 (depth<=8), "
            f"{prob.F} float32 features N(0,1), {prob.D} points, y = GT(len 31) + N(0,0.01^2); "
            f"forward + MSE")


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- helpers
def _src_hash():
    h = hashlib.sha256()
    for f in ("eval.cu", "stage.cu", "tgp_internal.cuh", "interp_fwd.cuh", "isa_fwd.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2501_17168_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _profile_traffic(workload):
    """DRAM bytes per launch of the evaluation kernel from the committed ncu
    summary, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"eval_kernel_{workload}.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != _src_hash():
        return None
    return float(t.group(1))


def _roofline_time(pop, D, sms, f_hz, hbm_gbs, n_outputs=1):
    """FP32-issue and SFU-issue times of one evaluation pass at the given clock."""
    n_fp32 = 0.0
    n_sfu = 0.0
    t, v = pop.type, pop.val
    L = pop.lengths()
    mask = np.arange(pop.ld)[None, :] < L[:, None]
    fn = mask & ((t == 2) | (t == 3) | (t == 18) | (t == 19))
    ids, counts = np.unique(np.mod(v[fn].astype(np.int64), 256), return_counts=True)
    for f, c in zip(ids, counts):
        n_fp32 += FP32_OPS[int(f)] * c * D
        n_sfu += SFU_CYC.get(int(f), 0.0) * c * D
    n_fp32 += MSE_FP32_PER_POINT * pop.pop * n_outputs * D
    t_fp32 = n_fp32 / (sms * 128 * f_hz)
    t_sfu = n_sfu / (sms * f_hz)
    return t_fp32, t_sfu


def _roofline_time_fwd_bwd(pop, D, sms, f_hz, n_outputs=1):
    """FP32-issue and SFU-issue times of one fused forward + adjoint pass."""
    t_fp32, t_sfu = _roofline_time(pop, D, sms, f_hz, 0.0, n_outputs)
    n_fp32, n_sfu = 0.0, 0.0
    t, v = pop.type, pop.val
    L = pop.lengths()
    mask = np.arange(pop.ld)[None, :] < L[:, None]
    fn = mask & ((t == 2) | (t == 3) | (t == 18) | (t == 19))
    ids, counts = np.unique(np.mod(v[fn].astype(np.int64), 256), return_counts=True)
    for f, c in zip(ids, counts):
        n_fp32 += ADJ_FP32_OPS[int(f)] * c * D
        n_sfu += ADJ_SFU_CYC.get(int(f), 0.0) * c * D
    n_leaf = int((mask & ((t == 0) | (t == 1))).sum())
    n_fp32 += ADJ_LEAF_FP32 * n_leaf * D + ADJ_SEED_FP32_PER_POINT * pop.pop * n_outputs * D
    return t_fp32 + n_fp32 / (sms * 128 * f_hz), t_sfu + n_sfu / (sms * f_hz)


def _bytes_once(pop, D, F, n_outputs=1):
    return 4.0 * D * F + 4.0 * D * n_outputs + 12.0 * pop.pop * pop.ld + 8.0 * pop.pop * n_outputs


# ----------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    import oracle
    from paper_2501_17168_gb300 import workloads as W
    if rank != 0:
        return 0
    prob = W.sr_scale(0, pop=a.pop, D=a.points)
    cores = os.cpu_count() or 1
    # bounded sample: every 50th tree over all points (about 1e9 node-points)
    pick = np.arange(0, prob.pop.pop, 50)
    sub = prob.pop.take(pick)
    gt, _ = oracle.evaluate(prob.gt.type, prob.gt.val, prob.gt.size, prob.X, threads=cores)
    y = (gt[0, 0] + prob.noise[:, 0]).astype(np.float32)
    units = float(sub.nodes()) * prob.D
    for _ in range(a.warmup):
        oracle.mse(sub.type, sub.val, sub.size, prob.X, y, threads=cores)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        oracle.mse(sub.type, sub.val, sub.size, prob.X, y, threads=cores)
        times.append(time.perf_counter() - t0)
    T = sum(times)
    value = units * a.steps / T
    sample = f"every 50th tree ({sub.pop} trees, {sub.nodes()} nodes) x all {prob.D} points"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * T / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": _workload_desc(prob), "pop": prob.pop.pop,
                                        "n_points": prob.D, "n_features": prob.F},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- our arm
def cpu_baseline(prob, seconds_target=15.0):
    import oracle
    cores = os.cpu_count() or 1
    gt, _ = oracle.evaluate(prob.gt.type, prob.gt.val, prob.gt.size, prob.X, threads=cores)
    y = (gt[0, 0] + prob.noise[:, 0]).astype(np.float32)
    # calibrate on a slice with a few trees per core, then time a sample of
    # about seconds_target
    pick = np.arange(0, prob.pop.pop, max(1, prob.pop.pop // (4 * cores)))
    sub = prob.pop.take(pick)
    t0 = time.perf_counter()
    oracle.mse(sub.type, sub.val, sub.size, prob.X, y, threads=cores)
    rate = sub.nodes() * prob.D / max(time.perf_counter() - t0, 1e-6)
    n_trees = int(min(prob.pop.pop, max(cores, rate * seconds_target / (prob.pop.nodes() / prob.pop.pop * prob.D))))
    stride = max(1, prob.pop.pop // n_trees)
    sub = prob.pop.take(np.arange(0, prob.pop.pop, stride))
    t0 = time.perf_counter()
    oracle.mse(sub.type, sub.val, sub.size, prob.X, y, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": sub.nodes() * prob.D / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"every {stride}th tree ({sub.pop} trees, {sub.nodes()} nodes) x all {prob.D} "
                      f"points, {dt:.1f} s wall"}


def run_ours(a, rank, world, local_rank):
    import torch
    from paper_2501_17168_gb300 import api, build, workloads as W
    build.build_all()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = W.sr_scale(rank, pop=a.pop, D=a.points)
    t, v, s = api.population_to(prob.pop, dev)
    X = torch.from_numpy(prob.X).to(dev)
    # targets: ground-truth tree evaluated by the library, plus noise
    gt_t, gt_v, gt_s = api.population_to(prob.gt, dev)
    gy, _ = api.tgp_eval_forward(gt_t, gt_v, gt_s, X, 1, max_len=prob.gt.max_len)
    y = (gy[0, 0] + torch.from_numpy(prob.noise[:, 0]).to(dev)).contiguous().view(-1, 1)
    P, D, F = prob.pop.pop, prob.D, prob.F
    mse = torch.empty((P, 1), dtype=torch.float64, device=dev)
    st = torch.empty(P, dtype=torch.int32, device=dev)
    units = float(prob.pop.nodes()) * D
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(cfg=None):
        api.tgp_fitness_mse(t, v, s, X, y, 1, max_len=prob.pop.max_len, config=cfg, mse=mse,
                            tree_status=st)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    api.tgp_check_device_error(dev)
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        time.sleep(0.3)
        for i in range(a.steps):
            flush.zero_()  # L2 flush outside the timed events
            ev[i][0].record()
            step({"eval_begin_event": ev[i][2], "eval_end_event": ev[i][3]})
            ev[i][1].record()
        torch.cuda.synchronize()
    api.tgp_check_device_error(dev)
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    eval_ms = [e[2].elapsed_time(e[3]) for e in ev]
    T = sum(step_ms) / 1e3
    if world > 1:
        tt = torch.tensor([T], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        T = float(tt.item())
    total_units = units * a.steps * world
    value = total_units / T
    assert (st.cpu().numpy() == 0).all()

    result = None
    if rank == 0:
        hbm_gbs, sm_max_mhz, peak_kind = _peaks()
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        f_hz = sm_max_mhz * 1e6
        t_fp32, t_sfu = _roofline_time(prob.pop, D, sms, f_hz, hbm_gbs)
        nbytes = _bytes_once(prob.pop, D, F)
        t_mem = nbytes / (hbm_gbs * 1e9)
        t_roof = max(t_fp32, t_sfu, t_mem)
        term = {t_fp32: "fp32", t_sfu: "sfu", t_mem: "hbm"}[t_roof]
        eval_s = statistics.mean(eval_ms) / 1e3
        achieved = units / eval_s
        peak = units / t_roof
        clocks = clk.summary()
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * T / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": _workload_desc(prob), "pop": P, "max_len": prob.pop.max_len,
                       "n_points": D, "n_features": F, "nodes": prob.pop.nodes(),
                       "node_points_per_step": units,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "parallelism": f"population replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": {"bound": "alu", "term": term, "achieved": achieved / 1e9,
                         "peak": peak / 1e9, "unit": "Gnode·pt/s", "frac": achieved / peak,
                         "traffic": _profile_traffic(a.workload),
                         "kernel": "eval_kernel<8,32,plain,mse>",
                         "kernel_ms": 1e3 * eval_s,
                         "peak_basis": f"{sms} SMs x (FP32 128 / SFU 16 (ex2 32) lanes per clock) at "
                                       f"{sm_max_mhz:.0f} MHz, HBM {hbm_gbs} GB/s ({peak_kind})",
                         "t_fp32_ms": 1e3 * t_fp32, "t_sfu_ms": 1e3 * t_sfu, "t_hbm_ms": 1e3 * t_mem,
                         "frac_at_sampled_clock": (achieved / peak) * (sm_max_mhz / clocks["sm_mhz"])
                         if clocks.get("sm_mhz") else None},
            "gpu_launches": 4 * a.steps,
            "clocks": clocks,
        }
        if not a.no_e2e:
            result["e2e"] = e2e(prob, dev, a, units)
        if not a.no_parts and world == 1:
            # the metric's other parts: fwd+bwd time, the batched schedule
            # against one launch per problem, and the multi-output workload
            peaks = (hbm_gbs, sm_max_mhz, peak_kind, sms)
            del flush
            for name, fn in (("fwd_bwd", part_fwd_bwd), ("batched", part_batched), ("modi", part_modi)):
                result[name] = fn(dev, a, local_rank, peaks)
                torch.cuda.empty_cache()
        if not a.no_cpu_baseline and world == 1:
            result["cpu_baseline"] = cpu_baseline(prob)
    return result


# ----------------------------------------------------------------- the metric's other parts
def _timed_clocked(fn, steps, warmup, index, flush=None):
    """Mean ms of fn over `steps` calls, each bracketed by its own CUDA events
    on the current stream (an L2 flush between calls, outside the events),
    with nvidia-smi clocks sampled during the timed calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    with ClockSampler(index) as clk:
        time.sleep(0.2)
        for e0, e1 in ev:
            if flush is not None:
                flush.zero_()
            e0.record()
            fn()
            e1.record()
        torch.cuda.synchronize()
    return statistics.mean(e0.elapsed_time(e1) for e0, e1 in ev), clk.summary()


def _roofline(units, t_fp32, t_sfu, t_mem, ms, kernel, sms, sm_max_mhz, hbm_gbs, peak_kind):
    t_roof = max(t_fp32, t_sfu, t_mem)
    term = "fp32" if t_roof == t_fp32 else "sfu" if t_roof == t_sfu else "hbm"
    achieved = units / (ms / 1e3)
    peak = units / t_roof
    return {"bound": "alu", "term": term, "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "Gnode·pt/s", "frac": achieved / peak, "traffic": None, "kernel": kernel,
            "kernel_ms": ms,
            "peak_basis": f"{sms} SMs x (FP32 128 / SFU 16 (ex2 32) lanes per clock) at "
                          f"{sm_max_mhz:.0f} MHz, HBM {hbm_gbs} GB/s ({peak_kind})",
            "t_fp32_ms": 1e3 * t_fp32, "t_sfu_ms": 1e3 * t_sfu, "t_hbm_ms": 1e3 * t_mem}


def _targets_multi(api, prob, X, dev):
    """y [D, O] = ground-truth trees (evaluated by the library) + noise."""
    import torch
    ys = []
    for k in range(prob.gt.pop):
        gt_t, gt_v, gt_s = api.population_to(prob.gt.take([k]), dev)
        gy, _ = api.tgp_eval_forward(gt_t, gt_v, gt_s, X, 1, max_len=prob.gt.max_len)
        ys.append(gy[0, 0])
    return (torch.stack(ys, 1) + torch.from_numpy(prob.noise).to(dev)).contiguous()


def part_fwd_bwd(dev, a, index, peaks):
    """Differentiation workload: 10,000 trees <= 127 nodes (<= 16 constants),
    200,000 points, F = 4 U(-3,3).  Forward + MSE, fused forward + adjoint
    (gradients of sum(g * MSE) w.r.t. every constant and X), and one Adam step
    on the constants through the autograd.Function."""
    import torch
    from paper_2501_17168_gb300 import api, autograd as ag, workloads as W
    hbm_gbs, sm_max_mhz, peak_kind, sms = peaks
    prob = W.diff(0)
    t, v, s = api.population_to(prob.pop, dev)
    X = torch.from_numpy(prob.X).to(dev)
    y = _targets_multi(api, prob, X, dev)
    P, D, L = prob.pop.pop, prob.D, prob.pop.max_len
    g = torch.full((P, 1), 1.0 / P, dtype=torch.float64, device=dev)
    gx = torch.zeros_like(X)
    units = float(prob.pop.nodes()) * D
    steps = max(a.steps, 3)
    ms_f, clk_f = _timed_clocked(lambda: api.tgp_fitness_mse(t, v, s, X, y, 1, max_len=L), steps, 2,
                                 index)
    ms_fb, clk = _timed_clocked(lambda: api.tgp_eval_backward(t, v, s, X, y, g, 1, max_len=L, grad_X=gx),
                                steps, 2, index)
    api.tgp_check_device_error(dev)
    # Adam on the constants gathered into [P, 16]
    const = (t == W.CONST)
    cnt = const.sum(1)
    order = torch.argsort((~const).to(torch.int8), dim=1, stable=True)[:, :16]
    mask = torch.arange(16, device=dev)[None, :] < cnt[:, None]
    idx = torch.where(mask, order, torch.zeros_like(order))
    consts = torch.gather(v, 1, idx).clone().requires_grad_(True)
    opt = torch.optim.Adam([consts], lr=1e-2)

    def adam_step():
        val = v.scatter(1, idx, torch.where(mask, consts, torch.gather(v, 1, idx)))
        mse = ag.fitness(val, X, t, s, y, 1, max_len=L)
        loss = torch.nan_to_num(mse, nan=0.0, posinf=0.0).clamp(max=1e6).sum()
        opt.zero_grad()
        loss.backward()
        consts.grad = torch.nan_to_num(consts.grad) * mask
        opt.step()
    ms_adam, _ = _timed_clocked(adam_step, min(steps, 20), 1, index)
    t_fp32, t_sfu = _roofline_time_fwd_bwd(prob.pop, D, sms, sm_max_mhz * 1e6)
    t_mem = (_bytes_once(prob.pop, D, prob.F) + 8.0 * D * prob.F + 12.0 * P * L) / (hbm_gbs * 1e9)
    tf32_f, tsfu_f = _roofline_time(prob.pop, D, sms, sm_max_mhz * 1e6, hbm_gbs)
    return {
        "workload": f"diff: {P} trees len<=127 (<=16 constants) x {D} points, F={prob.F} U(-3,3); "
                    "MSE gradient w.r.t. constants and X",
        "node_points": units, "steps": steps,
        "ms_forward_mse": ms_f, "ms_fwd_bwd": ms_fb, "ms_per_adam_step": ms_adam,
        "fwd_bwd_over_forward": ms_fb / ms_f,
        "node_points_per_s_fwd_bwd": units / (ms_fb / 1e3),
        "forward_roofline_frac": 1e3 * max(tf32_f, tsfu_f) / ms_f,
        "roofline": _roofline(units, t_fp32, t_sfu, t_mem, ms_fb, "adjoint (whole call)", sms,
                              sm_max_mhz, hbm_gbs, peak_kind),
        "clocks": clk, "clocks_forward": clk_f,
    }


def part_modi(dev, a, index, peaks):
    """Multi-output workload: 20,000 Modi trees <= 255 nodes, 8 outputs,
    1,000,000 points, F = 32 N(0,1).  Forward + per-output MSE on all points;
    forward + adjoint on every 10th point (stated)."""
    import torch
    from paper_2501_17168_gb300 import api, workloads as W
    hbm_gbs, sm_max_mhz, peak_kind, sms = peaks
    prob = W.modi(0)
    t, v, s = api.population_to(prob.pop, dev)
    X = torch.from_numpy(prob.X).to(dev)
    y = _targets_multi(api, prob, X, dev)
    P, D, L, O = prob.pop.pop, prob.D, prob.pop.max_len, prob.gt.pop
    units = float(prob.pop.nodes()) * D
    steps = max(min(a.steps, 4), 2)
    ms_f, clk = _timed_clocked(lambda: api.tgp_fitness_mse(t, v, s, X, y, O, max_len=L), steps, 1, index)
    Xs, ys = X[::10].contiguous(), y[::10].contiguous()
    g = torch.full((P, O), 1.0 / P, dtype=torch.float64, device=dev)
    gx = torch.zeros_like(Xs)
    ms_fb, clk_b = _timed_clocked(lambda: api.tgp_eval_backward(t, v, s, Xs, ys, g, O, max_len=L, grad_X=gx),
                                  2, 1, index)
    api.tgp_check_device_error(dev)
    t_fp32, t_sfu = _roofline_time(prob.pop, D, sms, sm_max_mhz * 1e6, hbm_gbs, O)
    t_mem = _bytes_once(prob.pop, D, prob.F, O) / (hbm_gbs * 1e9)
    units_s = float(prob.pop.nodes()) * Xs.shape[0]
    b_fp32, b_sfu = _roofline_time_fwd_bwd(prob.pop, Xs.shape[0], sms, sm_max_mhz * 1e6, O)
    return {
        "workload": f"modi: {P} Modi trees len<=255 x {D} points, F={prob.F} N(0,1), {O} outputs; "
                    "forward + MSE (all points); forward + adjoint on every 10th point",
        "node_points": units, "steps": steps,
        "ms_forward_mse": ms_f, "node_points_per_s_forward": units / (ms_f / 1e3),
        "roofline": _roofline(units, t_fp32, t_sfu, t_mem, ms_f, "eval_kernel<4,28,modi,mse> (whole call)",
                              sms, sm_max_mhz, hbm_gbs, peak_kind),
        "fwd_bwd_points": int(Xs.shape[0]), "ms_fwd_bwd_sample": ms_fb,
        "ms_fwd_bwd_extrapolated_all_points": ms_fb * D / Xs.shape[0],
        "fwd_bwd_roofline_frac": 1e3 * max(b_fp32, b_sfu) / ms_fb,
        "node_points_per_s_fwd_bwd": units_s / (ms_fb / 1e3),
        "clocks": clk, "clocks_fwd_bwd": clk_b,
    }


def part_batched(dev, a, index, peaks):
    """Uneven batch: 8 independent SR problems (P 1k-20k, D 1k-1M log-uniform,
    F 4-32, lengths U[7,511]) planned once with the autotuner's cache
    (tgp_batch_plan) and run as one CUDA graph replay, against one
    tgp_fitness_mse launch sequence per problem (library heuristic)."""
    import tempfile
    import torch
    from paper_2501_17168_gb300 import api, autotune, workloads as W
    hbm_gbs, sm_max_mhz, peak_kind, sms = peaks
    probs = W.batched_uneven(0)
    bps, units, t_fp32, t_sfu, t_mem = [], 0.0, 0.0, 0.0, 0.0
    for pr in probs:
        tt, vv, ss = api.population_to(pr.pop, dev)
        Xp, yp = _gpu_targets(api, pr, dev)
        bps.append(api.BatchProblem(tt, vv, ss, Xp, yp, 1, max_len=pr.pop.max_len))
        units += pr.pop.nodes() * pr.D
        f32, sfu = _roofline_time(pr.pop, pr.D, sms, sm_max_mhz * 1e6, hbm_gbs)
        t_fp32 += f32
        t_sfu += sfu
        t_mem += _bytes_once(pr.pop, pr.D, pr.F) / (hbm_gbs * 1e9)
    # autotune every problem into a cache file the C planner reads (points per
    # lane fixed at 8 so that one launch variant serves all of them)
    fd, cache = tempfile.mkstemp(prefix="tgp_tune_", suffix=".txt")
    os.close(fd)
    t0 = time.perf_counter()
    for bp in bps:
        tt, vv, ss, Xp, yp = bp.tensors
        cands = [c for c in autotune.candidates(bp.pop.pop, bp.data.n_points, 1)
                 if c and c.get("points_per_lane") == 8 and c.get("trees_per_block") >= 4]
        autotune.tune(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len, reps=2, cands=cands, path=cache)
    tune_s = time.perf_counter() - t0
    plan = api.BatchPlan(bps, tune_cache=cache)
    shapes = [plan.shape(i) for i in range(len(bps))]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.run()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.run()
    steps = max(min(a.steps, 5), 2)
    ms_graph, clk = _timed_clocked(graph.replay, steps, 1, index)
    plan.check_device_error()

    def per_problem():
        for bp in bps:
            tt, vv, ss, Xp, yp = bp.tensors
            api.tgp_fitness_mse(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len, mse=bp.mse,
                                tree_status=bp.status)
    ms_each, clk_e = _timed_clocked(per_problem, steps, 1, index)
    os.unlink(cache)
    return {
        "workload": "batched_uneven: 8 problems, " + ", ".join(
            f"P={p.pop.pop} D={p.D} F={p.F}" for p in probs) + "; lengths U[7,511]; forward + MSE",
        "node_points": units, "steps": steps,
        "ms_graph_replay_autotuned_plan": ms_graph, "ms_one_launch_per_problem": ms_each,
        "speedup_vs_one_launch_per_problem": ms_each / ms_graph,
        "node_points_per_s": units / (ms_graph / 1e3),
        "autotune_s": tune_s,
        "shapes": [dict(sh, from_cache=fc) for sh, fc in shapes],
        "roofline": _roofline(units, t_fp32, t_sfu, t_mem, ms_graph, "batched graph replay (whole)",
                              sms, sm_max_mhz, hbm_gbs, peak_kind),
        "clocks": clk, "clocks_per_problem": clk_e,
    }


def e2e(prob, dev, a, units):
    """Same metric through the C ABI from pinned host buffers: H2D copies of
    the population, X and y, the fitness call, D2H of MSE and status."""
    import torch
    from paper_2501_17168_gb300 import api
    pin = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()
    ht, hv, hs, hX = pin(prob.pop.type), pin(prob.pop.val), pin(prob.pop.size), pin(prob.X)
    dt_, dv_, ds_ = (torch.empty_like(x, device=dev) for x in (ht, hv, hs))
    dX = torch.empty_like(hX, device=dev)
    gt_t, gt_v, gt_s = api.population_to(prob.gt, dev)
    X0 = hX.to(dev)
    gy, _ = api.tgp_eval_forward(gt_t, gt_v, gt_s, X0, 1, max_len=prob.gt.max_len)
    hy = (gy[0, 0].cpu() + torch.from_numpy(prob.noise[:, 0])).contiguous().view(-1, 1).pin_memory()
    dy = torch.empty_like(hy, device=dev)
    P = prob.pop.pop
    hm = torch.empty((P, 1), dtype=torch.float64).pin_memory()
    hst = torch.empty(P, dtype=torch.int32).pin_memory()
    dm = torch.empty((P, 1), dtype=torch.float64, device=dev)
    dst = torch.empty(P, dtype=torch.int32, device=dev)

    def step():
        for d, h in ((dt_, ht), (dv_, hv), (ds_, hs), (dX, hX), (dy, hy)):
            d.copy_(h, non_blocking=True)
        api.tgp_fitness_mse(dt_, dv_, ds_, dX, dy, 1, max_len=prob.pop.max_len, mse=dm, tree_status=dst)
        hm.copy_(dm, non_blocking=True)
        hst.copy_(dst, non_blocking=True)

    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    T = e0.elapsed_time(e1) / 1e3
    h2d = sum(x.numel() * x.element_size() for x in (ht, hv, hs, hX, hy))
    d2h = hm.numel() * 8 + hst.numel() * 4
    return {"value": units * a.steps / T, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * T / a.steps}


# ----------------------------------------------------------------- other workloads
def _timed(fn, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _gpu_targets(api, prob, dev):
    import torch
    X = torch.from_numpy(prob.X).to(dev)
    gt_t, gt_v, gt_s = api.population_to(prob.gt, dev)
    gy, _ = api.tgp_eval_forward(gt_t, gt_v, gt_s, X, 1, max_len=prob.gt.max_len)
    noise = torch.from_numpy(prob.noise).to(dev)
    return X, (gy[:, 0, :].t() + noise).contiguous()


def suite_lines(dev, steps):
    """sr_small latency, batched uneven (one launch vs one launch per problem,
    graph replay), differentiation and Modi forward + adjoint."""
    import torch
    from paper_2501_17168_gb300 import api, autograd as ag, workloads as W
    hbm_gbs, sm_max_mhz, _ = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_hz = sm_max_mhz * 1e6
    out = []

    # sr_small: 64 trees x 256 points -- latency bound
    prob = W.sr_small(0)
    t, v, s = api.population_to(prob.pop, dev)
    X, y = _gpu_targets(api, prob, dev)
    ms = _timed(lambda: api.tgp_fitness_mse(t, v, s, X, y, 1, max_len=prob.pop.max_len), 200, 20)
    out.append({"workload": "sr_small: 64 trees len<=63 x 256 points, forward + MSE",
                "us_per_call": 1e3 * ms, "node_points_per_s": prob.pop.nodes() * prob.D / (ms / 1e3)})

    # batched uneven: 8 problems in one persistent launch vs one launch per problem
    probs = W.batched_uneven(0)
    bps, units, t_sfu = [], 0.0, 0.0
    for pr in probs:
        tt, vv, ss = api.population_to(pr.pop, dev)
        Xp, yp = _gpu_targets(api, pr, dev)
        bps.append(api.BatchProblem(tt, vv, ss, Xp, yp, 1, max_len=pr.pop.max_len))
        units += pr.pop.nodes() * pr.D
        t_sfu += _roofline_time(pr.pop, pr.D, sms, f_hz, hbm_gbs)[1]
    ms_batch = _timed(lambda: api.tgp_batch_fitness_mse(bps), steps, 2)

    def per_problem():
        for bp in bps:
            tt, vv, ss, Xp, yp = bp.tensors
            api.tgp_fitness_mse(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len, mse=bp.mse,
                                tree_status=bp.status)
    ms_each = _timed(per_problem, steps, 2)
    # autotuned schedule: every problem gets its measured-best launch shape
    # (points per lane fixed at 8 so that one launch serves all of them)
    from paper_2501_17168_gb300 import autotune
    tuned = []
    for bp in bps:
        tt, vv, ss, Xp, yp = bp.tensors
        cands = [c for c in autotune.candidates(bp.pop.pop, bp.data.n_points, 1)
                 if c.get("points_per_lane", 8) == 8 and c.get("trees_per_block", 16) >= 4]
        best, _ = autotune.tune(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len, reps=2, cands=cands,
                                store=False)
        tuned.append(api.BatchProblem(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len, config=best))
    ms_tuned = _timed(lambda: api.tgp_batch_fitness_mse(tuned), steps, 2)
    n = api.tgp_batch_workspace_size(tuned)
    ws = torch.empty(n, dtype=torch.uint8, device=dev)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        api.tgp_batch_fitness_mse(tuned, ws=ws)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        api.tgp_batch_fitness_mse(tuned, ws=ws)
    ms_graph = _timed(graph.replay, steps, 2)
    out.append({"workload": "batched_uneven: 8 problems, P 2,990-19,622, D 3,122-381,279, F 5-30, "
                            "len U[7,511]; forward + MSE",
                "node_points": units, "ms_batched_heuristic": ms_batch,
                "ms_batched_autotuned": ms_tuned, "ms_graph_replay_autotuned": ms_graph,
                "ms_one_launch_per_problem": ms_each,
                "node_points_per_s_graph": units / (ms_graph / 1e3),
                "node_points_per_s_per_problem": units / (ms_each / 1e3),
                "speedup_graph_vs_per_problem": ms_each / ms_graph,
                "roofline_frac_graph": (t_sfu * 1e3) / ms_graph,
                "configs": [{k: v for k, v in tp.cfg.__class__.__dict__.items() if False} or
                            {f: getattr(tp.cfg, f) for f in ("trees_per_block", "points_per_tile",
                                                            "tiles_per_item", "points_per_lane")}
                            for tp in tuned]})

    # many small problems (each too small to fill the GPU on its own)
    probs = W.batched_uneven(7, n_problems=16, pop_range=(500, 2000), d_range=(500, 5000))
    bps, units = [], 0.0
    for pr in probs:
        tt, vv, ss = api.population_to(pr.pop, dev)
        Xp, yp = _gpu_targets(api, pr, dev)
        bps.append(api.BatchProblem(tt, vv, ss, Xp, yp, 1, max_len=pr.pop.max_len))
        units += pr.pop.nodes() * pr.D
    n = api.tgp_batch_workspace_size(bps)
    ws = torch.empty(n, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(side):
        api.tgp_batch_fitness_mse(bps, ws=ws)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        api.tgp_batch_fitness_mse(bps, ws=ws)
    ms_graph = _timed(graph.replay, 20, 3)

    def per_problem_small():
        for bp in bps:
            tt, vv, ss, Xp, yp = bp.tensors
            api.tgp_fitness_mse(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len, mse=bp.mse,
                                tree_status=bp.status)
    ms_each = _timed(per_problem_small, 20, 3)
    out.append({"workload": "batched_small: 16 problems, P U{500..2000}, D log-U[500, 5000], F 4-32, "
                            "len U[7,511]; forward + MSE",
                "node_points": units, "ms_graph_replay": ms_graph, "ms_one_launch_per_problem": ms_each,
                "speedup_graph_vs_per_problem": ms_each / ms_graph,
                "node_points_per_s_graph": units / (ms_graph / 1e3)})

    # differentiation: forward MSE, fused forward + adjoint, one Adam step
    for name, prob, O in (("diff: 10,000 trees len<=127 (<=16 constants) x 200,000 points, F=4",
                           W.diff(0), 1),
                          ("modi: 20,000 Modi trees len<=255 x 1,000,000 points, F=32, 8 outputs",
                           W.modi(0), 8)):
        t, v, s = api.population_to(prob.pop, dev)
        X = torch.from_numpy(prob.X).to(dev)
        ys = []
        for k in range(prob.gt.pop):
            gt_t, gt_v, gt_s = api.population_to(prob.gt.take([k]), dev)
            gy, _ = api.tgp_eval_forward(gt_t, gt_v, gt_s, X, 1, max_len=prob.gt.max_len)
            ys.append(gy[0, 0])
        y = (torch.stack(ys, 1) + torch.from_numpy(prob.noise).to(dev)).contiguous()
        g = torch.full((prob.pop.pop, O), 1.0 / prob.pop.pop, dtype=torch.float64, device=dev)
        units = prob.pop.nodes() * prob.D
        ms_f = _timed(lambda: api.tgp_fitness_mse(t, v, s, X, y, O, max_len=prob.pop.max_len), 1, 1)
        ms_fb = _timed(lambda: api.tgp_eval_backward(t, v, s, X, y, g, O, max_len=prob.pop.max_len), 1, 1)
        t_fp32, t_sfu = _roofline_time(prob.pop, prob.D, sms, f_hz, hbm_gbs, O)
        line = {"workload": name + "; forward + adjoint", "node_points": units,
                "ms_forward_mse": ms_f, "ms_forward_plus_adjoint": ms_fb,
                "node_points_per_s_forward": units / (ms_f / 1e3),
                "node_points_per_s_fwd_bwd": units / (ms_fb / 1e3),
                "forward_roofline_frac": (max(t_fp32, t_sfu) * 1e3) / ms_f}
        if O == 1:
            const = (t == W.CONST)
            idx = torch.zeros((prob.pop.pop, 16), dtype=torch.long, device=dev)
            cnt = const.sum(1)
            order = torch.argsort((~const).to(torch.int8), dim=1, stable=True)[:, :16]
            mask = torch.arange(16, device=dev)[None, :] < cnt[:, None]
            idx = torch.where(mask, order, torch.zeros_like(order))
            consts = torch.gather(v, 1, idx).clone().requires_grad_(True)
            opt = torch.optim.Adam([consts], lr=1e-2)

            def adam_step():
                val = v.scatter(1, idx, torch.where(mask, consts, torch.gather(v, 1, idx)))
                mse = ag.fitness(val, X, t, s, y, 1, max_len=prob.pop.max_len)
                loss = torch.nan_to_num(mse, nan=0.0, posinf=0.0).clamp(max=1e6).sum()
                opt.zero_grad()
                loss.backward()
                consts.grad = torch.nan_to_num(consts.grad) * mask
                opt.step()
            line["ms_per_adam_step"] = _timed(adam_step, 20, 1)
        out.append(line)
    out.extend(genetic_lines(dev, steps))
    return out


def _timed_events(fn, steps, warmup, before=None):
    """Mean device time of fn over `steps` launches, each bracketed by its own
    CUDA events on the current stream (``before`` runs outside the events)."""
    import torch
    for _ in range(warmup):
        if before:
            before()
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for e0, e1 in evs:
        if before:
            before()
        e0.record()
        fn()
        e1.record()
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in evs) / steps


def genetic_lines(dev, steps):
    """The genetic operators: crossover (subtree exchange) of 100,000
    children of trees up to 512 nodes against the HBM roofline, tournament
    selection, and one whole generation (fitness -> selection -> crossover ->
    mutation) replayed from a CUDA graph."""
    import torch
    from paper_2501_17168_gb300 import _lib, api, evolve, workloads as W
    hbm_gbs, _, peak_kind = _peaks()
    out = []
    g = W.genetic(0)
    P = g.pop
    pop = api.population_to(P, dev)
    w = lambda a: torch.from_numpy(np.asarray(a, np.uint32).view(np.int32)).to(dev)
    oi, di = torch.from_numpy(g.old_index).to(dev), torch.from_numpy(g.donor_index).to(dev)
    k, j = w(g.node), w(g.donor_node)
    res = api.tgp_subtree_exchange(pop, oi, k, donor=pop, donor_index=di, donor_node=j,
                                   mode=_lib.PICK_RANDOM, max_size=512, out_ld=512)
    outs, st = res

    def xchg():
        api.tgp_subtree_exchange(pop, oi, k, donor=pop, donor_index=di, donor_node=j,
                                 mode=_lib.PICK_RANDOM, max_size=512, out_ld=512, out=outs, status=st)
    ms = _timed_events(xchg, steps, 3)
    child_nodes = float(outs[2][:, 0].double().sum())
    # algorithmic bytes: each child node read once from its source (3 floats),
    # the four index/word arrays, the full NaN-padded output rows and the status
    nbytes = 12 * child_nodes + 16 * g.n + g.n * (12 * 512 + 4)
    done = float((st == _lib.XCHG_DONE).sum())
    # the oracle beside it: its one-child-at-a-time exchange on a sample
    from oracle import genetic as ogen
    m = 2000
    t0 = time.perf_counter()
    ogen.subtree_exchange((P.type, P.val, P.size), (P.type, P.val, P.size), g.old_index[:m],
                          g.node[:m], g.donor_index[:m], g.donor_node[:m], ogen.RANDOM, 512, 512)
    dt = time.perf_counter() - t0
    out.append({"workload": "crossover: 100,000 children of 100,000 trees len U[1,511] "
                            "(max size 512, {+,-,*,/,sin,cos,tan}), random nodes",
                "ms_per_launch": ms, "children_per_s": g.n / (ms / 1e3),
                "exchanged_fraction": done / g.n,
                "cpu_baseline": {"value": m / dt, "unit": "children/s", "cores": 1, "kind": "oracle",
                                 "sample": f"the first {m} children, {dt:.2f} s wall"},
                "roofline": {"bound": "hbm", "achieved": nbytes / (ms / 1e3) / 1e9,
                             "peak": hbm_gbs, "unit": "GB/s",
                             "frac": nbytes / (ms / 1e3) / 1e9 / hbm_gbs, "peak_kind": peak_kind,
                             "algorithmic_bytes": nbytes}})
    fit = torch.rand(P.pop, dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(0))
    words = w(W.random_words(0, (2 * P.pop, 20), 11))
    win = torch.empty(2 * P.pop, dtype=torch.int32, device=dev)
    ms = _timed_events(lambda: api.tgp_tournament_select(fit, words, True, winners=win), steps, 3)
    m = 20_000
    fit_h = fit.cpu().numpy()
    words_h = W.random_words(0, (2 * P.pop, 20), 11)[:m]
    t0 = time.perf_counter()
    ogen.tournament(fit_h, words_h)
    dt = time.perf_counter() - t0
    out.append({"workload": "tournament selection: 200,000 tournaments of size 20 over 100,000 trees",
                "ms_per_launch": ms, "selections_per_s": 2 * P.pop / (ms / 1e3),
                "cpu_baseline": {"value": m / dt, "unit": "selections/s", "cores": 1,
                                 "kind": "oracle",
                                 "sample": f"the first {m} tournaments, {dt:.2f} s wall"}})
    # one generation of 5,000 trees on the sr_scale data (100,000 points, 16 features)
    prob = W.sr_scale(0)
    Xd, yd = _gpu_targets(api, prob, dev)
    g5 = W.genetic(1, pop=5000, len_range=(1, 255), n_features=16)
    start = api.population_to(g5.pop, dev)
    state = evolve.Generation(tuple(a.clone() for a in start), Xd, yd, api.population_to(g5.pool, dev))
    state.step()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        state.step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        state.step()

    def reset():  # every timed generation starts from the same population
        for dst, src in zip(state.pop, start):
            dst.copy_(src)
    ms_gen = _timed_events(lambda: graph.replay(), steps, 2, before=reset)
    reset()
    ms_fit = _timed_events(lambda: api.tgp_fitness_mse(*state.pop, Xd, yd, 1, max_len=512), steps, 2)
    # classification: 5,000 Modi trees (one output per class) on yeast-shaped data
    cp = W.classification(0, "yeast", pop=5000)
    ct, cv, cs = api.population_to(cp.pop, dev)
    cX = torch.from_numpy(cp.X).to(dev)
    clab = torch.from_numpy(cp.labels).to(dev)
    ms_acc = _timed_events(lambda: api.tgp_fitness_accuracy(ct, cv, cs, cX, clab, cp.n_classes,
                                                            max_len=cp.pop.max_len), steps, 2)
    out.append({"workload": "classification: 5,000 Modi trees len<=255 on yeast-shaped data "
                            "(1,484 points, 8 features, 10 classes): accuracy of every tree",
                "ms_per_call": ms_acc,
                "node_points_per_s": cp.pop.nodes() * cp.X.shape[0] / (ms_acc / 1e3)})
    out.append({"workload": "generation: 5,000 trees (max size 512) on sr_scale data (100,000 points, "
                            "F=16): fitness + tournament(20) + crossover(0.9) + subtree mutation(0.1), "
                            "one CUDA graph replay",
                "ms_per_generation": ms_gen, "ms_fitness_alone": ms_fit,
                "ms_selection_and_operators": ms_gen - ms_fit})
    return out


def sweep_lines(dev, steps):
    """Fitness throughput over the grid of the paper's GPops/s summary table:
    population sizes 100..1,000,000 x the four SR data set shapes, trees of
    300-511 nodes.  Node-point evaluations per second of tgp_fitness_mse
    (inputs resident, CUDA events per call)."""
    import torch
    from paper_2501_17168_gb300 import api, workloads as W
    big = W.sweep_population(0, max(W.SWEEP_POPS))
    lens = big.lengths()
    t, v, s = api.population_to(big, dev)
    out = []
    for name, (D, F) in W.SR_DATASET_SHAPES.items():
        Xn, yn = W.sweep_data(0, name)
        X, y = torch.from_numpy(Xn).to(dev), torch.from_numpy(yn).to(dev)
        for P in W.SWEEP_POPS:
            fn = lambda: api.tgp_fitness_mse(t[:P], v[:P], s[:P], X, y, 1, max_len=512)
            reps = steps if P * D <= 10 ** 9 else 2
            ms = _timed_events(fn, reps, 1)
            units = float(lens[:P].sum()) * D
            out.append({"workload": f"sweep {name}: {P} trees len U[300,511] x {D} points, F={F}",
                        "pop": P, "n_points": D, "ms_per_call": ms,
                        "node_points_per_s": units / (ms / 1e3)})
        del X, y
    return out


E1_POPULATION_PARALLEL = {"points_per_lane": 8, "trees_per_block": 32, "points_per_tile": 256}
E1_DATA_PARALLEL = {"points_per_lane": 8, "trees_per_block": 1, "points_per_tile": 4096}


def e1_lines(dev, steps):
    """Threshold study of Sec. V-B on GB300: the Pagie polynomial, populations
    100 / 1,000 / 5,000 / 10,000, data sets of 64 .. 262,144 points.  Per
    (P, D): the fitness call in the library's population-parallel shape (32
    trees per block over one 256-point chunk: the analogue of the paper's
    hybrid schedule), its data-parallel shape (one tree per block over
    4,096-point tiles: the analogue of the paper's one-tree-per-launch
    schedule), the library's heuristic and the autotuner's pick, each timed
    with CUDA events; then, per population, the data-set sizes at which the
    data-parallel shape is at least as fast as the population-parallel one."""
    import torch
    from paper_2501_17168_gb300 import api, autotune, workloads as W
    big = W.e1_population(0, max(W.E1_POPS))
    lens = big.lengths()
    t, v, s = api.population_to(big, dev)
    out, cross = [], {}
    for D in W.E1_POINTS:
        Xn, yn = W.e1_data(0, D)
        X, y = torch.from_numpy(Xn).to(dev), torch.from_numpy(yn).to(dev)
        for P in W.E1_POPS:
            tt, vv, ss = t[:P], v[:P], s[:P]
            units = float(lens[:P].sum()) * D
            reps = steps if P * D <= 2 ** 27 else 2
            ms = {}
            for name, cfg in (("population_parallel", E1_POPULATION_PARALLEL),
                              ("data_parallel", E1_DATA_PARALLEL), ("heuristic", None)):
                ms[name] = _timed_events(
                    lambda cfg=cfg: api.tgp_fitness_mse(tt, vv, ss, X, y, 1, max_len=256, config=cfg),
                    reps, 1)
            cands = [c for c in autotune.candidates(P, D, 1) if c.get("points_per_lane", 8) == 8]
            best, table = autotune.tune(tt, vv, ss, X, y, 1, max_len=256, reps=1, cands=cands,
                                        store_result=False)
            ms["autotuned"] = _timed_events(
                lambda: api.tgp_fitness_mse(tt, vv, ss, X, y, 1, max_len=256, config=best or None),
                reps, 1)
            api.tgp_check_device_error(dev)
            line = {"case": "e1", "pop": P, "n_points": D, "node_points": units,
                    "ms": ms, "autotuned_shape": best,
                    "node_points_per_s": {k: units / (m / 1e3) for k, m in ms.items()}}
            out.append(line)
            if ms["data_parallel"] <= ms["population_parallel"]:
                cross.setdefault(P, []).append(D)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out.append({"case": "e1_crossover", "D_where_data_parallel_not_slower": cross,
                "sm_count": sms, "sm_count_x_128": sms * 128,
                "paper_threshold_rtx3090": 10_496})
    return out


def run_case(a):
    """One small case for the kernel profiles: the fused forward + adjoint of
    the differentiation workload (constants and inputs), or the Modi forward
    (8 outputs), on --pop trees x --points points; prints one JSON line."""
    import torch
    from paper_2501_17168_gb300 import api, build, workloads as W
    build.build_all()
    dev = torch.device("cuda", 0)
    if a.case == "e1":
        for line in e1_lines(dev, a.steps):
            print(json.dumps(line), flush=True)
        return 0
    if a.case == "sweep":
        for line in sweep_lines(dev, a.steps):
            print(json.dumps(line), flush=True)
        return 0
    if a.case == "genetic":
        for line in genetic_lines(dev, a.steps):
            print(json.dumps(line), flush=True)
        return 0
    if a.case == "batched":
        bps = []
        for pr in W.batched_uneven(0):
            tt, vv, ss = api.population_to(pr.pop, dev)
            Xp, yp = _gpu_targets(api, pr, dev)
            bps.append(api.BatchProblem(tt, vv, ss, Xp, yp, 1, max_len=pr.pop.max_len))

        def per_problem():
            for bp in bps:
                tt, vv, ss, Xp, yp = bp.tensors
                api.tgp_fitness_mse(tt, vv, ss, Xp, yp, 1, max_len=bp.pop.max_len, mse=bp.mse,
                                    tree_status=bp.status)
        ms_b = _timed(lambda: api.tgp_batch_fitness_mse(bps), a.steps, a.warmup)
        ms_p = _timed(per_problem, a.steps, a.warmup)
        api.tgp_check_device_error(dev)
        print(json.dumps({"case": "batched", "ms_batched": ms_b, "ms_one_launch_per_problem": ms_p}),
              flush=True)
        return 0
    if a.case == "adjoint":
        prob, O = W.diff(0, pop=a.pop, D=a.points), 1
    else:
        prob, O = W.modi(0, pop=a.pop, D=a.points), 8
    t, v, s = api.population_to(prob.pop, dev)
    X = torch.from_numpy(prob.X).to(dev)
    y = torch.from_numpy(np.random.default_rng(0).standard_normal((prob.D, O)).astype(np.float32)).to(dev)
    g = torch.full((prob.pop.pop, O), 1.0 / prob.pop.pop, dtype=torch.float64, device=dev)
    if a.case == "adjoint":
        fn = lambda: api.tgp_eval_backward(t, v, s, X, y, g, O, max_len=prob.pop.max_len)
    else:
        fn = lambda: api.tgp_fitness_mse(t, v, s, X, y, O, max_len=prob.pop.max_len)
    ms = _timed(fn, a.steps, a.warmup)
    api.tgp_check_device_error(dev)
    print(json.dumps({"case": a.case, "pop": prob.pop.pop, "n_points": prob.D, "n_outputs": O,
                      "ms_per_call": ms, "node_points_per_s": prob.pop.nodes() * prob.D / (ms / 1e3)}),
          flush=True)
    return 0


def main():
    a = _args()
    if a.case:
        return run_case(a)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return run_reference(a, rank, world)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    res = run_ours(a, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
        if a.suite:
            import torch
            for line in suite_lines(torch.device("cuda", local_rank), max(a.steps // 2, 2)):
                print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
