"""Benchmark of the CoMET hot path on GB300: converged mode-TO solves/s.

Workload (the 4-segment pushing enumeration): square slider 0.09 m,
c = 0.04 m, mu = 0.3, 12 modes per segment, every order of 4 segments
(20,736 per instance), 20 intervals per segment (N = 80), 64 seeded
start/goal instances, cold start.  One step = the full enumeration of one
instance: every order solved by the persistent evaluator, scored
(Eq. inexact_mode_value, Eq. search_merit) and the enumeration argmin taken
(Eq. mode_selection).  Steps cycle through the instances.

Prints one JSON line (the benchmark line format): value = converged solves
(status CONVERGED and FP64-certified v_hat < 1e-5) per second over the timed
steps, device-timed with CUDA events on the problem's stream, inputs resident
in HBM; e2e = the same metric through the C ABI with host buffers (copies
inside the timed region); roofline of the evaluator kernel against the FP32
ALU peak; cpu_baseline = the FP64 oracle on the host cores over a bounded
sample of the same workload.

``--impl reference`` times the oracle alone (host cores) on the same workload
and prints the reference line.
"""
from __future__ import annotations

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

METRIC = "converged mode-TO solves/s (viol<1e-5) on 1 GB300; plan time vs plain evaluator"
UNIT = "solves/s"
N_INSTANCES = 64
SEG, K = 4, 20
N_STAGES = SEG * K
# the method's floating-point operations per stage and solver iteration on
# this workload, counted by the oracle's counting build over a seeded sample
# (python -m oracle.flop_count; tests/test_flop_count.py re-measures it):
# rows and Jacobians once per iteration, the local model on its nonzero
# pattern, the 7x7 factorisation and solves, the value function, the
# forward pass, the sequential trial merits up to the accepted step, retries
FLOP_PER_STAGE_ITER = 1989.2
# the same for timing optimisation (state x, y, theta, s, tau; control f_n,
# f_t, sdot, h), counted by the numpy oracle over 48 two-segment orders
# under each of the timing leg's bounds
TIMING_FLOP_PER_STAGE_ITER = {"slack": 3362.3, "binding": 3555.3}
# DRAM bytes (read + write) of one evaluator launch over the 20,736 orders,
# from the ncu capture of the current kernel on the 4,096-order case (9.37 MB
# read, 51.1 MB written: stage records and spills leaving L2;
# profiles/eval_kernel_push_l4.md), scaled by the TOs processed
EVAL_TRAFFIC_BYTES = (9.374208e6 + 51.054592e6) * 20736 / 4096
# nominal FP32 FMA rate at the maximum clock (152 SMs x 128 lanes x 2 flop x
# 2070 MHz), context only: the roofline's peak is measured at run time by the
# library's FMA microbenchmark (comet_fp32_fma_peak)
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def measure_fp32_peak(P, stream):
    """Best of five runs of the FMA microbenchmark (about 10 ms each) on the
    bench's stream, with the SM clock sampled around it."""
    import torch

    scratch = torch.empty(P.comet_fp32_fma_peak_threads(), dtype=torch.float32, device="cuda")
    clk = ClockSampler(torch.cuda.current_device())
    clk.start()
    runs = [P.comet_fp32_fma_peak(stream.cuda_stream, 6000, scratch) for _ in range(5)]
    c = clk.stop()
    best = max(runs)
    return {"tflops": best[0], "ms": best[1], "runs_tflops": [r[0] for r in runs], "sm_mhz": c.get("sm_mhz"),
            "how": "comet_fp32_fma_peak: 8 independent fmaf chains per thread, whole waves of 256-thread "
                   "blocks, CUDA events, best of 5"}


def rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def shard(n_items: int, rank: int, world: int) -> list:
    """Replicas: rank r takes items r, r + world, ... (no exchange on the data
    path; every item is taken by exactly one rank)."""
    return list(range(rank, n_items, world))


def reduce_over_ranks(t_dev: float, counts, device):
    """Max over ranks of the timed region and the sum of the work counts
    (one all_reduce each; no-op with one process)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_dev, [int(c) for c in counts]
    t = torch.tensor([t_dev], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(x) for x in counts], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t[0]), [int(round(float(x))) for x in c]


def instances():
    return [W.push_l4_instance(s) for s in range(N_INSTANCES)]


def oracle_rate(insts, seconds_target: float = 12.0, max_n: int = 20736):
    """The FP64 oracle as it stands, one TO per host thread on every core,
    over a bounded sample of the workload (orders of instance 0 in
    enumeration order).  Returns (converged solves/s, solves/s, sample)."""
    import oracle

    seqs = W.all_sequences(12, SEG)
    cores = os.cpu_count() or 1
    n = 64 * cores
    t0 = time.time()
    res, _ = oracle.solve_batch([insts[0]], np.zeros(n, np.int32), seqs[:n], np.full(n, SEG, np.int32),
                                nthreads=cores)
    dt = time.time() - t0
    # grow the sample to about `seconds_target` seconds of CPU work
    n2 = int(min(max_n, max(n, n * seconds_target / max(dt, 1e-3))))
    if n2 > n:
        t0 = time.time()
        res, _ = oracle.solve_batch([insts[0]], np.zeros(n2, np.int32), seqs[:n2], np.full(n2, SEG, np.int32),
                                    nthreads=cores)
        dt = time.time() - t0
        n = n2
    conv = int(np.sum((res["status"] == 0) & (res["viol"] < 1e-5)))
    return conv / dt, n / dt, n, cores, dt


WORKLOAD = ("push_l4 full enumeration: 20,736 orders (4 segments x 12 modes) x N=80 intervals per step, one seeded "
            "instance per step, cold start")


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return
    import oracle

    insts = instances()
    # untimed warm-up steps: a short oracle batch each (pages the library and
    # the thread pool in)
    cores = os.cpu_count() or 1
    seqs = W.all_sequences(12, SEG)
    for _ in range(args.warmup):
        oracle.solve_batch([insts[0]], np.zeros(cores, np.int32), seqs[:cores], np.full(cores, SEG, np.int32),
                           nthreads=cores)
    t_all = 0.0
    conv_all = 0
    for s in range(args.steps):
        r, _, n, cores, dt = oracle_rate(insts, seconds_target=max(2.0, 60.0 / max(1, args.steps)))
        t_all += dt
        conv_all += r * dt
    value = conv_all / t_all
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "instances": N_INSTANCES, "orders_per_step": 20736,
                                         "parallelism": f"replicas x{world}"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {n} orders of instance 0 per step, FP64 C oracle, one TO per thread"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2609_21803_gb300 as P

    rank, world, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    P.build.build()
    P.lib()
    insts = instances()
    seqs = W.all_sequences(12, SEG)
    if args.orders:
        seqs = seqs[: args.orders]  # profiling runs only: a prefix of the enumeration
    n = len(seqs)
    stream = torch.cuda.Stream()
    # one problem per instance; orders resident on the device (replicas: rank
    # r takes instances r, r + world, ...)
    my = shard(N_INSTANCES, rank, world)
    probs = []
    with torch.cuda.stream(stream):
        for i in my:
            probs.append(P.Problem([insts[i]], stream=stream))
    packed = P.pack_mode_seqs(seqs)
    d_seqs = torch.from_numpy(packed.view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
    cost = torch.empty(n, dtype=torch.float32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    viol = torch.empty(n, dtype=torch.float32, device="cuda")
    iters = torch.empty(n, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    torch.cuda.synchronize()

    def step(j):
        pr = probs[j % len(probs)]
        P.comet_eval_modes(pr.handle, d_seqs, n, None, cost, None, status)
        P.comet_eval_stats(pr.handle, viol, None, iters, None)
        conv = (status == 0) & (viol < 1e-5)
        # enumeration argmin (Eq. mode_selection): least merit among feasible
        key = torch.where(viol <= 1e-5, cost, torch.full_like(cost, float("inf")))
        best = torch.argmin(key)
        return conv.sum(), best, iters.sum()

    with torch.cuda.stream(stream):
        for w in range(args.warmup):
            step(w)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_dev = 0.0
    conv_total = 0
    iter_total = 0
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    outs = []
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            outs.append(step(args.warmup + s))
            ev[s][1].record(stream)
    torch.cuda.synchronize()
    for s in range(args.steps):
        t_dev += ev[s][0].elapsed_time(ev[s][1]) / 1e3
        conv_total += int(outs[s][0])
        iter_total += int(outs[s][2])
    # max over ranks of the timed region, sum of the work
    t_dev, (conv_total, iter_total) = reduce_over_ranks(t_dev, [conv_total, iter_total], "cuda")
    clk = clocks.stop()
    value = conv_total / t_dev

    # e2e: the C ABI with host buffers (orders in, cost/status out), copies
    # inside, over as many steps as the timed region
    host_seqs = packed
    h_cost = np.zeros(n, np.float32)
    h_status = np.zeros(n, np.int32)
    h_viol = np.zeros(n, np.float32)
    t0 = time.time()
    e2e_conv = 0
    e2e_steps = max(1, args.steps)
    for s in range(e2e_steps):
        pr = probs[(args.warmup + s) % len(probs)]
        P.comet_eval_modes(pr.handle, host_seqs, n, None, h_cost, None, h_status)
        P.comet_eval_stats(pr.handle, h_viol, None, None, None)
        e2e_conv += int(np.sum((h_status == 0) & (h_viol < 1e-5)))
    e2e_t = time.time() - t0
    e2e_value = e2e_conv * world / e2e_t

    flops = FLOP_PER_STAGE_ITER * N_STAGES * iter_total
    achieved = flops / t_dev / 1e12
    peak = measure_fp32_peak(P, stream)
    hbm_peak, hbm_kind = measured_peak("hbm_gbs", 6800.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances": N_INSTANCES, "orders_per_step": n, "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas x{world}"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(n * P.MODE_SEQ_BYTES),
                "d2h_bytes_per_step": int(n * (4 + 4 + 4) + 4)},  # cost, status, v_hat; the device flag
        # per step: the longest-first ordering (hist, scan, scatter kernels;
        # the problem holds orders of up to 4 segments) and the evaluator
        "gpu_launches": 4 * args.steps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak["tflops"], "unit": "TFLOP/s",
                     "frac": achieved / peak["tflops"], "traffic": EVAL_TRAFFIC_BYTES,
                     "hbm": {"achieved_gbs": EVAL_TRAFFIC_BYTES * args.steps / t_dev / 1e9, "peak_gbs": hbm_peak,
                             "frac": EVAL_TRAFFIC_BYTES * args.steps / t_dev / 1e9 / hbm_peak,
                             "peak_kind": f"of {hbm_kind} (STREAM-style copy; 6.8 TB/s when no measured figure is present)",
                             "note": "the captured DRAM traffic per launch x launches / device time"},
                     "peak_measured": peak, "nominal_tflops": FP32_NOMINAL_TFLOPS,
                     "note": f"achieved = {FLOP_PER_STAGE_ITER} flop (the oracle's count of the method per "
                             "stage and iteration) x 80 stages x solver iterations / device time; peak = "
                             "measured FP32 FMA rate (of measured)",
                     "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the current kernel on a "
                                     "4,096-order launch (same workload), scaled by the TOs processed to 20,736"},
        "iterations_per_solve": iter_total / (args.steps * n * world),
    }
    if rank == 0 and args.plan_instances > 0:
        line["plan"] = plan_times(P, insts[: args.plan_instances])
    if rank == 0 and args.hetero:
        line["hetero"] = hetero_times(P)
    if rank == 0 and args.batch_plan:
        line["batch_plan"] = batch_plan_times(P)
    if rank == 0 and args.grammar:
        line["grammar"] = grammar_times(P)
    if rank == 0 and args.bimanual:
        line["bimanual"] = bimanual_times(P, per=args.bim_per, fp32_peak=peak["tflops"],
                                          oracle_s=0.0 if args.no_cpu_baseline else 10.0)
    if rank == 0 and args.cfg5:
        line["cfg5"] = cfg5_times(P)
    if rank == 0 and args.timing:
        line["timing"] = timing_times(P, fp32_peak=peak["tflops"],
                                      oracle_n=None if args.no_cpu_baseline else 2 * (os.cpu_count() or 1),
                                      l4_orders=args.orders)
    if rank == 0 and args.learned_instances > 0:
        line["learned"] = learned_times(P, insts, args.learned_instances, oracle_on=not args.no_cpu_baseline)
    if rank == 0 and args.mcts:
        try:
            line["mcts"] = mcts_times(P)
        except Exception as e:  # a failing comparison leg must not cost the line its other figures
            line["mcts"] = {"error": f"{type(e).__name__}: {e}"[:300]}
    if rank == 0 and not args.no_cpu_baseline:
        conv_rate, rate, ns, cores, dt = oracle_rate(insts)
        line["cpu_baseline"] = {"value": conv_rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"first {ns} orders of instance 0 ({dt:.1f} s), FP64 C oracle, "
                                          f"one TO per host thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for pr in probs:
        pr.close()
    if world > 1:
        dist.destroy_process_group()


def plan_times(P, insts):
    """Plan time of CoMET's expansion (Algorithm 1: seed batch of all orders
    of <= 2 segments, beam 64, B = 4096, s_max = 3, K_ref = 256 refined with
    t_ref = 1500) against full enumeration of the same order space (every
    order of <= 4 segments, 22,620, then the same refinement), both through
    the device planner; device time per instance."""
    seeds = [(m,) for m in range(12)] + [tuple(s) for s in W.all_sequences(12, 2)]
    every = seeds + [tuple(s) for s in W.all_sequences(12, 3)] + [tuple(s) for s in W.all_sequences(12, 4)]
    out = {"instances": len(insts), "expansion_ms": [], "enumeration_ms": [], "expansion_evals": [],
           "enumeration_evals": [], "recovered": 0}
    for inst in insts:
        prob = P.Problem([inst])
        ps = P.pack_mode_seqs(seeds)
        pe = P.pack_mode_seqs(every)
        ex = P.comet_plan(prob.handle, 0, ps, len(ps), dict(k=64, batch=4096, rounds=3, k_ref=256))
        en = P.comet_plan(prob.handle, 0, pe, len(pe), dict(k=64, batch=4096, rounds=0, k_ref=256))
        out["expansion_ms"].append(ex["explore_ms"] + ex["refine_ms"])
        out["enumeration_ms"].append(en["explore_ms"] + en["refine_ms"])
        out["expansion_evals"].append(ex["evaluations"])
        out["enumeration_evals"].append(en["evaluations"])
        if ex["best_cost"] <= en["best_cost"] * (1 + 1e-3) + 1e-9:
            out["recovered"] += 1
        prob.close()
    for key in ("expansion_ms", "enumeration_ms", "expansion_evals", "enumeration_evals"):
        out[key] = float(np.median(out[key]))
    out["speedup"] = out["enumeration_ms"] / out["expansion_ms"]
    out["note"] = "median over instances; recovered = expansion's refined best within 1e-3 of enumeration's"
    return out


def hetero_times(P, n_inst=256, per=512, n_split=32):
    """The mixed workload (rectangular sliders of side 0.05-0.15 m and aspect
    1-3, mu ~ U[0.2, 0.6], length caps 1..6, 10..30 knots per segment, seeds
    0..255), 512 random orders per instance (length uniform in 1..cap):
    every order of every instance in ONE persistent launch (longest TO
    first, launch shape from the autotuner), against one launch per instance
    for the first `n_split` instances.  Device time, converged solves/s."""
    import torch

    insts = [W.push_mixed_instance(s) for s in range(n_inst)]
    rng = np.random.default_rng(7)
    seqs, idx = [], []
    for i, inst in enumerate(insts):
        for _ in range(per):
            L = int(rng.integers(1, inst["max_segments"] + 1))
            seqs.append(tuple(int(m) for m in rng.integers(0, 12, L)))
            idx.append(i)
    packed = P.pack_mode_seqs(seqs, np.array(idx, np.int32))
    d = torch.from_numpy(packed.view(np.uint8).reshape(len(seqs), P.MODE_SEQ_BYTES)).cuda()
    stream = torch.cuda.current_stream()

    def timed(prob, dd):
        prob.eval(dd)  # warm (workspace, attributes)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = prob.eval(dd)
        e1.record(stream)
        torch.cuda.synchronize()
        conv = int(((r["status"] == 0) & (r["viol"] < 1e-5)).sum())
        return e0.elapsed_time(e1) / 1e3, conv

    prob = P.Problem(insts)
    pick, times = P.comet_autotune(prob.handle, d[:8192], 8192, 40)
    t_one, c_one = timed(prob, d)
    # the same first n_split instances: one launch vs one per instance
    m = n_split * per
    t_sub, c_sub = timed(prob, d[:m])
    prob.close()
    t_per, c_per = 0.0, 0
    for i in range(n_split):
        pr = P.Problem([insts[i]])
        sub = P.pack_mode_seqs(seqs[i * per:(i + 1) * per])
        t, c = timed(pr, torch.from_numpy(sub.view(np.uint8).reshape(per, P.MODE_SEQ_BYTES)).cuda())
        t_per += t
        c_per += c
        pr.close()
    return {
        "instances": n_inst, "orders": len(seqs), "n_max": int(max(x["knots_per_segment"] * x["max_segments"]
                                                                    for x in insts)),
        "autotuned": pick, "autotune_candidate_ms": times,
        "one_launch_solves_per_s": c_one / t_one, "one_launch_ms": t_one * 1e3,
        "split_instances": n_split, "split_one_launch_solves_per_s": c_sub / t_sub,
        "split_per_instance_solves_per_s": c_per / t_per, "split_per_instance_ms": t_per * 1e3,
        "split_one_launch_ms": t_sub * 1e3,
        "note": "converged solves/s (device time); one launch over all instances vs one launch per instance",
    }


def batch_plan_times(P, n_inst=256, n_seq=16):
    """Algorithm 1 on the mixed workload as configured: 256 instances
    (rectangular sliders, 1-6 segments, 10-30 knots per segment), each seeded
    with all its orders of at most two segments (156), beam k = 64, batch
    B = 1,024 per instance, three rounds, an evaluation budget of 2e5 per
    instance, the K_ref = 64 best refined with t_ref = 1,500.  All instances
    through the batched planner (one persistent evaluator launch per round
    for all of them, the round captured as a CUDA graph, the launch shape
    autotuned) against the single-instance planner called once per instance
    on the first `n_seq` instances.  Device time of exploration +
    refinement."""
    insts = [W.push_mixed_instance(s) for s in range(n_inst)]

    def seeds(inst):
        two = [(a, b) for a in range(12) for b in range(12)] if inst["max_segments"] >= 2 else []
        return [(m,) for m in range(12)] + two

    sd = [seeds(i) for i in insts]
    opts = dict(k=64, batch=1024, rounds=3, k_ref=64, ref_iters=1500, budget=200000)
    prob = P.Problem(insts)
    sample = P.pack_mode_seqs([s for i in range(n_seq) for s in sd[i]],
                              np.concatenate([np.full(len(sd[i]), i, np.int32) for i in range(n_seq)]))
    P.comet_autotune(prob.handle, sample, len(sample), 60)
    P.comet_plan_batch(prob.handle, list(range(n_seq)), sd[:n_seq], opts)  # warm
    rb = P.comet_plan_batch(prob.handle, list(range(n_inst)), sd, opts)
    t_all = (rb[0]["explore_ms"] + rb[0]["refine_ms"]) / 1e3
    t_explore = rb[0]["explore_ms"] / 1e3
    rs = P.comet_plan_batch(prob.handle, list(range(n_seq)), sd[:n_seq], opts)
    t_sub = (rs[0]["explore_ms"] + rs[0]["refine_ms"]) / 1e3
    t_one, same = 0.0, 0
    for i in range(n_seq):
        r = P.comet_plan(prob.handle, i, P.pack_mode_seqs(sd[i], np.full(len(sd[i]), i, np.int32)), len(sd[i]),
                         opts)
        t_one += (r["explore_ms"] + r["refine_ms"]) / 1e3
        same += int(r["best"] == rs[i]["best"] and r["best_cost"] == rs[i]["best_cost"])
    prob.close()
    feas = sum(int(r["best_status"] == 0) for r in rb)
    evals = [r["evaluations"] for r in rb]
    return {
        "instances": n_inst, "config": "beam 64, B 1024, 3 rounds, budget 2e5/instance, seeds 156, K_ref 64 at 1500",
        "batched_ms": t_all * 1e3, "plan_ms_per_instance": t_all * 1e3 / n_inst, "batched_plans_per_s": n_inst / t_all,
        "explore_solves_per_s": float(np.sum(evals)) / t_explore, "feasible_plans": feas,
        "evaluations_median": float(np.median(evals)), "evaluations_max": int(np.max(evals)),
        "subset": n_seq, "subset_batched_ms": t_sub * 1e3, "subset_one_by_one_ms": t_one * 1e3,
        "subset_speedup": t_one / t_sub, "subset_same_plans": same,
        "note": "device time (exploration + refinement); one-by-one = the single-instance planner per instance; "
                "explore_solves_per_s = evaluations of all instances / exploration time",
    }


def mcts_times(P, n_inst=4, pools=(1024, 256, 64)):
    """The MCTS comparison policy (Sec. IV-A) on the grammar leg's box
    instances: UCT (c = 0.8) with virtual loss and random rollouts, pools of
    P orders per evaluator launch, capped at the evaluation count of the
    expansion (beam 64, B = 1,024, r = 2, three rounds) on the same instance,
    then the same refinement (K_ref = 256 at t_ref = 1,500).  MCTS times are
    wall time of the search (host tree + GPU pools) plus device time of the
    refinement; expansion times are device time."""
    seeds = W.admissible_push_orders(6)
    every = W.admissible_push_orders(8)
    ps, pe = P.pack_mode_seqs(seeds), P.pack_mode_seqs(every)
    base = dict(k=64, batch=1024, k_ref=256, ref_iters=1500)
    res = {q: {"ms": [], "evals": [], "pools": [], "recovered": 0, "feasible": 0} for q in pools}
    ex_ms, ex_rec = [], 0
    for s in range(n_inst):
        prob = P.Problem([W.push_grammar_instance(s)])
        ex = P.comet_plan(prob.handle, 0, ps, len(seeds), dict(base, rounds=3, radius=2, grammar=1))
        en = P.comet_plan(prob.handle, 0, pe, len(every), dict(base, rounds=0))
        tol = en["best_cost"] * (1 + 1e-3) + 1e-9
        ex_ms.append(ex["explore_ms"] + ex["refine_ms"])
        ex_rec += int(ex["best_status"] == 0 and ex["best_cost"] <= tol)
        for q in pools:
            mc = P.comet_plan_mcts(prob.handle, 0, dict(grammar=P.GRAMMAR_PUSH, seed=3000 + s,
                                                        max_evals=ex["evaluations"]), q, base)
            r = res[q]
            r["ms"].append(mc["explore_ms"] + mc["refine_ms"])
            r["evals"].append(mc["evaluations"])
            r["pools"].append(mc["rounds_run"])
            r["recovered"] += int(mc["best_status"] == 0 and mc["best_cost"] <= tol)
            r["feasible"] += int(mc["best_status"] == 0)
        prob.close()
    out = {"instances": n_inst, "expansion_ms": float(np.median(ex_ms)), "expansion_recovered": ex_rec}
    for q in pools:
        r = res[q]
        out[f"pool_{q}"] = {"ms": float(np.median(r["ms"])), "evaluations": float(np.median(r["evals"])),
                            "pools": float(np.median(r["pools"])), "recovered": r["recovered"],
                            "feasible": r["feasible"]}
    out["note"] = ("medians over instances; recovered = refined best within 1e-3 of full enumeration's; "
                   "MCTS capped at the expansion's evaluation count on each instance")
    return out


def first_distinct(recs, n_modes, k):
    """The first k distinct orders of a stream of packed records, in stream
    order.  The first occurrences in a stream of independent uniform draws
    come in uniformly random order, so the first k distinct draws are a
    uniform sample of k orders without replacement."""
    base = np.uint64(n_modes + 1)
    code = recs["len"].astype(np.uint64)
    p = base.copy()
    for i in range(recs["modes"].shape[1]):
        live = recs["len"] > i
        code = code + np.where(live, (recs["modes"][:, i].astype(np.uint64) + np.uint64(1)) * p, np.uint64(0))
        p = p * base if i + 1 < recs["modes"].shape[1] else p
    _, first = np.unique(code, return_index=True)
    return recs[np.sort(first)[:k]]


def grammar_times(P, n_inst=4):
    """The paper's pushing grammar on the four-faced box (Sec. IV-A): modes
    are stick on a face or free motion, orders of at most 8 segments
    (6,297 admissible).  Seed only (the 601 admissible orders of at most 6
    segments), expansion from that seed (beam 64, B = 1,024, r = 2, three
    rounds), uniform sampling without replacement of as many admissible
    orders as the expansion evaluated, and full enumeration of all 6,297,
    each followed by the same
    refinement (K_ref = 256 at t_ref = 1,500).  Device time per instance."""
    seeds = W.admissible_push_orders(6)
    every = W.admissible_push_orders(8)
    ps, pe = P.pack_mode_seqs(seeds), P.pack_mode_seqs(every)
    out = {"instances": n_inst, "seed_orders": len(seeds), "admissible_orders": len(every),
           "expansion_ms": [], "seed_only_ms": [], "uniform_ms": [], "enumeration_ms": [], "expansion_evals": [],
           "recovered": 0, "seed_only_recovered": 0, "uniform_recovered": 0, "feasible": 0}
    for s in range(n_inst):
        prob = P.Problem([W.push_grammar_instance(s)])
        base = dict(k=64, batch=1024, k_ref=256, ref_iters=1500)
        ex = P.comet_plan(prob.handle, 0, ps, len(seeds), dict(base, rounds=3, radius=2, grammar=1))
        so = P.comet_plan(prob.handle, 0, ps, len(seeds), dict(base, rounds=0))
        en = P.comet_plan(prob.handle, 0, pe, len(every), dict(base, rounds=0))
        # uniform sampling without replacement (Sec. IV-B): the first distinct
        # orders of the sampler's stream, as many as the expansion evaluated
        pu = first_distinct(P.comet_sample_orders(prob.handle, 0, 1000 + s, 0, 4 * ex["evaluations"],
                                                  P.GRAMMAR_PUSH), 13, ex["evaluations"])
        un = P.comet_plan(prob.handle, 0, pu, len(pu), dict(base, rounds=0))
        out["expansion_ms"].append(ex["explore_ms"] + ex["refine_ms"])
        out["seed_only_ms"].append(so["explore_ms"] + so["refine_ms"])
        out["uniform_ms"].append(un["explore_ms"] + un["refine_ms"])
        out["enumeration_ms"].append(en["explore_ms"] + en["refine_ms"])
        out["expansion_evals"].append(ex["evaluations"])
        tol = en["best_cost"] * (1 + 1e-3) + 1e-9
        out["recovered"] += int(ex["best_status"] == 0 and ex["best_cost"] <= tol)
        out["seed_only_recovered"] += int(so["best_status"] == 0 and so["best_cost"] <= tol)
        out["uniform_recovered"] += int(un["best_status"] == 0 and un["best_cost"] <= tol)
        out["feasible"] += int(en["best_status"] == 0)
        prob.close()
    for key in ("expansion_ms", "seed_only_ms", "uniform_ms", "enumeration_ms", "expansion_evals"):
        out[key] = float(np.median(out[key]))
    out["note"] = ("medians over instances; recovered = refined best within 1e-3 of the enumeration's; "
                   "free-motion orders converge a little less often in FP32 than in FP64: 89 % against "
                   "93 % within 300 iterations on 2-4-segment box orders")
    return out


# the bimanual method's floating-point operations per stage and iteration,
# counted by the oracle's counting build on random 1..6-segment orders of
# the bimanual workload (python -m oracle.flop_count; tests/test_flop_count.py)
BIM_FLOP_PER_STAGE_ITER = 8185.0


def bim_oracle_rate(insts, seqs, idx, seconds_target=10.0):
    """The bimanual FP64 C oracle as it stands on the leg's orders (in the
    leg's order), one TO per host thread on every core, over a sample grown
    to about `seconds_target` seconds.  Returns (converged solves/s, sample
    size, cores, seconds)."""
    import oracle

    cores = os.cpu_count() or 1
    n = min(len(seqs), 4 * cores)
    while True:
        t0 = time.time()
        res, _ = oracle.bim_solve_batch(insts, idx[:n], seqs[:n], [len(q) for q in seqs[:n]], nthreads=cores)
        dt = time.time() - t0
        n2 = int(min(len(seqs), n * seconds_target / max(dt, 1e-3)))
        if n2 <= 1.5 * n or n >= len(seqs):
            break
        n = n2
    conv = int(np.sum((res["status"] == 0) & (res["viol"] < 1e-5)))
    return conv / dt, n, cores, dt


def bimanual_times(P, n_inst=8, per=512, n_plan=2, fp32_peak=None, oracle_s=10.0):
    """The bimanual variant (box flipped by two point hands on a ground
    contact, 507 modes per segment, 15 knots per segment, one CTA per TO):
    random orders of 1..6 segments (512 per instance, 8 instances) in one
    persistent launch, and Algorithm 1 on `n_plan` instances (seed = the 507
    one-segment orders, beam 16, B = 1,024, s_max = 3, K_ref = 64)."""
    import torch

    insts = [W.bimanual_instance(s) for s in range(n_inst)]
    rng = np.random.default_rng(11)
    seqs, idx = [], []
    for i in range(n_inst):
        for _ in range(per):
            L = int(rng.integers(1, 7))
            seqs.append(tuple(int(m) for m in rng.integers(0, 507, L)))
            idx.append(i)
    packed = P.pack_mode_seqs(seqs, np.array(idx, np.int32))
    d = torch.from_numpy(packed.view(np.uint8).reshape(len(seqs), P.MODE_SEQ_BYTES)).cuda()
    prob = P.Problem(insts)
    prob.eval(d[:256])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = prob.eval(d)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    conv = int(((r["status"] == 0) & (r["viol"] < 1e-5)).sum())
    iters = float(r["iters"].float().mean())
    # stage-iterations of the launch: iterations x intervals (15 per segment)
    lens = torch.tensor([len(q) for q in seqs], dtype=torch.float64, device="cuda")
    stage_iters = float((r["iters"].double() * 15.0 * lens).sum())
    cfg = P.comet_get_launch_config(prob.handle)
    prob.close()
    plans = []
    seeds = P.pack_mode_seqs([(m,) for m in range(507)])
    for i in range(n_plan):
        pr = P.Problem([insts[i]])
        res = P.comet_plan(pr.handle, 0, seeds, 507, dict(k=16, batch=1024, rounds=3, k_ref=64))
        plans.append({"plan_ms": res["explore_ms"] + res["refine_ms"], "evaluations": res["evaluations"],
                      "best_len": len(res["best"]), "best_cost": res["best_cost"],
                      "feasible": bool(res["best_status"] == 0 and res["best_viol"] <= 1e-5)})
        pr.close()
    achieved = BIM_FLOP_PER_STAGE_ITER * stage_iters / t / 1e12
    roof = {"kernel": "bimanual_kernel (one CTA per TO)", "bound": "alu", "achieved": achieved, "unit": "TFLOP/s",
            "peak": fp32_peak, "frac": achieved / fp32_peak if fp32_peak else None,
            "note": f"achieved = {BIM_FLOP_PER_STAGE_ITER} flop (the oracle's count per stage and iteration) x "
                    "stage-iterations of the launch / device time; peak = measured FP32 FMA rate (of measured)"}
    out = {"orders": len(seqs), "converged_solves_per_s": conv / t, "solves_per_s": len(seqs) / t,
           "converged_fraction": conv / len(seqs), "iterations_per_solve": iters, "ms": t * 1e3,
           "ctas_per_sm": cfg["blocks_per_sm"], "plans": plans, "roofline": roof,
           "note": "one CTA (128 threads) per TO; device time; v_hat in physical units"}
    if oracle_s > 0:
        rate, ns, cores, dt = bim_oracle_rate(insts, seqs, np.array(idx, np.int32), oracle_s)
        out["oracle"] = {"converged_solves_per_s": rate, "cores": cores, "kind": "oracle",
                         "sample": f"first {ns} orders of the leg ({dt:.1f} s), FP64 C oracle, one TO per thread"}
    return out


def _timing_oracle_job(job):
    from oracle import timing as TM

    inst, modes, tm, max_iters = job
    _, _, r = TM.solve(inst, modes, timing=tm, max_iters=max_iters)
    return r["status"], r["viol"]


def timing_oracle_rate(insts, orders, idx, tm, max_iters, n):
    """The numpy FP64 timing oracle as it stands on the first `n` orders of
    the leg, one TO per spawned worker (one BLAS thread each) on every core.
    Returns (converged solves/s, seconds, cores)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    cores = os.cpu_count() or 1
    tmo = dict(h_min=tm["h_min"], h_max=tm["h_max"], T=tm["T_max"])
    jobs = [(insts[int(idx[i])], orders[i], tmo, max_iters) for i in range(n)]
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    old = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    try:
        with ProcessPoolExecutor(min(cores, n), mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_timing_oracle_job, jobs[:1]))  # workers up (numpy imported) before the clock
            t0 = time.time()
            res = list(ex.map(_timing_oracle_job, jobs))
            dt = time.time() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    conv = sum(1 for st, v in res if st == 0 and v < 1e-5)
    return conv / dt, dt, cores


def timing_times(P, per_inst=(3, 4, 5, 6, 7, 8, 9, 10), l4_inst=3, max_iters=1500, fp32_peak=None,
                 oracle_n=None, l4_orders=0):
    """Timing optimisation (interval durations among the controls, the
    elapsed time tau carrying the duration bound): the 2-segment
    enumerations (144 orders, N = 16) of the listed instances and the
    4-segment enumeration (20,736 orders, N = 80) of one instance, each under
    a bound with room (h in [dt/2, 2 dt], T twice the fixed schedule's
    length) and a binding one (h in [dt/5, 3 dt], T = 3/4 of it); one launch
    each after a warm-up launch, device time."""
    import torch

    out = {}
    stream = torch.cuda.current_stream()
    work = [("l2", [W.push_l2_instance(s) for s in per_inst], 2), ("l4", [W.push_l4_instance(l4_inst)], 4)]
    for name, insts, L in work:
        orders = [tuple(int(v) for v in q) for q in W.all_sequences(12, L)]
        if L == 4 and l4_orders:
            orders = orders[:l4_orders]  # profiling: a prefix of the enumeration
        seqs = [q for _ in insts for q in orders]
        idx = np.repeat(np.arange(len(insts), dtype=np.int32), len(orders))
        n = len(seqs)
        d = torch.from_numpy(P.pack_mode_seqs(seqs, idx).view(np.uint8).reshape(n, P.MODE_SEQ_BYTES)).cuda()
        dt, nint = insts[0]["dt"], insts[0]["knots_per_segment"] * L
        bounds = {"slack": dict(h_min=0.5 * dt, h_max=2.0 * dt, T_max=2.0 * nint * dt),
                  "binding": dict(h_min=0.2 * dt, h_max=3.0 * dt, T_max=0.75 * nint * dt)}
        prob = P.Problem(insts)
        cost = torch.empty(n, dtype=torch.float32, device="cuda")
        status = torch.empty(n, dtype=torch.int32, device="cuda")
        viol = torch.empty(n, dtype=torch.float32, device="cuda")
        iters = torch.empty(n, dtype=torch.int32, device="cuda")
        for bname, tm in bounds.items():
            nw = min(n, 256)
            P.comet_eval_modes_timed(prob.handle, tm, d[:nw], nw, None, max_iters, cost, None, status)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.comet_eval_modes_timed(prob.handle, tm, d, n, None, max_iters, cost, None, status)
            e1.record(stream)
            P.comet_eval_stats(prob.handle, viol, None, iters, None)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            conv = int(((status == 0) & (viol <= 1e-5)).sum())
            it_sum = float(iters.double().sum())
            achieved = TIMING_FLOP_PER_STAGE_ITER[bname] * it_sum * nint / t / 1e12
            leg = {"orders": n, "intervals": nint, "bounds": tm, "ms": t * 1e3,
                   "converged_solves_per_s": conv / t, "converged_fraction": conv / n,
                   "iterations_per_solve": it_sum / n, "max_iters": max_iters,
                   "roofline": {"bound": "alu", "achieved": achieved, "unit": "TFLOP/s", "peak": fp32_peak,
                                "frac": achieved / fp32_peak if fp32_peak else None}}
            if name == "l2" and oracle_n:
                seqs_i = [tuple(q) for q in seqs]
                rate, dt_o, cores = timing_oracle_rate(insts, seqs_i, idx, tm, max_iters, min(oracle_n, n))
                leg["oracle"] = {"converged_solves_per_s": rate, "cores": cores, "kind": "oracle",
                                 "sample": f"first {min(oracle_n, n)} orders of the leg ({dt_o:.1f} s), numpy FP64 "
                                           "oracle, one TO per spawned worker"}
            out[f"{name}_{bname}"] = leg
        prob.close()
    out["note"] = ("timing_kernel: one warp per TO, state (x, y, theta, s, tau), control (f_n, f_t, sdot, h); "
                   "cold start h_k = dt clipped into the bounds; device time of one launch; roofline achieved = "
                   f"{TIMING_FLOP_PER_STAGE_ITER} flop per stage-iteration (the numpy oracle's count under each "
                   "bound) x iterations x intervals / device time, peak = measured FP32 FMA rate (of measured)")
    return out


def cfg5_times(P, n_inst=128, n_train=64, per_train=768):
    """Bimanual flipping at the configured scale: 128 seeded instances (seeds
    0..127), Algorithm 1 from the 507 one-segment seeds (beam 16, s_max = 3,
    K_ref = 64 at t_ref, budget 1e6 evaluations per instance), FP32 solves
    with FP64 certification, all instances in one batched planner call:
    plain (B = 1,024) and with the learned proposal (the 256 best of each
    round's whole neighbourhood by predicted merit, warm-started).  The proposal is trained first on evaluator results
    of separate instances (seeds 1000.., 768 random orders of 1..4 segments
    each)."""
    import torch

    budget = 1000000
    rng = np.random.default_rng(2)
    tr = [W.bimanual_instance(1000 + s) for s in range(n_train)]
    prob = P.Problem(tr)
    q = P.comet_proposal_create(prob.handle, {"dataset_cap": n_train * per_train})
    seqs = [tuple(int(m) for m in rng.integers(0, 507, rng.integers(1, 5))) for _ in range(n_train * per_train)]
    packed = P.pack_mode_seqs(seqs, np.repeat(np.arange(n_train, dtype=np.int32), per_train))
    torch.cuda.synchronize()
    t0 = time.time()
    for a in range(0, len(packed), 16384):
        d = torch.from_numpy(packed[a:a + 16384].view(np.uint8).reshape(-1, P.MODE_SEQ_BYTES)).cuda()
        r = prob.eval(d, want_traj=True)
        P.comet_proposal_add_samples(q, d, len(d), r["cost"], r["viol"], r["status"], r["traj"])
    torch.cuda.synchronize()
    t_data = time.time() - t0
    t0 = time.time()
    losses = np.concatenate([P.comet_proposal_train(q, 600, 2048, {"lr": 1e-3}, seed=1),
                             P.comet_proposal_train(q, 400, 2048, {"lr": 3e-4}, seed=2)])
    t_train = time.time() - t0
    _, _, _, npar = P.comet_proposal_dims(q)
    flat = np.zeros(npar, np.float32)
    P.comet_proposal_get_params(q, flat)
    P.comet_proposal_destroy(q)
    prob.close()
    insts = [W.bimanual_instance(s) for s in range(n_inst)]
    one = [(m,) for m in range(507)]
    prob = P.Problem(insts)
    plain_opts = dict(k=16, batch=1024, rounds=3, k_ref=64, budget=budget)
    t0 = time.time()
    plain = P.comet_plan_batch(prob.handle, list(range(n_inst)), [one] * n_inst, plain_opts)
    t_plain_wall = time.time() - t0
    t_plain = (plain[0]["explore_ms"] + plain[0]["refine_ms"]) / 1e3
    q = P.comet_proposal_create(prob.handle)
    P.comet_proposal_set_params(q, flat)
    t0 = time.time()
    learned = P.comet_plan_batch(prob.handle, list(range(n_inst)), [one] * n_inst,
                                 dict(k=16, batch=256, rounds=3, k_ref=64, budget=budget), proposal=q)
    t_learned_wall = time.time() - t0
    t_learned = (learned[0]["explore_ms"] + learned[0]["refine_ms"]) / 1e3
    P.comet_proposal_destroy(q)
    prob.close()
    ok = lambda r: bool(r["best_status"] == 0 and r["best_viol"] <= 1e-5)
    feas_p = [ok(r) for r in plain]
    feas_l = [ok(r) for r in learned]
    both = [i for i in range(n_inst) if feas_p[i] and feas_l[i]]
    gaps = np.array([(learned[i]["best_cost"] - plain[i]["best_cost"]) / abs(plain[i]["best_cost"]) for i in both])
    ev_p = [r["evaluations"] for r in plain]
    ev_l = [r["evaluations"] for r in learned]
    return {
        "instances": n_inst, "budget_per_instance": budget,
        "config": "bimanual box flip, 507 modes, 15 knots/segment, L <= 6; beam 16, 3 rounds, K_ref 64 at t_ref 1500",
        "train": {"instances": n_train, "samples": n_train * per_train, "dataset_s": t_data, "train_s": t_train,
                  "steps": 1000, "batch": 2048, "loss_first": float(losses[:10].mean()),
                  "loss_last": float(losses[-50:].mean())},
        "plain": {"feasible_plans": int(sum(feas_p)), "evaluations_total": int(np.sum(ev_p)),
                  "evaluations_median": float(np.median(ev_p)), "batched_ms": t_plain * 1e3,
                  "ms_per_instance": t_plain * 1e3 / n_inst, "wall_s": t_plain_wall,
                  "best_len_median": float(np.median([len(r["best"]) for r in plain])), "batch": 1024},
        "learned": {"feasible_plans": int(sum(feas_l)), "evaluations_total": int(np.sum(ev_l)),
                    "evaluations_median": float(np.median(ev_l)), "batched_ms": t_learned * 1e3,
                    "ms_per_instance": t_learned * 1e3 / n_inst, "wall_s": t_learned_wall,
                    "best_len_median": float(np.median([len(r["best"]) for r in learned])), "batch": 256},
        "plan_time_ratio_plain_over_learned": t_plain / t_learned,
        "evaluations_saved": 1.0 - float(np.sum(ev_l)) / float(np.sum(ev_p)),
        "cost_gap_learned_vs_plain": {"n": len(both), "p10": float(np.percentile(gaps, 10)) if len(both) else None,
                                      "p50": float(np.median(gaps)) if len(both) else None,
                                      "p90": float(np.percentile(gaps, 90)) if len(both) else None,
                                      "learned_better_by_1e-3": int(np.sum(gaps < -1e-3)),
                                      "learned_worse_by_1e-3": int(np.sum(gaps > 1e-3))},
        "note": "feasible = certified plan (FP64 v_hat <= 1e-5); plan times are device time of one batched "
                "planner call over all instances (exploration + refinement)",
    }


def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


# multiply-adds per row of the proposal MLP (64 -> 256 -> 256 -> 256 -> 256)
MLP_MACS = 64 * 256 + 2 * 256 * 256 + 256 * 256


def learned_times(P, insts, n_eval, oracle_on=True):
    """The learned proposal on the same workload family: a training set of
    about 1M evaluator results (512 random 4-segment instances, seeds
    1000..1511, 2,048 random orders each, solved by the GPU evaluator), 3,000
    AdamW steps of 4,096 samples on the tensor cores, then the planner with
    and without the proposal on held-out instances (seeds 48.., plain: B =
    4096; learned: the 512 best neighbours by predicted merit, warm-started;
    both beam 64, s_max = 3, K_ref = 256)."""
    import torch

    every = [(m,) for m in range(12)] + [tuple(s) for s in W.all_sequences(12, 2)] + \
        [tuple(s) for s in W.all_sequences(12, 3)] + [tuple(s) for s in W.all_sequences(12, 4)]
    n_inst, per = 512, 2048
    tr = [W.push_l4_instance(1000 + s) for s in range(n_inst)]
    prob = P.Problem(tr)
    q = P.comet_proposal_create(prob.handle, {"dataset_cap": n_inst * per})
    rng = np.random.default_rng(0)
    pick = rng.integers(0, len(every), size=n_inst * per)
    packed = P.pack_mode_seqs([every[j] for j in pick], np.repeat(np.arange(n_inst, dtype=np.int32), per))
    torch.cuda.synchronize()
    t0 = time.time()
    for a in range(0, len(packed), 65536):
        d = torch.from_numpy(packed[a:a + 65536].view(np.uint8).reshape(-1, P.MODE_SEQ_BYTES)).cuda()
        r = prob.eval(d, want_traj=True)
        P.comet_proposal_add_samples(q, d, len(d), r["cost"], r["viol"], r["status"], r["traj"])
    torch.cuda.synchronize()
    t_data = time.time() - t0
    steps = 3000
    t0 = time.time()
    losses = np.concatenate([P.comet_proposal_train(q, steps // 2, 4096, {"lr": 1e-3}, seed=1),
                             P.comet_proposal_train(q, steps // 4, 4096, {"lr": 3e-4}, seed=2),
                             P.comet_proposal_train(q, steps // 4, 4096, {"lr": 1e-4}, seed=3)])
    t_train = time.time() - t0
    _, _, _, npar = P.comet_proposal_dims(q)
    flat = np.zeros(npar, np.float32)
    P.comet_proposal_get_params(q, flat)
    # forward over one 4-segment enumeration (20,736 rows), device buffers
    rows = 20736
    x = torch.zeros((rows, 64), dtype=torch.int16, device="cuda")
    P.comet_proposal_features(q, torch.from_numpy(packed[:rows].view(np.uint8).reshape(-1, P.MODE_SEQ_BYTES)).cuda(), rows, x)
    # device time of the fused forward kernel, events on its own stream
    fwd_s = P.comet_proposal_time_forward(q, x, rows, 50) / 1e3
    din, width, dout, _ = P.comet_proposal_dims(q)
    oracle_fwd = None
    if oracle_on:
        # the FP64 oracle's forward on the host over the same features
        # (numpy, its BLAS on the host cores), repeated for about a second
        from oracle import mlp as OM

        bits = x.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
        X = bits.view(np.float32).astype(np.float64)
        params = OM.unflatten(flat.astype(np.float64), din, width, dout)
        nr, done, t0 = 4096, 0, time.time()
        while time.time() - t0 < 1.0:
            OM.forward(params, X[:nr])
            done += nr
        dt_o = time.time() - t0
        oracle_fwd = {"rows_per_s": done / dt_o, "cores": os.cpu_count() or 1, "kind": "oracle",
                      "sample": f"{done} rows of the enumeration's features in {dt_o:.1f} s, numpy FP64 forward"}
    P.comet_proposal_destroy(q)
    prob.close()
    peak, kind = measured_peak("bf16_tflops", 1900.0)
    fwd_tflops = 2.0 * MLP_MACS * rows / fwd_s / 1e12
    train_flop = 2.0 * (3 * MLP_MACS - 64 * 256) * 4096
    train_tflops = train_flop * steps / t_train / 1e12
    # the ablation on held-out instances
    seeds = [(m,) for m in range(12)] + [tuple(s) for s in W.all_sequences(12, 2)]
    ps = P.pack_mode_seqs(seeds)
    same, pl_ms, le_ms, pl_ev, le_ev, gaps = 0, [], [], [], [], []
    for i in range(48, 48 + n_eval):
        # held-out instances: seeds 48.. (the training set uses seeds 1000..1511)
        pr = P.Problem([W.push_l4_instance(i)])
        a = P.comet_plan(pr.handle, 0, ps, len(ps), dict(k=64, batch=4096, rounds=3, k_ref=256))
        qq = P.comet_proposal_create(pr.handle)
        P.comet_proposal_set_params(qq, flat)
        b = P.comet_plan(pr.handle, 0, ps, len(ps), dict(k=64, batch=512, rounds=3, k_ref=256), proposal=qq)
        P.comet_proposal_destroy(qq)
        pr.close()
        same += b["best_cost"] <= a["best_cost"] * (1 + 1e-3) + 1e-9
        gaps.append((b["best_cost"] - a["best_cost"]) / abs(a["best_cost"]))
        pl_ms.append(a["explore_ms"] + a["refine_ms"])
        le_ms.append(b["explore_ms"] + b["refine_ms"])
        pl_ev.append(a["evaluations"])
        le_ev.append(b["evaluations"])
    return {
        "dataset_samples": n_inst * per, "dataset_s": t_data, "train_steps": steps, "train_batch": 4096,
        "train_s": t_train, "train_samples_per_s": steps * 4096 / t_train,
        "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-100:].mean()),
        "forward_rows": rows, "forward_ms": fwd_s * 1e3, "forward_rows_per_s": rows / fwd_s,
        "oracle_forward": oracle_fwd,
        "roofline": {"kernel": "mlp_fused_forward_kernel (4 tcgen05 layers chained through TMEM)", "bound": "tensor",
                     "achieved": fwd_tflops, "peak": peak, "unit": "TFLOP/s", "frac": fwd_tflops / peak,
                     "peak_kind": f"{kind} bf16 (burst)", "train_step_tflops": train_tflops},
        "instances": n_eval, "same_best": same,
        "plain_ms": float(np.median(pl_ms)), "learned_ms": float(np.median(le_ms)),
        "plain_evals": float(np.median(pl_ev)), "learned_evals": float(np.median(le_ev)),
        "plan_speedup": float(np.median(pl_ms) / np.median(le_ms)),
        "cost_gap": {"p10": float(np.percentile(gaps, 10)), "p50": float(np.median(gaps)),
                     "p90": float(np.percentile(gaps, 90)), "max": float(np.max(gaps)), "min": float(np.min(gaps)),
                     "learned_better_by_1e-3": int(np.sum(np.array(gaps) < -1e-3)),
                     "learned_worse_by_1e-3": int(np.sum(np.array(gaps) > 1e-3))},
        "note": "plan times are device time (medians); same_best = learned plan within 1e-3 of plain expansion's; "
                "cost_gap = (J_learned - J_plain) / J_plain of the returned plans over the held-out instances",
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--orders", type=int, default=0, help="profiling only: solve this prefix of each enumeration")
    ap.add_argument("--plan-instances", type=int, default=4, help="instances for the plan-time comparison (0 = skip)")
    ap.add_argument("--hetero", type=int, default=1, help="mixed-workload leg (1) or skip it (0)")
    ap.add_argument("--batch-plan", type=int, default=1, help="batched multi-instance planner leg (1) or skip it (0)")
    ap.add_argument("--grammar", type=int, default=1, help="pushing-grammar planning leg (1) or skip it (0)")
    ap.add_argument("--bim-per", type=int, default=512, help="random orders per instance in the bimanual leg")
    ap.add_argument("--bimanual", type=int, default=1, help="bimanual leg (1) or skip it (0)")
    ap.add_argument("--mcts", type=int, default=1, help="MCTS comparison leg (1) or skip it (0)")
    ap.add_argument("--timing", type=int, default=1, help="timing-optimisation leg (1) or skip it (0)")
    ap.add_argument("--cfg5", type=int, default=1,
                    help="bimanual planning at scale with the learned proposal (1) or skip it (0)")
    ap.add_argument("--learned-instances", type=int, default=32,
                    help="held-out instances of the learned-planner ablation (0 = skip training and ablation)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
