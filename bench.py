#!/usr/bin/env python3
"""Batched Pair-HMM forward + adjoint throughput on GB300, in GCUPS (Eq. 5).

One step = the whole hot path over one batch: preparation, length binning, the FP32
wavefront forward (with the FP64 rescue of any underflowed pair), the adjoint wavefront and
the FP64 per-read gradient reduction.  Inputs are seeded synthetic batches shaped like the
paper's workloads (see paper_2411_11547_gb300/synth.py); the default workload is the
persistent-kernel batch: 65,536 regions x 4 haplotypes x 16 reads = 2^22 pairs with read
lengths log-uniform in 36..300 and haplotype lengths log-uniform in 64..2048.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line on rank 0.  `--impl reference` times the FP64 CPU oracle (the only
reference that exists for this method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Pair-HMM GCUPS fwd and fwd+bwd vs plain FP32 kernel; % of FP32-pipe peak"
UNIT = "GCUPS"
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# FP32 pipe operations per cell, algorithmic.  With beta folded into the emission table and
# the deletion state carried as D' = D/zeta: M = E (a' M_diag + S_diag) with S = I + D (2),
# I = delta M_up + eps I_up (2), D' = M_left + eps D'_left (1), S = I + zeta D' (1): 6.
FWD_OPS_PER_CELL = 6
# Adjoint, algorithmic: the forward values of the cell (6, above) plus the reverse
# recurrences (u = beta lambda M^: 1; M^: 3; I^: 1; D^: 1) plus the partials (alpha, beta:
# 2; Q: I+D, alpha' M + S, w M^ G: 3; delta, zeta: 2; eps: 2): 6 + 6 + 9 + 1 = 22.
BWD_OPS_PER_CELL = 22
# The hot-path scope's own per-cell counts (7 FP32-pipe operations per forward cell with the
# lambda-alpha / lambda-beta fold, about 25 per adjoint cell including the recompute).  The
# roofline line uses these; the reduced counts above are reported beside them.
FWD_OPS_SCOPE = 7
BWD_OPS_SCOPE = 25
# subset size of the end-to-end host call (phmm_grad_host): with the ramp at both ends about 5
# subsets on the 3e11-cell step (measured on GB300, per step: 2^35 739, 2^36 734, 2^37 725,
# 2^38 721 ms)
E2E_SUBSET_CELLS = 1 << 38
# DRAM bytes per cell of the adjoint kernel (read + written: its checkpoints), from an ncu
# capture of wf_backward<float,16,10> on the 4.5e9-cell c3_grad batch (8.30 GB read, 10.74 GB
# written); the c4 step's traffic is this times its cells.
BWD_DRAM_BYTES_PER_CELL = (8.298 + 10.743) * 1e9 / 4.5e9

WORKLOAD_DESC = {
    "c4_persistent": "65,536 regions x 4 haplotypes x 16 reads = 2^22 pairs; read length "
                     "log-uniform 36..300, haplotype length log-uniform 64..2048; bq 10..40, "
                     "gap-open quals 45, GCP 10",
    "c1_batched": "2,000 regions, 2..16 haplotypes (100..600) x 20..200 reads (lognormal mean "
                  "150, 50..250), all-vs-all",
    "c3_grad": "100,000 pairs in 16 x 64 regions, m = 150, n = 300, float quals",
}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi SM clock and throttle-reason samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="phmm_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(batch, target_s, seed=12345):
    """Time the FP64 CPU oracle (forward + adjoint) on a seeded random subset of pairs sized
    for about target_s seconds on this host; returns (GCUPS, cells, pairs, seconds, cores)."""
    import numpy as np

    import oracle
    from paper_2411_11547_gb300 import synth
    rng = np.random.default_rng(seed)
    P = len(batch["pair_read"])
    cores = oracle.default_threads()
    # calibration: grow a subset until it takes about a second
    k = 8 * cores
    while True:
        cal = synth.subset_pairs(batch, rng.choice(P, size=min(P, k), replace=False))
        t0 = time.perf_counter()
        oracle.backward_batch(cal, np.ones(len(cal["pair_read"])))
        dt = time.perf_counter() - t0
        if dt > 1.0 or k >= P:
            break
        k *= 4
    rate = synth.cells(cal) / dt
    mean_cells = synth.cells(batch) / P
    k = int(min(P, max(4 * cores, target_s * rate / mean_cells)))
    idx = np.sort(rng.choice(P, size=k, replace=False))
    sb = synth.subset_pairs(batch, idx)
    cells = synth.cells(sb)
    t0 = time.perf_counter()
    oracle.backward_batch(sb, np.ones(k))
    dt = time.perf_counter() - t0
    return cells / dt / 1e9, cells, k, dt, cores


def run_reference(args, batch, ws, rank):
    """The FP64 CPU oracle as the reference arm: each step scores a bounded random sample."""
    if rank != 0:
        return
    budget = 150.0 / max(1, args.steps + args.warmup)
    for w in range(args.warmup):
        oracle_sample(batch, min(budget, 5.0), seed=100 + w)
    vals, cells_tot, t_tot, pairs = [], 0, 0.0, 0
    for k in range(args.steps):
        g, cells, kp, dt, cores = oracle_sample(batch, budget, seed=1000 + k)
        vals.append(g)
        cells_tot += cells
        t_tot += dt
        pairs += kp
    value = cells_tot / t_tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOAD_DESC.get(args.workload, '')}",
                   "pairs_per_step": pairs // args.steps},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{pairs // args.steps} pairs per step, seeded random subset "
                                   f"of {args.workload}, forward + adjoint in FP64"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=("gb300", "reference"))
    ap.add_argument("--workload", default="c4_persistent",
                    choices=("c4_persistent", "c1_batched", "c3_grad"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="use the built-in group tables instead of phmm_autotune's")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: the ranks split ONE batch by read (every read's "
                         "pairs on one rank) and sum d/dgcp with one all-reduce per step; "
                         "default: every rank scores its own batch of the same shape")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_env()
    from paper_2411_11547_gb300 import synth
    seed_base = {"c4_persistent": 4, "c1_batched": 1, "c3_grad": 3}[args.workload]
    if args.shard:
        # strong scaling: one batch, split by read over the ranks (shard.py)
        from paper_2411_11547_gb300 import shard
        full = synth.make(args.workload, seed=seed_base)
        full_cells = synth.cells(full)
        full_pairs = len(full["pair_read"])
        batch, _, _ = shard.shard(full, rank, ws)
        del full
    else:
        # weak scaling: every rank scores its own batch of the same shape (seeds per rank)
        batch = synth.make(args.workload, seed=seed_base + 1000 * rank)
    if args.impl == "reference":
        return run_reference(args, batch, ws, rank)

    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2411_11547_gb300 import phmm
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    cells = synth.cells(batch)
    P = len(batch["pair_read"])
    dbatch = phmm.DeviceBatch(batch, dev)
    # measured read-length -> group tables for this workload shape (outside the timed region,
    # like plan creation)
    t_tune = time.perf_counter()
    opts = phmm.options() if args.no_tune else phmm.autotune(dbatch, which=3, sample_pairs=32768)
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t_tune

    def opts_with(**kw):
        o = phmm.Options.from_buffer_copy(opts)
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    plan = phmm.Plan(dbatch, opts)
    stream = torch.cuda.current_stream()
    dL = torch.ones(P, dtype=torch.float64, device=dev)
    out, flags = plan.forward()
    rescued = float((flags & phmm.FLAG_RESCUED64).ne(0).float().mean().item())

    # one training step: the fused forward (log10 L of every pair and its partials from the
    # adjoint sweep) and the FP64 per-read reduction weighted by dL
    def step():
        plan.forward_partials(out, flags)
        g = plan.backward_partials(dL)
        if args.shard and dist is not None:
            # the one cross-rank sum of the sharded step: d/dgcp (8 bytes, in stream order)
            from paper_2411_11547_gb300 import shard as _sh
            _sh.allreduce_tensor_(g[3])
        return g

    # the same step as two independent calls: the forward graph, then the whole backward
    def step_two_call():
        plan.forward(out, flags)
        return plan.backward(dL)

    for _ in range(args.warmup):
        step()
    barrier()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    adj_ms, red_ms = [], []
    # NVTX range around the timed steps, so a profiler can be limited to them
    torch.cuda.nvtx.range_push("timed_steps")
    e0.record(stream)
    for _ in range(args.steps):
        step()
        a, r = plan.backward_ms()
        if a >= 0:
            adj_ms.append(a)
            red_ms.append(r)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    a, r = plan.backward_ms()
    if a >= 0 and len(adj_ms) < args.steps:
        adj_ms.append(a)
        red_ms.append(r)
    launches = plan.launch_count(0) + plan.launch_count(1)

    # the two-call step, timed the same way
    for _ in range(2):
        step_two_call()
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step_two_call()
    e1.record(stream)
    barrier()
    ms_two = e0.elapsed_time(e1) / args.steps

    # forward alone (graph replay), timed the same way
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        plan.forward(out, flags)
    e1.record(stream)
    barrier()
    ms_fwd = e0.elapsed_time(e1) / args.steps
    sample_clk = clocks.stop()

    # per-kernel times of the forward from an event-instrumented (non-graph) plan
    plan_t = phmm.Plan(dbatch, opts_with(use_graph=0))
    plan_t.forward()
    wf_ms, resc_ms = [], []
    for _ in range(args.steps):
        plan_t.forward(out, flags)
        torch.cuda.synchronize()
        x, y = plan_t.wavefront_ms()
        wf_ms.append(x)
        resc_ms.append(y)
    del plan_t

    # the plain FP32 wavefront kernel (no binning, no rescue, one group) on the 1,024-pair
    # equal-length batch, repeated back to back
    c0 = synth.c0_plain()
    c0_cells = synth.cells(c0)
    c0_plan = phmm.Plan(phmm.DeviceBatch(c0, dev),
                        phmm.options(binning=0, lanes=16, rows=12, first_line=0, rescue=0,
                                     persistent=0, use_graph=0))
    o0, f0 = c0_plan.forward()
    for _ in range(5):
        c0_plan.forward(o0, f0)
    reps = 200
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        c0_plan.forward(o0, f0)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1) / reps
    c0_wf = []
    for _ in range(20):
        c0_plan.forward(o0, f0)
        torch.cuda.synchronize()
        c0_wf.append(c0_plan.wavefront_ms()[0])
    del c0_plan

    # the plain kernel on this step's own batch: one fixed group covering the longest read
    # (16 lanes x 20 rows = 320 rows), plain FP32 tier, no binning, no rescue, persistent
    pl_plain = phmm.Plan(dbatch, phmm.options(binning=0, lanes=16, rows=20, first_line=0,
                                              rescue=0, persistent=1, use_graph=0))
    pl_plain.forward(out, flags)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        pl_plain.forward(out, flags)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_same_ms = e0.elapsed_time(e1) / 3
    del pl_plain

    # pipe probes (lane operations per second) on this GPU
    ffma = phmm.probe_pipe(0, 4000)[0]
    ffma2 = phmm.probe_pipe(1, 4000)[0]
    dfma = phmm.probe_pipe(2, 400)[0]

    # end to end from host memory through phmm_grad_host, the library's call for a batch in
    # host memory: every step packs the batch into pinned staging, copies it and dL = 1 to
    # the device, runs the fused step per subset (plan with validation, forward with
    # partials, weighted reduction) and copies log10 L, flags and the gradients back, the
    # copies of one subset overlapping the computation of the previous one
    e2e = None
    e2e_dev = None
    if not args.no_e2e:
        sum_m = int(batch["read_off"][-1])
        dL_h = np.ones(P)
        outs = (np.empty(P), np.empty(P, dtype=np.uint8), np.empty(sum_m, dtype=np.float32),
                np.empty(sum_m, dtype=np.float32), np.empty(sum_m, dtype=np.float32))
        h2d = sum(np.asarray(batch[k]).nbytes for k in
                  ("read_bases", "base_q", "ins_q", "del_q", "read_off", "hap_bases", "hap_off",
                   "pair_read", "pair_hap")) + dL_h.nbytes
        d2h = sum(x.nbytes for x in outs) + 8
        phmm.grad_host(batch, dL_h, opts, subset_cells=E2E_SUBSET_CELLS, out=outs)  # buffers
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            phmm.grad_host(batch, dL_h, opts, subset_cells=E2E_SUBSET_CELLS, out=outs)
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
               "call": f"phmm_grad_host (host arrays in and out, subsets of "
                       f"{E2E_SUBSET_CELLS:.3g} cells)"}
        phmm.lib().phmm_score_host_release()

    # the same through the device API, unpipelined: every step copies the batch from pinned
    # host tensors, builds a plan, runs the fused step and copies the results back
    if not args.no_e2e:
        hb = {k: (torch.from_numpy(np.ascontiguousarray(v)).pin_memory()
                  if isinstance(v, np.ndarray) else v) for k, v in batch.items()}
        h2d = sum(t.numel() * t.element_size() for t in hb.values() if torch.is_tensor(t))
        out_h = torch.empty(P, dtype=torch.float64).pin_memory()
        sum_m = int(batch["read_off"][-1])
        g_h = torch.empty(3 * sum_m, dtype=torch.float32).pin_memory()
        d2h = out_h.numel() * 8 + g_h.numel() * 4 + 8

        def e2e_step():
            td = {k: hb[k].to(dev, non_blocking=True)
                  for k in ("read_bases", "base_q", "ins_q", "del_q", "read_off", "hap_bases",
                            "hap_off", "pair_read", "pair_hap")}
            db = phmm.DeviceBatch.from_tensors(gcp=float(batch["gcp"]), alpha_mode=0, **td)
            pl = phmm.Plan(db, opts)
            o, _ = pl.forward_partials()
            gb, gi, gd, gg = pl.backward_partials(dL)
            out_h.copy_(o, non_blocking=True)
            g_h[:sum_m].copy_(gb, non_blocking=True)
            g_h[sum_m:2 * sum_m].copy_(gi, non_blocking=True)
            g_h[2 * sum_m:].copy_(gd, non_blocking=True)
            torch.cuda.synchronize()
            pl.close()

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e2e_dev = {"ms_per_step": (time.perf_counter() - t0) * 1e3 / args.steps,
                   "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                   "call": "DeviceBatch from pinned tensors + Plan + forward_partials + "
                           "backward_partials + copies back, one step at a time"}

    # end-to-end forward scoring from host memory (the host workflow of Sec. III-A) on the
    # NA12878-shaped stand-in of Table I: pipelined subsets, host packing and copies included
    hostpipe = None
    if not args.no_e2e and rank == 0:
        na = synth.na12878_like()
        na_cells = synth.cells(na)
        na_opts = phmm.autotune(phmm.DeviceBatch(na, dev), which=1, sample_pairs=32768)
        sub_cells = 1 << 33
        phmm.score_host(na, na_opts, subset_cells=sub_cells)
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            phmm.score_host(na, na_opts, subset_cells=sub_cells)
            ts.append(time.perf_counter() - t0)
        t_na = statistics.median(ts)
        na_in = sum(np.asarray(na[k]).nbytes for k in ("read_bases", "base_q", "ins_q", "del_q",
                                                       "read_off", "hap_bases", "hap_off",
                                                       "pair_read", "pair_hap"))
        hostpipe = {"workload": "na12878_like: 100,000 regions of 1..6 haplotypes (30..521) x "
                                "2..30 reads (10..151), "
                                f"{len(na['pair_read'])} pairs, {na_cells} cells",
                    "call": "phmm_score_host (forward, host arrays in and out)",
                    "subset_cells": sub_cells, "ms": t_na * 1e3,
                    "gcups": na_cells / t_na / 1e9, "h2d_bytes": int(na_in),
                    "d2h_bytes": int(len(na["pair_read"]) * 9)}
        del na

    # max over ranks of the step time
    if dist is not None:
        t = torch.tensor([ms, ms_fwd, e2e["ms_per_step"] if e2e else 0.0, ms_two], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ms_fwd, ms_two = float(t[0]), float(t[1]), float(t[3])
        if e2e:
            e2e["ms_per_step"] = float(t[2])
    total_cells = full_cells if args.shard else cells * ws
    value = total_cells / (ms * 1e-3) / 1e9
    fwd_gcups = total_cells / (ms_fwd * 1e-3) / 1e9
    if e2e:
        e2e["value"] = total_cells / (e2e["ms_per_step"] * 1e-3) / 1e9
    if e2e_dev:
        e2e_dev["value"] = total_cells / (e2e_dev["ms_per_step"] * 1e-3) / 1e9

    # roofline of the dominant kernel: the adjoint wavefront (FP32 pipe bound)
    peak = SMS * FP32_LANES * SM_MAX_MHZ * 1e6 / 1e12  # T lane-ops/s at the max SM clock
    adj = statistics.median(adj_ms) if adj_ms else float("nan")
    wf = statistics.median(wf_ms)
    dom_bwd = adj > wf
    if dom_bwd:
        achieved = cells * BWD_OPS_SCOPE / (adj * 1e-3) / 1e12
        achieved_min = cells * BWD_OPS_PER_CELL / (adj * 1e-3) / 1e12
        kname = "wf_backward (adjoint wavefront, all groups of a step)"
    else:
        achieved = cells * FWD_OPS_SCOPE / (wf * 1e-3) / 1e12
        achieved_min = cells * FWD_OPS_PER_CELL / (wf * 1e-3) / 1e12
        kname = "wf_forward (FP32 wavefront, all groups of a step)"
    fwd_wf_achieved = cells * FWD_OPS_SCOPE / (wf * 1e-3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {WORKLOAD_DESC[args.workload]}",
                   "pairs": full_pairs if args.shard else P * ws, "cells": total_cells,
                   "step": ("log10 L and d(loss)/d(quals, gcp) of every pair with dL = 1: "
                            "phmm_forward_partials (the adjoint sweep's own forward gives "
                            "log10 L; pairs it cannot represent finished in FP64) + "
                            "phmm_backward_partials (FP64 per-read reduction weighted by dL)"),
                   "first_line": "FP32 with per-lane exponents (FP64 rescue when unrepresentable)",
                   "l2": "inputs larger than L2 (no flush)",
                   "parallelism": (f"one batch split by read over {ws} ranks (d/dgcp "
                                   f"all-reduced per step)" if args.shard else f"weak x{ws}"),
                   "group_tables": ("built-in" if args.no_tune else
                                    f"phmm_autotune (32768-pair samples per 16-row read-length "
                                    f"range, {t_tune:.2f} s, outside the timed region)"),
                   "warps_per_block": {"forward": int(opts.warps_per_block),
                                       "adjoint": int(opts.bwd_warps_per_block)}},
        "two_call_step": {"calls": "phmm_forward (graph) + phmm_backward",
                          "ms_per_step": ms_two, "gcups": total_cells / (ms_two * 1e-3) / 1e9},
        "fwd_gcups": fwd_gcups,
        "fwd_wavefront_gcups": cells / (wf * 1e-3) / 1e9,
        "fwd_rescue_ms": statistics.median(resc_ms),
        "adjoint_ms": adj, "grad_reduce_ms": statistics.median(red_ms) if red_ms else None,
        "rescued_fraction": rescued,
        "plain_fp32_kernel": {"workload": "c0_plain: 16 haplotypes (300) x 64 reads (150), "
                                          "1,024 pairs, 46.08 M cells; 16 lanes x 12 rows, "
                                          "no binning, no rescue",
                              "gcups": c0_cells / (plain_ms * 1e-3) / 1e9,
                              "wavefront_gcups": c0_cells / (statistics.median(c0_wf) * 1e-3) / 1e9,
                              "same_batch": {"group": "16 lanes x 20 rows, plain FP32, no "
                                                      "binning, no rescue",
                                             "gcups": cells / (plain_same_ms * 1e-3) / 1e9}},
        "fp32_pipe": {"ffma_tops": ffma / 1e12, "ffma2_tops": ffma2 / 1e12,
                      "dfma_tops": dfma / 1e12, "derived_peak_tops": peak,
                      "fwd_frac": fwd_wf_achieved / peak,
                      "fwd_frac_reduced_count": fwd_wf_achieved * FWD_OPS_PER_CELL
                      / FWD_OPS_SCOPE / peak,
                      "ops_per_cell": {"scope_table": {"fwd": FWD_OPS_SCOPE, "bwd": BWD_OPS_SCOPE},
                                       "reduced": {"fwd": FWD_OPS_PER_CELL,
                                                   "bwd": BWD_OPS_PER_CELL}}},
        "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                     "unit": "T FP32 lane-ops/s", "frac": achieved / peak,
                     "ops_per_cell": BWD_OPS_SCOPE if dom_bwd else FWD_OPS_SCOPE,
                     "achieved_reduced_count": achieved_min,
                     "frac_reduced_count": achieved_min / peak,
                     "traffic": cells * BWD_DRAM_BYTES_PER_CELL if dom_bwd else None,
                     "traffic_source": ("ncu dram__bytes_read+write of the adjoint on c3_grad "
                                        f"({BWD_DRAM_BYTES_PER_CELL:.2f} B/cell), scaled by this "
                                        "step's cells"
                                        if dom_bwd else None)},
        "gpu_launches": launches * args.steps,
        "clocks": sample_clk,
    }
    if e2e:
        line["e2e"] = e2e
    if e2e_dev:
        line["e2e_device_api"] = e2e_dev
    if hostpipe:
        line["host_pipeline_fwd"] = hostpipe
    if rank == 0 and not args.no_cpu_baseline:
        g, ocells, kp, dt, cores = oracle_sample(batch, 15.0)
        line["cpu_baseline"] = {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{kp} pairs (seeded random subset of {args.workload}),"
                                          f" forward + adjoint in FP64, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
