"""Benchmark of the FMM cell-interaction hot path on one or more B300s.

One step = the whole path over the uniform 64^3 polytrope workload (512 leaf
sub-grids plus the coarse levels 0-2: 585 sub-grids, 299,520 cells):
moments from densities, both interaction passes as persistent launches
replayed from a CUDA graph (multipole pass at the coarse levels, point-mass
pass with near field at the leaves), the adjoint of both passes (multipole
sources gather over the transposed stencil, point masses receive theirs by
target) for a seeded L-bar, and the adjoint of the moments.  Throughput =
(forward + adjoint pairs) / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the same
workload (the path needs no data exchange between replicas); value = pairs of
all ranks / max over ranks of the timed region.  The reference arm times the
CPU oracle (the slow, plain FP64 implementation the tests check against) on a
bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-cell interactions/s FP64 (fwd, fwd+adjoint) and % of B300 FP64 roofline"
UNIT = "interactions/s"
WORKLOAD = ("uniform level: 512 leaf sub-grids (64^3 cells, h=1) + coarse levels 0-2, n=1 polytrope "
            "R=28 rho_c=1 floor 1e-10 centred; multipole and monopole passes as batched launches, then the adjoint")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--schedule", choices=["persistent", "per_subgrid"], default="persistent")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile", default=None, help="WxB: warps per block x blocks per SM (skips the autotuner)")
    ap.add_argument("--workload", choices=["polytrope64", "adaptive", "binary", "integration"], default="polytrope64",
                    help="polytrope64: the headline workload; adaptive: 4,641-sub-grid octree (levels 3-6); "
                         "binary: rotating binary star, levels 3-7, a new octree every step")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = os.environ.get("OT_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    on_gpu = dist.get_backend() == "nccl"
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if on_gpu else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        busy = [s for s in sm if mx and s > 0.25 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the workload
# ---------------------------------------------------------------------------

WORKLOADS = {
    "polytrope64": WORKLOAD,
    "adaptive": ("adaptive octree, levels 3-6 (4,641 sub-grids, 4,061 leaves), n=1 polytrope with seeded centre, "
                 "refined where rho > 1e-3 rho_c, 2:1 balanced; both passes as batched launches, then the adjoint"),
    "binary": ("rotating binary star: two n=1 polytropes (q=0.5, R=24 and 19, 60 apart), levels 3-7 "
               "(~9,500 sub-grids, ~8,300 leaves, 4.25M leaf cells), rotated 0.01 rad per step, octree rebuilt "
               "each step; both passes + adjoint per step"),
}


def make_workload(name="polytrope64", step=0):
    import synth
    if name == "adaptive":
        tree, rho, _ = synth.config3()
    elif name == "binary":
        tree, rho = synth.config5_step(step)
    else:
        tree, rho = synth.config2()
    # a seeded N(0,1) L-bar on all 20 components of every cell, so every
    # adjoint lane does full work
    rng = np.random.default_rng(4 + step)
    Lbar = rng.standard_normal((tree.n, 20, 512))
    return tree, rho, Lbar, None


def fwd_flops(info):
    """algorithmic FP64 flops of one forward launch over the in-domain pairs,
    counted by the library from its stencil lists (2 per FMA, 1 per add)"""
    return info["flops_fwd"]


# DRAM bytes (read + written) of one forward_kernel<1> launch (the multipole
# pass) on the 64^3 polytrope workload with the 8x2 tile, from an ncu capture
# of that kernel (dram__bytes_read.sum + dram__bytes_write.sum).  Reported
# only for that workload and tile; None once the kernel changes.
MULTIPOLE_DRAM_BYTES_POLYTROPE64 = 174_318_080     # 140.63 MB read + 33.69 MB written
MULTIPOLE_DRAM_TILE = (8, 2)

# Nominal FP64 rate of a B300 (1.25 TFLOP/s) at its maximum SM clock (2032 MHz):
# 1.25e12 / (148 SMs * 2.032e9) = 4.16 FP64 flop per clock per SM.
NOMINAL_FP64_TFLOPS = 1.25
NOMINAL_SM_MHZ = 2032.0


def fp64_peak(ot, dev, stream):
    """Best FP64 FMA rate of the probe kernel over both operand patterns and
    1, 2, 4, 8 resident blocks of 256 threads per SM."""
    import torch
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    best, cfg = 0.0, None
    for variant in (0, 1):
        for per_sm in (1, 2, 4, 8):
            blocks, iters = nsm * per_sm, 16000 // per_sm
            out = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
            ot.fp64_fma_probe(out, blocks, 100, variant)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
            for a, b in ev:
                a.record(stream)
                ot.fp64_fma_probe(out, blocks, iters, variant)
                b.record(stream)
            torch.cuda.synchronize()
            ms = min(a.elapsed_time(b) for a, b in ev)
            tf = 2.0 * blocks * 256 * iters * 16 / (ms * 1e-3) / 1e12
            if tf > best:
                best, cfg = tf, {"variant": variant, "blocks_per_sm": per_sm, "ms": round(ms, 3)}
    return best, cfg


def aggregate(world, steps, pairs_step, local_seconds):
    """Whole-job throughput: pairs of all ranks / the slowest rank's time."""
    total_s = max_over_ranks(local_seconds, world)
    return world * steps * pairs_step / total_s, total_s * 1e3 / steps


def run_ours(args, rank, world):
    import torch
    import paper_2303_08058_b300 as ot

    dev = torch.device("cuda", torch.cuda.current_device())
    if args.workload == "binary":
        return run_binary(args, rank, world)
    if args.workload == "integration":
        return run_integration(args, rank, world)
    tree, rho_h, Lbar_h, _ = make_workload(args.workload)
    g = ot.OTGrid.from_tree(tree)
    sched = ot.OT_SCHED_PER_SUBGRID if args.schedule == "per_subgrid" else ot.OT_SCHED_PERSISTENT
    g.set_schedule(sched, 4, 0, not args.no_graph)
    rho = torch.as_tensor(rho_h, device=dev)
    Lbar = torch.as_tensor(Lbar_h, device=dev)
    M, m = g.moments(rho)
    L = g.zeros(tree.n, 20, 512)
    Lc = g.zeros(tree.n, 3, 512)
    tuned = None
    if args.tile:
        w, b = (int(x) for x in args.tile.lower().split("x"))
        g.set_schedule(sched, w, b, not args.no_graph)
    elif not args.no_autotune and sched == ot.OT_SCHED_PERSISTENT:
        tuned = g.autotune(M, m, L, Lc)      # tile shape of the persistent launch
    info = g.info()
    Mb = g.zeros(tree.n, 20, 512)
    mb = g.zeros(tree.n, 512)
    rb = g.zeros(tree.n, 512)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step():
        g.moments(rho, M, m)
        g.interactions(M, m, L, Lc)
        g.backward(Lbar, Mb, mb)
        g.moments_backward(Mb, mb, rb)

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.check()

    # -- timed region: K steps, L2 flushed between steps (outside the events) --
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    g.check()

    # -- the forward and the adjoint calls, each timed alone ------------------
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in fe:
        flush.zero_()
        a.record(stream)
        g.interactions(M, m, L, Lc)
        b.record(stream)
    be = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in be:
        flush.zero_()
        a.record(stream)
        g.backward(Lbar, Mb, mb)
        b.record(stream)
    torch.cuda.synchronize()
    fwd_ms = statistics.median(a.elapsed_time(b) for a, b in fe)
    adj_ms = statistics.median(a.elapsed_time(b) for a, b in be)
    # the same forward launch with double-float point-mass contractions
    g.set_precision(ot.OT_PREC_DF64_POINT_MASS)
    g.interactions(M, m, L, Lc)
    de = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in de:
        flush.zero_()
        a.record(stream)
        g.interactions(M, m, L, Lc)
        b.record(stream)
    torch.cuda.synchronize()
    df_ms = statistics.median(a.elapsed_time(b) for a, b in de)
    # and with the multipole contractions in double-float too
    g.set_precision(ot.OT_PREC_DF64)
    g.interactions(M, m, L, Lc)
    de2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in de2:
        flush.zero_()
        a.record(stream)
        g.interactions(M, m, L, Lc)
        b.record(stream)
    torch.cuda.synchronize()
    df2_ms = statistics.median(a.elapsed_time(b) for a, b in de2)
    g.backward(Lbar, Mb, mb)
    da = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in da:
        flush.zero_()
        a.record(stream)
        g.backward(Lbar, Mb, mb)
        b.record(stream)
    torch.cuda.synchronize()
    dfa_ms = statistics.median(a.elapsed_time(b) for a, b in da)
    g.set_precision(ot.OT_PREC_FP64)
    # each variant as its own launch: the multipole pass, the point-mass pass
    variant_ms = {}
    for name, call in (("multipole", lambda: g.multipole(M, L, Lc)), ("monopole", lambda: g.monopole(m, L))):
        call()
        ve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a, b in ve:
            flush.zero_()
            a.record(stream)
            call()
            b.record(stream)
        torch.cuda.synchronize()
        variant_ms[name] = statistics.median(a.elapsed_time(b) for a, b in ve)
    # the same passes about centres of mass (derivatives evaluated per pair)
    Mc, mc, Cc = g.moments_com(rho)
    g.interactions_com(Mc, mc, Cc, L, Lc)
    g.backward_com(Lbar, Cc, Mb, mb)
    ce = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in ce:
        flush.zero_()
        a.record(stream)
        g.interactions_com(Mc, mc, Cc, L, Lc)
        b.record(stream)
    cb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in cb:
        flush.zero_()
        a.record(stream)
        g.backward_com(Lbar, Cc, Mb, mb)
        b.record(stream)
    torch.cuda.synchronize()
    g.check()
    com_fwd_ms = statistics.median(a.elapsed_time(b) for a, b in ce)
    com_adj_ms = statistics.median(a.elapsed_time(b) for a, b in cb)
    del Mc, mc, Cc
    clk = clocks.stop()

    # -- FP64 FMA peak, measured on this GPU at the clocks it runs now --------
    peak_tflops, probe_cfg = fp64_peak(ot, dev, stream)

    # -- end to end: host buffers, copies inside the timed region -------------
    rho_pin = torch.as_tensor(rho_h).pin_memory()
    Lbar_pin = torch.as_tensor(Lbar_h).pin_memory()
    L_out = torch.empty((tree.n, 20, 512), dtype=torch.float64).pin_memory()
    rb_out = torch.empty((tree.n, 512), dtype=torch.float64).pin_memory()
    # one step through OTGrid.step_host: the copies of L-bar (in) and L (out)
    # overlap the forward and the adjoint on a side stream
    work = {}
    g.step_host(rho_pin, Lbar_pin, L_out, rb_out, work)
    e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in e2e_ev:
        flush.zero_()
        a.record(stream)
        g.step_host(rho_pin, Lbar_pin, L_out, rb_out, work)
        b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = statistics.median(a.elapsed_time(b) for a, b in e2e_ev)

    pairs_fwd = info["pairs_multipole"] + info["pairs_monopole"]
    pairs_step = 2 * pairs_fwd
    value, ms_per_step = aggregate(world, args.steps, pairs_step, sum(step_ms) / 1e3)
    sm_mhz = clk.get("sm_mhz") or NOMINAL_SM_MHZ
    peak = NOMINAL_FP64_TFLOPS * sm_mhz / NOMINAL_SM_MHZ
    ach = fwd_flops(info) / (fwd_ms * 1e-3) / 1e12
    peak_ops = peak / 2                       # FP64 pipe slots: one per FMA
    ach_ops = info["fp64_ops_fwd"] / (fwd_ms * 1e-3) / 1e12
    adj_ops = info["fp64_ops_adj"] / (adj_ms * 1e-3) / 1e12
    multi_ms = variant_ms["multipole"]
    multi_ops = info["fp64_ops_fwd_multi"] / (multi_ms * 1e-3) / 1e12
    tile = (info["warps_per_block"], info["blocks_per_sm"])
    traffic = (MULTIPOLE_DRAM_BYTES_POLYTROPE64
               if args.workload == "polytrope64" and tile == MULTIPOLE_DRAM_TILE else None)
    n_m2m = int(len({int(l) for l in tree.level[tree.is_leaf == 0]}))
    # moments (cube + M2M levels); forward: prescale, the multipole x table,
    # the multipole launch, the masses' x and (x, y) tables, the point-mass
    # launch; adjoint: prescale, the L-bar x butterflies, the gather launch,
    # the scatter launch, the deferred scatter pass; moment adjoint
    launches_step = (1 + n_m2m) + 6 + 5 + (1 if info["n_virtual"] else 0) + (1 + n_m2m + 1)
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded polytrope densities, seeded L-bar)",
        "config": {"workload": WORKLOADS[args.workload], "subgrids": tree.n, "cells": tree.n * 512,
                   "pairs_fwd": pairs_fwd, "pairs_adj": pairs_fwd,
                   "pairs_multipole": info["pairs_multipole"], "pairs_monopole": info["pairs_monopole"],
                   "schedule": args.schedule, "graph": not args.no_graph,
                   "tile": {"warps_per_block": info["warps_per_block"], "blocks_per_sm": info["blocks_per_sm"]},
                   "autotuned": tuned, "l2": "flushed between steps (256 MB write outside the events)",
                   "parallelism": f"replicas x{world}"},
        "fwd": {"value": pairs_fwd / (fwd_ms * 1e-3), "unit": UNIT, "ms": fwd_ms,
                "pairs_in_domain": pairs_fwd, "pairs_padded": info["pairs_padded_fwd"]},
        "variants": {
            "multipole": {"value": info["pairs_multipole"] / (variant_ms["multipole"] * 1e-3), "unit": UNIT,
                          "ms": variant_ms["multipole"], "pairs": info["pairs_multipole"],
                          "pairs_with_angular_term": info["pairs_angular"]},
            "monopole": {"value": info["pairs_monopole"] / (variant_ms["monopole"] * 1e-3), "unit": UNIT,
                         "ms": variant_ms["monopole"], "pairs": info["pairs_monopole"]},
            "boundary": {"pairs": info["pairs_virtual"] + info["pairs_refined"],
                         "pairs_virtual_source": info["pairs_virtual"],
                         "pairs_refined_target": info["pairs_refined"],
                         "note": "coarse-fine pairs: point masses that are virtual descendants of a coarser "
                                 "leaf, and coarse leaf targets refined virtually against a refined neighbour's "
                                 "children; both run inside the monopole launch"},
            "note": "one pass per call; fwd runs both passes (two persistent launches)"},
        "adjoint": {"value": pairs_fwd / (adj_ms * 1e-3), "unit": UNIT, "ms": adj_ms},
        "fwd_df64_point_mass": {"value": pairs_fwd / (df_ms * 1e-3), "unit": UNIT, "ms": df_ms,
                                "note": "point-mass pairs in double-float on the FP32 pipe (within 1e-12 of "
                                        "the FP64 result; leaves without x tables keep FP64 point-mass classes); "
                                        "reported beside the FP64 numbers, not as them"},
        "fwd_df64": {"value": pairs_fwd / (df2_ms * 1e-3), "unit": UNIT, "ms": df2_ms,
                     "note": "point-mass and multipole contractions (with the angular term) in double-float "
                             "on the FP32 pipe, within 1e-12 of the oracle's sum of |terms| (leaves without x "
                             "tables keep FP64 point-mass classes); beside the FP64 numbers, not as them"},
        "adjoint_df64": {"value": pairs_fwd / (dfa_ms * 1e-3), "unit": UNIT, "ms": dfa_ms,
                         "fwd_plus_adjoint": 2 * pairs_fwd / ((df2_ms + dfa_ms) * 1e-3),
                         "note": "the adjoint's multipole gather and point-mass scatter in double-float "
                                 "(OT_PREC_DF64); beside the FP64 numbers, not as them"},
        "com": {"fwd": {"value": pairs_fwd / (com_fwd_ms * 1e-3), "unit": UNIT, "ms": com_fwd_ms,
                        "tflops": info["flops_fwd_com"] / (com_fwd_ms * 1e-3) / 1e12,
                        "frac": info["flops_fwd_com"] / (com_fwd_ms * 1e-3) / 1e12 / peak},
                "adjoint": {"value": pairs_fwd / (com_adj_ms * 1e-3), "unit": UNIT, "ms": com_adj_ms,
                            "tflops": info["flops_adj_com"] / (com_adj_ms * 1e-3) / 1e12,
                            "frac": info["flops_adj_com"] / (com_adj_ms * 1e-3) / 1e12 / peak},
                "note": "centre-of-mass expansion centres: the same pairs, derivatives of G evaluated "
                        "per pair at R = C_A - C_B; fractions of the same FP64 peak"},
        "roofline": {"bound": "alu",
                     "kernel": ("forward_kernel<1> (the multipole pass: non-leaf targets, multipole sources "
                                "with the angular term; one launch, the step's largest)"),
                     "achieved": multi_ops, "peak": peak_ops, "unit": "Tinst/s", "frac": multi_ops / peak_ops,
                     "traffic": traffic,
                     "traffic_unit": "bytes per launch (ncu, %dx%d tile)" % MULTIPOLE_DRAM_TILE,
                     "unit_note": ("FP64 pipe thread-instructions per second (an FMA or an add is one pipe slot); "
                                   "achieved: the algorithmic FP64 instructions of the in-domain pairs per "
                                   "launch (library count) over the CUDA-event time of the multipole call (the "
                                   "launch and its O(cells) prologue kernels)"),
                     "peak_source": (f"nominal B300 FP64 {NOMINAL_FP64_TFLOPS} TFLOP/s = "
                                     f"{NOMINAL_FP64_TFLOPS / 2} T FMA/s at {NOMINAL_SM_MHZ:.0f} MHz, "
                                     f"scaled to the median SM clock sampled in this run ({sm_mhz:.0f} MHz)"),
                     "fp64_pipe_busy": info["ops_fwd_multi"] / (multi_ms * 1e-3) / (peak_ops * 1e12),
                     "forward": {"kernels": "forward_kernel<1> then forward_kernel<2> (the two passes)",
                                 "achieved": ach_ops, "frac": ach_ops / peak_ops,
                                 "fp64_pipe_busy": info["ops_fwd"] / (fwd_ms * 1e-3) / (peak_ops * 1e12)},
                     "adjoint": {"kernels": ("adjoint_kernel<1> (multipole gather) then adjoint_kernel<4> "
                                             "(point masses by target)"),
                                 "achieved": adj_ops, "frac": adj_ops / peak_ops,
                                 "fp64_pipe_busy": info["ops_adj"] / (adj_ms * 1e-3) / (peak_ops * 1e12)},
                     "flops": {"forward_achieved": ach, "adjoint_achieved": info["flops_adj"] / (adj_ms * 1e-3) / 1e12,
                               "peak": peak, "unit": "TFLOP/s", "forward_frac": ach / peak,
                               "note": "algorithmic FLOPs of the algorithm run (2 per FMA, 1 per add)"},
                     "probe_tflops": peak_tflops, "probe": probe_cfg},
        "e2e": {"value": world * pairs_step / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": int(rho_pin.numel() * 8 + Lbar_pin.numel() * 8),
                "d2h_bytes_per_step": int(L_out.numel() * 8 + rb_out.numel() * 8), "ms": e2e_ms},
        "gpu_launches": launches_step * args.steps,
        "clocks": clk,
        "wall_s": wall,
    }
    return res, tree, rho_h


def run_binary(args, rank, world):
    """Rotating binary star: each of `--steps` rotation steps builds its
    octree (host, untimed), then runs the path (moments, both passes,
    adjoint, moment adjoint) timed with events on the stream."""
    import torch
    import paper_2303_08058_b300 as ot
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    step_ms, pairs, setup_s, tile = [], 0, 0.0, None
    sched = ot.OT_SCHED_PER_SUBGRID if args.schedule == "per_subgrid" else ot.OT_SCHED_PERSISTENT
    clocks.start()
    for k in range(-1, args.steps):        # step -1: warm-up (step 0 untimed)
        t0 = time.perf_counter()
        tree, rho_h, Lbar_h, _ = make_workload("binary", max(k, 0))
        g = ot.OTGrid.from_tree(tree)
        rho = torch.as_tensor(rho_h, device="cuda")
        Lbar = torch.as_tensor(Lbar_h, device="cuda")
        M, m = g.moments(rho)
        L, Lc = g.zeros(tree.n, 20, 512), g.zeros(tree.n, 3, 512)
        if tile is None and sched == ot.OT_SCHED_PERSISTENT and not args.tile:
            tuned = g.autotune(M, m, L, Lc)
            tile = (tuned["warps_per_block"], tuned["blocks_per_sm"])
        elif args.tile:
            tile = tuple(int(x) for x in args.tile.lower().split("x"))
        g.set_schedule(sched, *(tile or (4, 0)), not args.no_graph)
        Mb, mb, rb = g.zeros(tree.n, 20, 512), g.zeros(tree.n, 512), g.zeros(tree.n, 512)
        g.interactions(M, m, L, Lc)          # records the graph (untimed)
        g.backward(Lbar, Mb, mb)
        torch.cuda.synchronize()
        setup_s += time.perf_counter() - t0
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        g.moments(rho, M, m)
        g.interactions(M, m, L, Lc)
        g.backward(Lbar, Mb, mb)
        g.moments_backward(Mb, mb, rb)
        b.record(stream)
        torch.cuda.synchronize()
        g.check()
        if k >= 0:
            step_ms.append(a.elapsed_time(b))
            info = g.info()
            pairs += 2 * (info["pairs_multipole"] + info["pairs_monopole"])
        g.close()
    clk = clocks.stop()
    value, ms_per_step = aggregate(world, args.steps, pairs / max(args.steps, 1), sum(step_ms) / 1e3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": 1,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (analytic binary-star densities, seeded L-bar)",
            "config": {"workload": WORKLOADS["binary"], "schedule": args.schedule, "graph": not args.no_graph,
                       "tile": tile, "pairs_per_step": pairs / max(args.steps, 1),
                       "host_setup_s_per_step": setup_s / (args.steps + 1)},
            "step_ms": step_ms, "clocks": clk}, None, None


def run_integration(args, rank, world):
    """The completion-notification study on the 64^3 and adaptive workloads:
    per-sub-grid forward launches over 1-32 streams with completions seen by
    stream sync, host callbacks or event polling, against one batched
    persistent launch (median of --steps repetitions)."""
    import torch
    import paper_2303_08058_b300 as ot
    names = {0: "stream_sync", 1: "host_callback", 2: "event_polling", 3: "batched_persistent"}
    out = {}
    for wl in ("polytrope64", "adaptive"):
        tree, rho_h, _, _ = make_workload(wl)
        g = ot.OTGrid.from_tree(tree)
        g.set_schedule(ot.OT_SCHED_PERSISTENT, 4, 2, False)
        M, m = g.moments(torch.as_tensor(rho_h, device="cuda"))
        rows = []
        for mech in (0, 1, 2, 3):
            for ns in ((1,) if mech == 3 else (1, 4, 16, 32)):
                g.completion_study(M, m, mech, ns)            # warm-up
                runs = [g.completion_study(M, m, mech, ns)[0] for _ in range(max(args.steps, 1))]
                med = sorted(runs, key=lambda r: r["wall_ms"])[len(runs) // 2]
                rows.append({"mechanism": names[mech], "streams": ns, "wall_ms": med["wall_ms"],
                             "mean_latency_us": med["mean_latency_us"], "max_latency_us": med["max_latency_us"],
                             "launches": med["launches"]})
        out[wl] = {"subgrids": tree.n, "rows": rows}
        g.close()
    return {"metric": "completion notification of per-sub-grid launches (wall ms per forward pass)",
            "workload": "integration study", "impl": "ours", "results": out, "steps": args.steps}, None, None


def cpu_baseline(tree, rho_h, seconds, seed=7):
    """The oracle as it stands on this host's cores: forward of both passes on
    seeded random target cells, batches until `seconds` have elapsed."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    M = oracle.moments(tree, rho_h)
    m = np.ascontiguousarray(M[:, 0, :])
    rng = np.random.default_rng(seed)
    pairs, t_used, ntg = 0, 0.0, 0
    while t_used < seconds:
        tg = np.stack([rng.integers(0, tree.n, 64 * cores), rng.integers(0, 512, 64 * cores)], 1).astype(np.int32)
        t0 = time.perf_counter()
        r1 = oracle.run_pass(tree, "multipole", M=M, targets=tg)
        r2 = oracle.run_pass(tree, "monopole", m=m, targets=tg)
        t_used += time.perf_counter() - t0
        pairs += r1["npairs"] + r2["npairs"]
        ntg += len(tg)
    # the same oracle on one thread, a shorter sample
    oracle.set_threads(1)
    pairs1, t1 = 0, 0.0
    while t1 < max(2.0, seconds / 6):
        tg = np.stack([rng.integers(0, tree.n, 64), rng.integers(0, 512, 64)], 1).astype(np.int32)
        t0 = time.perf_counter()
        r1 = oracle.run_pass(tree, "multipole", M=M, targets=tg)
        r2 = oracle.run_pass(tree, "monopole", m=m, targets=tg)
        t1 += time.perf_counter() - t0
        pairs1 += r1["npairs"] + r2["npairs"]
    oracle.set_threads(cores)
    cpu = ""
    try:
        with open("/proc/cpuinfo") as f:
            cpu = next((ln.split(":", 1)[1].strip() for ln in f if ln.startswith("model name")), "")
    except OSError:
        pass
    return {"value": pairs / t_used, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"forward of both passes for {ntg} random target cells of the workload "
                      f"({pairs} pairs, {t_used:.1f} s)",
            "single_thread": {"value": pairs1 / t1, "unit": UNIT, "sample": f"{pairs1} pairs, {t1:.1f} s"},
            "cpu": cpu}


def run_reference(args, rank, world):
    """The oracle on the host cores, each step a bounded sample: forward of both
    passes and the transposed sums for 32 x cores random target cells."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    tree, rho_h, Lbar_h, _ = make_workload()
    M = oracle.moments(tree, rho_h)
    m = np.ascontiguousarray(M[:, 0, :])
    rng = np.random.default_rng(8)
    per = 32 * cores

    per_adj = max(8, per // cores)   # the transposed sums scatter, so they run on one core

    def step():
        tg = np.stack([rng.integers(0, tree.n, per), rng.integers(0, 512, per)], 1).astype(np.int32)
        r1 = oracle.run_pass(tree, "multipole", M=M, targets=tg)
        r2 = oracle.run_pass(tree, "monopole", m=m, targets=tg)
        _, a1 = oracle.pass_adjoint(tree, "multipole", Lbar_h, with_s="pairs", targets=tg[:per_adj])
        _, a2 = oracle.pass_adjoint(tree, "monopole", Lbar_h, with_s="pairs", targets=tg[:per_adj])
        return r1["npairs"] + r2["npairs"] + a1 + a2
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    pairs = sum(step() for _ in range(args.steps))
    dt = time.perf_counter() - t0
    value = pairs / dt
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "subgrids": tree.n, "cells": tree.n * 512,
                       "parallelism": "host cores (OpenMP)"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"per step: forward of both passes for {per} random target cells "
                                       f"(OpenMP) and the transposed sums of both passes for {per_adj} of them "
                                       f"(serial scatter)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        world = int(os.environ.get("WORLD_SIZE", "1"))
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank, world)))
        return 0
    rank, world = dist_init(args)
    res, tree, rho_h = run_ours(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1 and tree is not None:
            res["cpu_baseline"] = cpu_baseline(tree, rho_h, args.cpu_seconds)
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
