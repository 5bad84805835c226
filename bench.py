"""Benchmark of the FMM cell-interaction hot path on one or more B300s.

Default workload: the rotating binary star -- two n = 1 polytropes (mass
ratio 0.5, radii 24 and 19, 60 apart) on an adaptive octree of levels 3-7
(about 9,500 sub-grids, 8,300 leaves, 4.25M leaf cells), rotated by 0.01 rad
per step; every step has its own octree.  One step = the whole path on that
step's tree: moments from densities, both interaction passes as persistent
launches replayed from CUDA graphs (multipole pass at the non-leaf levels,
point-mass pass with near field, virtual descendants and refined coarse
targets at the leaves), the adjoint of both passes for a seeded L-bar, and
the adjoint of the moments.  Throughput = (forward + adjoint pairs) / step
time, summed over the timed steps.  Building each step's octree, grid and
graphs is host set-up outside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload binary|polytrope64|adaptive|integration]

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

WORKLOADS = {
    "binary": ("rotating binary star: two n=1 polytropes (q=0.5, R=24 and 19, 60 apart, domain side 390), "
               "adaptive octree levels 3-7 refined where rho > 1e-3 rho_c and 2:1 balanced (~9,500 sub-grids, "
               "~8,300 leaves, ~4.25M leaf cells), rotated 0.01 rad per step, octree rebuilt each step; "
               "moments, both passes as batched persistent launches in CUDA graphs, adjoint of both passes "
               "and of the moments per step"),
    "polytrope64": ("uniform level: 512 leaf sub-grids (64^3 cells, h=1) + coarse levels 0-2, n=1 polytrope "
                    "R=28 rho_c=1 floor 1e-10 centred; multipole and monopole passes as batched launches, "
                    "then the adjoint"),
    "adaptive": ("adaptive octree, levels 3-6 (4,641 sub-grids, 4,061 leaves), n=1 polytrope with seeded centre, "
                 "refined where rho > 1e-3 rho_c, 2:1 balanced; both passes as batched launches, then the adjoint"),
    "adaptive_small": ("adaptive octree, levels 3-6, the same recipe with a smaller star (R = 3 level-3 cells, 1,385 "
                       "sub-grids), "
                       "for profiler captures that must stay within a few GB; both passes, then the adjoint"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--schedule", choices=["persistent", "per_subgrid"], default="persistent")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measurements beside the headline (per-launch roofline, per-sub-grid "
                         "launches, the 64^3 workload, double-float and centre-of-mass variants)")
    ap.add_argument("--tile", default=None, help="WxB: warps per block x blocks per SM (skips the autotuner)")
    ap.add_argument("--workload", choices=["binary", "polytrope64", "adaptive", "adaptive_small", "integration"],
                    default="binary")
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


def aggregate(world, pairs_local, local_seconds, steps):
    """Whole-job throughput: pairs of all ranks / the slowest rank's time."""
    total_s = max_over_ranks(local_seconds, world)
    return world * pairs_local / total_s, total_s * 1e3 / max(steps, 1)


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
# inputs
# ---------------------------------------------------------------------------

def _binary_step(k):
    import synth
    return synth.config5_step(k)


def binary_inputs(steps, world):
    """The octrees and densities of binary-star steps 0..steps-1, built on
    the host by a pool of spawned processes (no CUDA state is inherited)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    procs = max(1, min(steps, (os.cpu_count() or 1) // max(world, 1)))
    if procs == 1:
        return [_binary_step(k) for k in range(steps)]
    with ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_binary_step, range(steps)))


def make_workload(name):
    import synth
    if name == "adaptive":
        tree, rho, _ = synth.config3()
    elif name == "adaptive_small":
        tree, rho, _ = synth.config3(radius_l3_cells=3.0)
    elif name == "binary":
        tree, rho = synth.config5_step(0)
    else:
        tree, rho = synth.config2()
    return tree, rho


def lbar_pool(n_max, seed=4):
    """A seeded N(0,1) L-bar on all 20 components of n_max sub-grids (every
    adjoint lane does full work); a step with n sub-grids uses the first n."""
    import torch
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.standard_normal((n_max, 20, 512))).pin_memory()


# ---------------------------------------------------------------------------
# timing helpers
# ---------------------------------------------------------------------------

def time_call(fn, stream, reps=5, flush=None, warm=True):
    """Median CUDA-event time (ms) of `fn` on `stream` over `reps` calls."""
    import torch
    if warm:
        fn()
    evs = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in evs)


def launch_breakdown(g, work, stream, flush=None):
    """The step's four interaction launches, each timed alone through its
    ABI call (the launch and its O(cells) prologue kernels), with the
    algorithmic and executed FP64 instructions the library counts for it."""
    info = g.info()
    W = work
    ms = {
        "multipole": time_call(lambda: g.multipole(W["M"], W["L"], W["Lc"]), stream, flush=flush),
        "monopole": time_call(lambda: g.monopole(W["m"], W["L"]), stream, flush=flush),
        "gather": time_call(lambda: g.backward(W["Lbar"], W["Mb"], None, want=(True, False)), stream, flush=flush),
        "scatter": time_call(lambda: g.backward(W["Lbar"], None, W["mb"], want=(False, True)), stream, flush=flush),
    }
    alg = {"multipole": info["fp64_ops_fwd_multi"], "monopole": info["fp64_ops_fwd"] - info["fp64_ops_fwd_multi"],
           "gather": info["fp64_ops_adj_multi"], "scatter": info["fp64_ops_adj"] - info["fp64_ops_adj_multi"]}
    exe = {"multipole": info["ops_fwd_multi"], "monopole": info["ops_fwd"] - info["ops_fwd_multi"],
           "gather": info["ops_adj_multi"], "scatter": info["ops_adj"] - info["ops_adj_multi"]}
    kernels = {"multipole": "forward_kernel<1> (multipole pass: non-leaf targets, multipole sources, angular term)",
               "monopole": "forward_kernel<2> (point-mass pass: leaf targets, near field, coarse-fine boundary)",
               "gather": "adjoint_kernel<1> (multipole sources gather over the transposed far stencil)",
               "scatter": "adjoint_kernel<4> (point masses receive their adjoint by target)"}
    return {k: {"ms": ms[k], "kernel": kernels[k], "fp64_inst": alg[k], "fp64_inst_executed": exe[k],
                "achieved": alg[k] / (ms[k] * 1e-3) / 1e12, "executed": exe[k] / (ms[k] * 1e-3) / 1e12}
            for k in ms}


# FP64 pipe of a B300: NVIDIA's nominal 1.25 TFLOP/s (0.625 T FMA/s) at the
# maximum SM clock of 2032 MHz is 2.08 thread-instructions per SM per clock.
NOMINAL_FP64_TFLOPS = 1.25
NOMINAL_SM_MHZ = 2032.0

# DRAM bytes (read + written) per launch of a launch's kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum, one pass) of that
# kernel as it is now, keyed by (workload, launch, tile); a key not here
# reports null.
DRAM_BYTES = {
    ("binary", "multipole", (8, 1)): 62_989_917_440 + 257_027_584,
    ("polytrope64", "multipole", (8, 2)): 3_366_929_664 + 152_704_256,
}


def fp64_peak(ot, dev, stream):
    """The FP64 pipe's measured issue rate: the probe kernel (independent
    FP64 chains in the instruction mix and operand pattern that keeps the pipe
    busiest) at 1, 2 and 4 resident blocks of 256 threads per SM; returns
    (thread-instructions per second, config)."""
    import torch
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    best, cfg = 0.0, None
    for variant in (0, 1, 2):
        for per_sm in (1, 2, 4):
            blocks = nsm * per_sm
            iters = (8000 if variant < 2 else 125) // per_sm
            out = torch.empty(blocks * 256, dtype=torch.float64, device=dev)
            ot.fp64_fma_probe(out, blocks, 50, variant)
            ms = time_call(lambda: ot.fp64_fma_probe(out, blocks, iters, variant), stream, reps=3, warm=False)
            inst = blocks * 256 * iters * ot.FP64_PROBE_FMA_PER_ROUND[variant]
            rate = inst / (ms * 1e-3)
            if rate > best:
                best, cfg = rate, {"variant": variant, "blocks_per_sm": per_sm, "ms": round(ms, 3)}
    return best, cfg


def roofline_block(launches, peak_inst, probe_cfg, sm_mhz, workload, info, pairs_fwd, fwd_ms, adj_ms):
    """The dominant launch's roofline in FP64 pipe thread-instructions per
    second against the probe's measured rate, with the nominal peak and the
    naive contraction's per-pair FLOP counts beside it."""
    tile = (info["warps_per_block"], info["blocks_per_sm"])
    dom = max(launches, key=lambda k: launches[k]["ms"])
    L = launches[dom]
    peak = peak_inst / 1e12
    nominal = NOMINAL_FP64_TFLOPS / 2 * (sm_mhz or NOMINAL_SM_MHZ) / NOMINAL_SM_MHZ
    # the naive contraction's per-pair FLOP counts (all 20 components, no
    # pairing, no classes): a multipole pair 84 FMAs (+40 for the angular
    # term at non-leaf targets), a point-mass pair 20 FMAs; the adjoint the
    # same; 2 flops per FMA
    naive_fwd = 2 * (84 * info["pairs_multipole"] + 40 * info["pairs_angular"] + 20 * info["pairs_monopole"])
    traffic = DRAM_BYTES.get((workload, dom, tile))
    return {
        "bound": "alu", "kernel": L["kernel"], "launch": dom,
        "achieved": L["achieved"], "peak": peak, "unit": "Tinst/s", "frac": L["achieved"] / peak,
        "traffic": traffic,
        "traffic_unit": ("bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, tile %dx%d)" % tile),
        "unit_note": ("FP64 pipe thread-instructions per second (one per FMA, add or multiply); achieved: the "
                      "algorithmic FP64 instructions of the launch's in-domain pairs (library count) over the "
                      "CUDA-event time of its ABI call (the launch and its O(cells) prologue kernels)"),
        "peak_source": (f"measured: the library's FP64 probe kernel on this GPU in this run ({probe_cfg}), "
                        f"of measured"),
        "executed_frac": L["executed"] / peak,
        "nominal": {"peak": nominal, "frac": L["achieved"] / nominal,
                    "note": (f"NVIDIA's nominal {NOMINAL_FP64_TFLOPS} TFLOP/s = {NOMINAL_FP64_TFLOPS / 2} T FMA/s "
                             f"at {NOMINAL_SM_MHZ:.0f} MHz, scaled to the median SM clock of the timed region")},
        "launches": {k: {"ms": v["ms"], "achieved": v["achieved"], "frac": v["achieved"] / peak,
                         "executed_frac": v["executed"] / peak} for k, v in launches.items()},
        "naive_flops": {"fwd_flop": naive_fwd, "forward_tflops": naive_fwd / (fwd_ms * 1e-3) / 1e12,
                        "adjoint_tflops": naive_fwd / (adj_ms * 1e-3) / 1e12,
                        "note": ("effective rate: the naive per-pair counts (multipole 168 flop + 80 for the angular "
                                 "term, point mass 40 flop) over the forward / adjoint time; above the FP64 peak "
                                 "because the kernels share one derivative row among up to 8 reflected sources "
                                 "(reflection classes), the traceless reduction and the pairings")},
    }


# ---------------------------------------------------------------------------
# the headline: rotating binary star
# ---------------------------------------------------------------------------

def run_binary(args, rank, world):
    import torch
    import paper_2303_08058_b300 as ot
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    sched = ot.OT_SCHED_PER_SUBGRID if args.schedule == "per_subgrid" else ot.OT_SCHED_PERSISTENT
    t_in = time.perf_counter()
    inputs = binary_inputs(args.steps, world)
    inputs_s = time.perf_counter() - t_in
    n_max = max(tree.n for tree, _ in inputs)
    Lbar_pin = lbar_pool(n_max)
    rho_pin = torch.empty((n_max, 512), dtype=torch.float64).pin_memory()
    L_out = torch.empty((n_max, 20, 512), dtype=torch.float64).pin_memory()
    rb_out = torch.empty((n_max, 512), dtype=torch.float64).pin_memory()

    clocks = ClockSampler(torch.cuda.current_device())
    tile, tuned = None, None
    step_ms, e2e_ms, pairs, launches, setup_s = [], [], 0, 0, 0.0
    h2d, d2h = 0, 0
    keep = None
    clocks.start()
    for k in range(args.steps):
        tree, rho_h = inputs[k]
        n = tree.n
        t0 = time.perf_counter()
        g = ot.OTGrid.from_tree(tree)
        work = g.step_buffers()
        rho_pin[:n].copy_(torch.from_numpy(rho_h))
        work["rho"].copy_(rho_pin[:n])
        work["Lbar"].copy_(Lbar_pin[:n])
        if args.tile:
            tile = tuple(int(x) for x in args.tile.lower().split("x"))
        if tile is None and sched == ot.OT_SCHED_PERSISTENT and not args.no_autotune:
            g.moments(work["rho"], work["M"], work["m"])
            tuned = g.autotune(work["M"], work["m"], work["L"], work["Lc"])
            tile = (tuned["warps_per_block"], tuned["blocks_per_sm"])
        g.set_schedule(sched, *(tile or (4, 0)), not args.no_graph)

        def device_step():
            g.moments(work["rho"], work["M"], work["m"])
            g.interactions(work["M"], work["m"], work["L"], work["Lc"])
            g.backward(work["Lbar"], work["Mb"], work["mb"])
            g.moments_backward(work["Mb"], work["mb"], work["rb"])

        device_step()                                  # records this grid's graphs (untimed)
        if k == 0:
            for _ in range(args.warmup):               # warm-up steps on step 0's tree
                device_step()
        torch.cuda.synchronize()
        g.check()
        setup_s += time.perf_counter() - t0

        # -- timed: the step on device-resident inputs ------------------------
        barrier(world)
        torch.cuda.synchronize()
        c0 = ot.launch_count()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        device_step()
        b.record(stream)
        launches += ot.launch_count() - c0
        torch.cuda.synchronize()
        barrier(world)
        step_ms.append(a.elapsed_time(b))
        # -- end to end: host buffers in, results out, copies inside ----------
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(stream)
        g.step_host(rho_pin[:n], Lbar_pin[:n], L_out[:n], rb_out[:n], work)
        b2.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(a2.elapsed_time(b2))
        g.check()
        info = g.info()
        pairs += 2 * (info["pairs_multipole"] + info["pairs_monopole"])
        h2d += (rho_pin[:n].numel() + Lbar_pin[:n].numel()) * 8
        d2h += (L_out[:n].numel() + rb_out[:n].numel()) * 8
        if k == 0:
            keep = (tree, rho_h, g, work, info)
        else:
            del work
            g.close()
    clk = clocks.stop()
    value, ms_per_step = aggregate(world, pairs, sum(step_ms) / 1e3, args.steps)
    e2e_value, _ = aggregate(world, pairs, sum(e2e_ms) / 1e3, args.steps)
    tree0, rho0, g0, work0, info0 = keep
    subgrids = [t.n for t, _ in inputs]
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (analytic binary-star densities sampled at cell centres, seeded L-bar)",
        "config": {"workload": WORKLOADS["binary"], "steps_are": "rotation steps 0..K-1, each its own octree",
                   "subgrids": {"min": min(subgrids), "max": max(subgrids), "mean": statistics.mean(subgrids)},
                   "leaf_cells_step0": int(tree0.is_leaf.sum()) * 512,
                   "pairs_per_step": pairs / args.steps, "schedule": args.schedule, "graph": not args.no_graph,
                   "tile": {"warps_per_block": tile[0], "blocks_per_sm": tile[1]} if tile else None,
                   "autotuned": tuned,
                   "l2": "not flushed: every step's inputs and outputs (M alone > 700 MB) exceed the 126 MB L2",
                   "host_setup_untimed_s": {"inputs_all_steps": inputs_s, "grid_and_graphs_per_step":
                                            setup_s / args.steps},
                   "warmup_steps_on": "step 0's tree",
                   "parallelism": f"replicas x{world}"},
        "step_ms": step_ms,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d / args.steps),
                "d2h_bytes_per_step": int(d2h / args.steps), "ms": sum(e2e_ms) / args.steps,
                "note": ("OTGrid.step_host per step: densities and L-bar from pinned host memory in, L and the "
                         "density adjoint out; the L-bar upload overlaps the forward and the L download the "
                         "adjoint on a side stream")},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if args.no_extras:
        return res, tree0, rho0

    # -- beside the headline, on step 0's grid ------------------------------
    W = work0
    fwd_ms = time_call(lambda: g0.interactions(W["M"], W["m"], W["L"], W["Lc"]), stream)
    adj_ms = time_call(lambda: g0.backward(W["Lbar"], W["Mb"], W["mb"]), stream)
    launches0 = launch_breakdown(g0, W, stream)
    pairs_fwd0 = info0["pairs_multipole"] + info0["pairs_monopole"]
    res["fwd"] = {"value": pairs_fwd0 / (fwd_ms * 1e-3), "unit": UNIT, "ms": fwd_ms, "pairs_in_domain": pairs_fwd0,
                  "pairs_padded": info0["pairs_padded_fwd"], "step": 0}
    res["adjoint"] = {"value": pairs_fwd0 / (adj_ms * 1e-3), "unit": UNIT, "ms": adj_ms, "step": 0}
    res["variants"] = {
        "multipole": {"pairs": info0["pairs_multipole"], "pairs_with_angular_term": info0["pairs_angular"],
                      "ms": launches0["multipole"]["ms"]},
        "monopole": {"pairs": info0["pairs_monopole"], "ms": launches0["monopole"]["ms"]},
        "boundary": {"pairs": info0["pairs_virtual"] + info0["pairs_refined"],
                     "pairs_virtual_source": info0["pairs_virtual"], "pairs_refined_target": info0["pairs_refined"],
                     "note": "coarse-fine pairs; they run inside the point-mass launch"}}
    # the same forward as one launch per sub-grid (the paper's many small kernels)
    g0.set_schedule(ot.OT_SCHED_PER_SUBGRID, *(tile or (4, 0)), False)
    plain_ms = time_call(lambda: g0.interactions(W["M"], W["m"], W["L"], W["Lc"]), stream, reps=1, warm=False)
    g0.set_schedule(sched, *(tile or (4, 0)), not args.no_graph)
    res["batched_vs_plain"] = {"batched_fwd_ms": fwd_ms, "plain_fwd_ms": plain_ms, "speedup": plain_ms / fwd_ms,
                               "plain_launches": tree0.n,
                               "note": ("the forward of step 0's tree: one persistent launch per pass in a CUDA "
                                        "graph against one launch per target sub-grid of the same kernels, "
                                        "same GPU, same stream")}
    peak_inst, probe_cfg = fp64_peak(ot, dev, stream)
    res["roofline"] = roofline_block(launches0, peak_inst, probe_cfg, clk.get("sm_mhz"), "binary", info0,
                                     pairs_fwd0, fwd_ms, adj_ms)
    res["fp64_peak"] = {"value": peak_inst / 1e12, "unit": "Tinst/s", "probe": probe_cfg,
                        "per_sm_per_clock": peak_inst / (torch.cuda.get_device_properties(dev).multi_processor_count
                                                         * (clk.get("sm_mhz") or NOMINAL_SM_MHZ) * 1e6)}
    del W, work0
    g0.close()
    res["polytrope64"] = run_polytrope64_brief(ot, dev, stream, args, peak_inst, probe_cfg, clk)
    return res, tree0, rho0


def run_polytrope64_brief(ot, dev, stream, args, peak_inst, probe_cfg, clk):
    """The uniform 64^3 workload beside the headline: device-resident steps
    with L2 flushed between them, the launch breakdown and its roofline."""
    import torch
    tree, rho_h = make_workload("polytrope64")
    g = ot.OTGrid.from_tree(tree)
    W = g.step_buffers()
    W["rho"].copy_(torch.from_numpy(rho_h))
    W["Lbar"].copy_(lbar_pool(tree.n, seed=5))
    g.moments(W["rho"], W["M"], W["m"])
    tuned = g.autotune(W["M"], W["m"], W["L"], W["Lc"])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def device_step():
        g.moments(W["rho"], W["M"], W["m"])
        g.interactions(W["M"], W["m"], W["L"], W["Lc"])
        g.backward(W["Lbar"], W["Mb"], W["mb"])
        g.moments_backward(W["Mb"], W["mb"], W["rb"])

    ms = time_call(device_step, stream, reps=max(args.steps, 5), flush=flush)
    info = g.info()
    pairs_fwd = info["pairs_multipole"] + info["pairs_monopole"]
    fwd_ms = time_call(lambda: g.interactions(W["M"], W["m"], W["L"], W["Lc"]), stream, flush=flush)
    adj_ms = time_call(lambda: g.backward(W["Lbar"], W["Mb"], W["mb"]), stream, flush=flush)
    launches = launch_breakdown(g, W, stream, flush=flush)
    g.set_schedule(ot.OT_SCHED_PER_SUBGRID, tuned["warps_per_block"], tuned["blocks_per_sm"], False)
    plain_ms = time_call(lambda: g.interactions(W["M"], W["m"], W["L"], W["Lc"]), stream, reps=3, flush=flush)
    out = {"workload": WORKLOADS["polytrope64"], "subgrids": tree.n, "value": 2 * pairs_fwd / (ms * 1e-3),
           "unit": UNIT, "ms_per_step": ms, "pairs_fwd": pairs_fwd, "fwd_ms": fwd_ms, "adj_ms": adj_ms,
           "tile": [tuned["warps_per_block"], tuned["blocks_per_sm"]],
           "l2": "flushed between steps (256 MB write outside the events)",
           "batched_vs_plain": {"batched_fwd_ms": fwd_ms, "plain_fwd_ms": plain_ms, "speedup": plain_ms / fwd_ms},
           "roofline": roofline_block(launches, peak_inst, probe_cfg, clk.get("sm_mhz"), "polytrope64", info,
                                      pairs_fwd, fwd_ms, adj_ms)}
    del W
    g.close()
    return out


# ---------------------------------------------------------------------------
# the other workloads
# ---------------------------------------------------------------------------

def run_fixed(args, rank, world):
    """One fixed tree (the 64^3 level or the adaptive octree), K steps with
    L2 flushed between them, plus the variants measured on it."""
    import torch
    import paper_2303_08058_b300 as ot

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    tree, rho_h = make_workload(args.workload)
    g = ot.OTGrid.from_tree(tree)
    sched = ot.OT_SCHED_PER_SUBGRID if args.schedule == "per_subgrid" else ot.OT_SCHED_PERSISTENT
    g.set_schedule(sched, 4, 0, not args.no_graph)
    W = g.step_buffers()
    W["rho"].copy_(torch.from_numpy(rho_h))
    Lbar_pin = lbar_pool(tree.n)
    W["Lbar"].copy_(Lbar_pin)
    g.moments(W["rho"], W["M"], W["m"])
    tuned = None
    if args.tile:
        w, b = (int(x) for x in args.tile.lower().split("x"))
        g.set_schedule(sched, w, b, not args.no_graph)
    elif not args.no_autotune and sched == ot.OT_SCHED_PERSISTENT:
        tuned = g.autotune(W["M"], W["m"], W["L"], W["Lc"])
    info = g.info()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        g.moments(W["rho"], W["M"], W["m"])
        g.interactions(W["M"], W["m"], W["L"], W["Lc"])
        g.backward(W["Lbar"], W["Mb"], W["mb"])
        g.moments_backward(W["Mb"], W["mb"], W["rb"])

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    g.check()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    c0 = ot.launch_count()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    launches = ot.launch_count() - c0
    torch.cuda.synchronize()
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    g.check()
    clk = clocks.stop()
    pairs_fwd = info["pairs_multipole"] + info["pairs_monopole"]
    value, ms_per_step = aggregate(world, 2 * pairs_fwd * args.steps, sum(step_ms) / 1e3, args.steps)

    res = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded polytrope densities, seeded L-bar)",
           "config": {"workload": WORKLOADS[args.workload], "subgrids": tree.n, "cells": tree.n * 512,
                      "pairs_fwd": pairs_fwd, "pairs_adj": pairs_fwd, "schedule": args.schedule,
                      "graph": not args.no_graph,
                      "tile": {"warps_per_block": info["warps_per_block"], "blocks_per_sm": info["blocks_per_sm"]},
                      "autotuned": tuned, "l2": "flushed between steps (256 MB write outside the events)",
                      "parallelism": f"replicas x{world}"},
           "gpu_launches": launches, "clocks": clk}
    if args.no_extras:
        return res, tree, rho_h
    fwd_ms = time_call(lambda: g.interactions(W["M"], W["m"], W["L"], W["Lc"]), stream, flush=flush)
    adj_ms = time_call(lambda: g.backward(W["Lbar"], W["Mb"], W["mb"]), stream, flush=flush)
    launches0 = launch_breakdown(g, W, stream, flush=flush)
    res["fwd"] = {"value": pairs_fwd / (fwd_ms * 1e-3), "unit": UNIT, "ms": fwd_ms}
    res["adjoint"] = {"value": pairs_fwd / (adj_ms * 1e-3), "unit": UNIT, "ms": adj_ms}
    # double-float contractions (NEXT-4), beside the FP64 numbers
    dfl = {}
    for name, mode in (("fwd_df64_point_mass", ot.OT_PREC_DF64_POINT_MASS), ("fwd_df64", ot.OT_PREC_DF64)):
        g.set_precision(mode)
        dfl[name] = time_call(lambda: g.interactions(W["M"], W["m"], W["L"], W["Lc"]), stream, flush=flush)
    dfa = time_call(lambda: g.backward(W["Lbar"], W["Mb"], W["mb"]), stream, flush=flush)
    g.set_precision(ot.OT_PREC_FP64)
    res["df64"] = {"fwd_point_mass_ms": dfl["fwd_df64_point_mass"], "fwd_ms": dfl["fwd_df64"], "adjoint_ms": dfa,
                   "fwd_plus_adjoint": 2 * pairs_fwd / ((dfl["fwd_df64"] + dfa) * 1e-3),
                   "note": ("contractions in double-float on the FP32 pipe (OT_PREC_DF64; the point-mass variant "
                            "OT_PREC_DF64_POINT_MASS), within 1e-12 of the oracle's scale; beside the FP64 "
                            "numbers, not as them")}
    # centre-of-mass expansion centres (NEXT-2)
    Mc, mc, Cc = g.moments_com(W["rho"])
    com_f = time_call(lambda: g.interactions_com(Mc, mc, Cc, W["L"], W["Lc"]), stream, flush=flush)
    com_a = time_call(lambda: g.backward_com(W["Lbar"], Cc, W["Mb"], W["mb"]), stream, flush=flush)
    res["com"] = {"fwd_ms": com_f, "adjoint_ms": com_a, "fwd_flops": info["flops_fwd_com"],
                  "adj_flops": info["flops_adj_com"],
                  "fwd_tflops": info["flops_fwd_com"] / (com_f * 1e-3) / 1e12,
                  "adj_tflops": info["flops_adj_com"] / (com_a * 1e-3) / 1e12}
    del Mc, mc, Cc
    peak_inst, probe_cfg = fp64_peak(ot, dev, stream)
    res["roofline"] = roofline_block(launches0, peak_inst, probe_cfg, clk.get("sm_mhz"), args.workload, info,
                                     pairs_fwd, fwd_ms, adj_ms)
    # end to end through OTGrid.step_host
    L_out = torch.empty((tree.n, 20, 512), dtype=torch.float64).pin_memory()
    rb_out = torch.empty((tree.n, 512), dtype=torch.float64).pin_memory()
    rho_pin = torch.from_numpy(rho_h).pin_memory()
    e2e_ms = time_call(lambda: g.step_host(rho_pin, Lbar_pin, L_out, rb_out, W), stream, flush=flush)
    res["e2e"] = {"value": world * 2 * pairs_fwd / (e2e_ms * 1e-3), "unit": UNIT,
                  "h2d_bytes_per_step": int((rho_pin.numel() + Lbar_pin.numel()) * 8),
                  "d2h_bytes_per_step": int((L_out.numel() + rb_out.numel()) * 8), "ms": e2e_ms}
    return res, tree, rho_h


def run_integration(args, rank, world):
    """The completion-notification study on the 64^3 and adaptive workloads:
    per-sub-grid forward launches over 1-32 streams with completions seen by
    stream sync, host callbacks, event polling from the launching thread or
    from a host thread pool, against one batched persistent launch (median
    of --steps repetitions)."""
    import torch
    import paper_2303_08058_b300 as ot
    names = {0: "stream_sync", 1: "host_callback", 2: "event_polling", 3: "batched_persistent",
             4: "event_polling_pool"}
    out = {}
    for wl in ("polytrope64", "adaptive"):
        tree, rho_h = make_workload(wl)
        g = ot.OTGrid.from_tree(tree)
        g.set_schedule(ot.OT_SCHED_PERSISTENT, 4, 2, False)
        M, m = g.moments(torch.as_tensor(rho_h, device="cuda"))
        rows = []
        for mech in (0, 1, 2, 4, 3):
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


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

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
        r1 = oracle.run_pass(tree, "multipole", M=M, targets=tg, with_sd=False)
        r2 = oracle.run_pass(tree, "monopole", m=m, targets=tg, with_sd=False)
        t_used += time.perf_counter() - t0
        pairs += r1["npairs"] + r2["npairs"]
        ntg += len(tg)
    # the same oracle on one thread, a shorter sample
    oracle.set_threads(1)
    pairs1, t1 = 0, 0.0
    while t1 < max(2.0, seconds / 6):
        tg = np.stack([rng.integers(0, tree.n, 64), rng.integers(0, 512, 64)], 1).astype(np.int32)
        t0 = time.perf_counter()
        r1 = oracle.run_pass(tree, "multipole", M=M, targets=tg, with_sd=False)
        r2 = oracle.run_pass(tree, "monopole", m=m, targets=tg, with_sd=False)
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
            "sample": f"forward of both passes for {ntg} random target cells of the workload's first tree "
                      f"({pairs} pairs, {t_used:.1f} s)",
            "single_thread": {"value": pairs1 / t1, "unit": UNIT, "sample": f"{pairs1} pairs, {t1:.1f} s"},
            "cpu": cpu}


def run_reference(args, rank, world):
    """The oracle on the host cores, each step a bounded sample of the same
    workload's first tree: forward of both passes and the transposed sums for
    random target cells."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    wl = args.workload if args.workload in WORKLOADS else "binary"
    tree, rho_h = make_workload(wl)
    Lbar_h = np.random.default_rng(4).standard_normal((tree.n, 20, 512))
    M = oracle.moments(tree, rho_h)
    m = np.ascontiguousarray(M[:, 0, :])
    rng = np.random.default_rng(8)
    per = 32 * cores
    per_adj = max(8, per // cores)   # the transposed sums scatter, so they run on one core

    def step():
        tg = np.stack([rng.integers(0, tree.n, per), rng.integers(0, 512, per)], 1).astype(np.int32)
        r1 = oracle.run_pass(tree, "multipole", M=M, targets=tg, with_sd=False)
        r2 = oracle.run_pass(tree, "monopole", m=m, targets=tg, with_sd=False)
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
            "config": {"workload": WORKLOADS[wl], "subgrids": tree.n, "cells": tree.n * 512,
                       "parallelism": "host cores (OpenMP)"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"per step: forward of both passes for {per} random target cells of the "
                                       f"workload's first tree (OpenMP) and the transposed sums of both passes "
                                       f"for {per_adj} of them (serial scatter)"},
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
    if args.workload == "binary":
        res, tree, rho_h = run_binary(args, rank, world)
    elif args.workload == "integration":
        res, tree, rho_h = run_integration(args, rank, world)
    else:
        res, tree, rho_h = run_fixed(args, rank, world)
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
