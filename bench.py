#!/usr/bin/env python
"""Benchmark of the coupled cell/fluid time step on one GB300 (per rank).

Workload: single cell in linear shear at production size - 128^3 D3Q19
lattice (tau = 1, walls at -/+0.05), one R = 16 sphere of ~4.2k vertices and
~20k tets, Mooney-Rivlin mu from Ca = 0.2, kappa = 50 mu, w = 0.5, FP32.
One benchmark step is one full coupled time step (tet forces, vertex sums +
spread, stream-collide, interpolate + advect). Populations (2 x 159 MB) are
larger than the 129 MB L2, so no flush is needed between steps.

Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU
oracle on the same workload instead (bounded samples per step).

Multi-GPU (``torchrun --nproc-per-node N``): N independent replicas of the
workload, one per GPU, no data exchange (weak scaling); the timed region is
bracketed by barriers and the slowest rank's time is used.
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
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled LBM-IBM steps/s & MLUPS (% HBM roofline); tet-forces/s; FP16 vs FP32 error"
POP_BYTES_PER_NODE = 2 * 19 * 4  # read + write of 19 FP32 populations
NEAR_BYTES_PER_NODE = POP_BYTES_PER_NODE + 16 + 16  # + force read, velocity written (float4 per node)
MULTICELL_R = 16.0  # cell radius of the multicell workload (its d_ref = 2R for the cell strain)
CONSUME_BYTES_PER_SUPPORT_NODE = 16  # the near field zeroes the force it read on the spread's support
# cell kernels (FP32): per tet, K1 reads the int4 indices (16) and the packed B rows (48) and writes
# four float4 corner forces (64); K23 reads four incidence entries (16) and the corner forces (64).
# Per vertex, K1 reads xr and u (32); K23 reads the row bounds (8), xr and u (32), writes the vertex
# force (16) and adds one float4 per support node into F (16 W^3).
CELL_BYTES_PER_TET = 16 + 48 + 64 + 16 + 64
CELL_BYTES_PER_VERTEX = 32 + 8 + 32 + 16


# interpolation + advection: per vertex xr and u read (32), u written (16), and the velocity (float4)
# of each support node read (16 W^3)
INTERP_BYTES_PER_VERTEX = 32 + 16


def cell_bytes(n_tets, n_verts, width):
    """Algorithmic bytes of the tet forces + vertex sums + spread of one step."""
    return CELL_BYTES_PER_TET * n_tets + (CELL_BYTES_PER_VERTEX + 16 * width**3) * n_verts


def step_roofline(wl, roof, pop_format, ms_per_step, peak):
    """The whole step against the HBM peak: the algorithmic bytes of every
    kernel of one step (far and near stream-collide, tet forces, vertex sums
    + spread, interpolation + advection) over the measured time per step."""
    pop_b = POP_BYTES_PER_NODE // (1 if pop_format == "f32" else 2)
    near_nodes, n_sup = roof["near_region_nodes"], roof["support_nodes"]
    parts = {
        "far": pop_b * (wl.n_nodes - near_nodes),
        "near": (pop_b + NEAR_BYTES_PER_NODE - POP_BYTES_PER_NODE) * near_nodes
        + CONSUME_BYTES_PER_SUPPORT_NODE * n_sup,
        "cells": cell_bytes(wl.n_tets, wl.n_verts, wl.delta) if wl.n_tets else 0,
        "interp": (INTERP_BYTES_PER_VERTEX + 16 * wl.delta**3) * wl.n_verts,
    }
    total = sum(parts.values())
    achieved = total / (ms_per_step / 1e3) / 1e9
    return {"bound": "hbm", "algorithmic_bytes_per_step": total, "parts": parts, "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak}


def cell_roofline(wl, kms, peak):
    """Tet forces + vertex sums + spread by their CUDA-event times (kernel
    slots 0 and 1): tets/s and the fraction of the HBM peak their algorithmic
    bytes reach."""
    s = (kms[0] + kms[1]) / 1e3
    b = cell_bytes(wl.n_tets, wl.n_verts, wl.delta)
    return {"kernels": "k_tet_force + k_gather_spread", "tets_per_s": wl.n_tets / s, "bound": "hbm",
            "algorithmic_bytes_per_step": b, "achieved": b / s / 1e9, "peak": peak, "unit": "GB/s",
            "frac": b / s / 1e9 / peak,
            "bytes_model": f"{CELL_BYTES_PER_TET} B/tet + ({CELL_BYTES_PER_VERTEX} + 16 W^3) B/vertex"}
KERNELS = ("k_tet_force", "k_gather_spread", "k_lbm_far", "k_lbm_near", "k_interp_advect")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=128, help="cubic lattice extent")
    ap.add_argument("--workload", choices=("shear", "paperbox", "multicell", "suspension", "compression"),
                    default="shear",
                    help="shear: one R = 16 cell in a 128^3 Couette box; paperbox: the same cell in the "
                         "paper's 10 x 15 x 5 R box (160 x 240 x 80); multicell: 4 or 8 R = 16 cells "
                         "(--phi 0.11 / 0.22) in the paper's 5 x 8 x 4 R sheared box; suspension: 400 cells in a "
                         "512 x 256 x 256 channel; compression: fit the moduli of 64 cells to synthetic "
                         "force-strain curves with the adjoint")
    ap.add_argument("--fit-iters", type=int, default=10, help="Adam iterations of the compression fit")
    ap.add_argument("--cells", type=int, default=400, help="cells of the suspension workload")
    ap.add_argument("--phi", type=float, choices=(0.11, 0.22), default=0.22,
                    help="volume fraction of the multicell workload (4 or 8 cells)")
    ap.add_argument("--box", default="512,256,256", help="lattice of the suspension workload")
    ap.add_argument("--delta", choices=("trilinear", "peskin4"), default="trilinear",
                    help="immersed-boundary delta kernel")
    ap.add_argument("--spread", choices=("float", "fixed"), default="float",
                    help="force-field accumulation: float atomics, or the deterministic fixed-point field")
    ap.add_argument("--fused", type=int, default=-1, choices=(-1, 0, 1),
                    help="cell chain as one persistent launch (1) or two (0); -1: default / autotuner")
    ap.add_argument("--pop-format", choices=("f32", "f16", "bf16", "f16sr", "bf16sr"), default="f32",
                    help="population storage (the collide is FP32 in every format)")
    ap.add_argument("--tile", default="", help="force-region tile x,y,z (e.g. 32,2,4); default: autotuner's")
    ap.add_argument("--shape", default="", help="launch-shape knobs set after the autotuner, e.g. far_blocks=4")
    ap.add_argument("--autotune-steps", type=int, default=40,
                    help="steps per launch-shape candidate of the autotuner in the warm-up (0: default shape)")
    ap.add_argument("--ca", type=float, default=0.2)
    ap.add_argument("--w", type=float, default=0.5)
    ap.add_argument("--profile-steps", type=int, default=2000)
    ap.add_argument("--e2e-steps", type=int, default=2000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample length for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision-steps", type=int, default=12500,
                    help="steps of the storage-format comparison on the channel workload (0 = skip)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of K steps each; value = K / median region time")
    ap.add_argument("--suspension-steps", type=int, default=300,
                    help="with the default shear workload: also time the 400-cell suspension "
                         "(512 x 256 x 256) for this many steps per region (0 = skip)")
    ap.add_argument("--compression-iters", type=int, default=1,
                    help="with the default shear workload: also time the 64-cell compression (forward "
                         "relaxation rate) and this many adjoint gradients of its fit (0 = skip)")
    ap.add_argument("--sweep", action="store_true",
                    help="shear workload: run the 9 (Ca, w) cases of the production shear for "
                         "--sweep-steps steps each and print the Taylor deformation, inclination and "
                         "cell strain every 100 steps")
    ap.add_argument("--paper-sweep-steps", type=int, default=0,
                    help="also run the paper's single-cell shear setup (160 x 240 x 80 box, R = 16, neo-Hookean "
                         "w = 1) at Ca in {0.05, 0.1, 0.2, 0.3, 0.5} for this many steps each (0 = skip)")
    ap.add_argument("--sweep-steps", type=int, default=10000,
                    help="steps per (Ca, w) case of the production-shear sweep (0 = skip it in the "
                         "default run, which reports every 1,000th step)")
    return ap.parse_args()


def workload(args):
    from workloads import configs

    if args.workload == "suspension":
        nx, ny, nz = (int(v) for v in args.box.split(","))
        wl = configs.batched_channel(ncells=args.cells, nx=nx, ny=ny, nz=nz)
    elif args.workload == "paperbox":
        wl = configs.paper_box_shear(ca=args.ca, w=args.w)
    elif args.workload == "multicell":
        wl = configs.multicell_shear(ncells=4 if args.phi == 0.11 else 8, R=MULTICELL_R, ca=args.ca, w=args.w)
    else:
        wl = configs.production_shear(ca=args.ca, w=args.w, n=args.n)
    wl.delta = {"trilinear": 2, "peskin4": 4}[args.delta]
    return wl


def config_of(wl):
    return {
        "workload": wl.name,
        "lattice": [wl.nx, wl.ny, wl.nz],
        "n_verts": wl.n_verts,
        "n_tets": wl.n_tets,
        "tau": wl.tau,
        "u_wall": [wl.u_wall_lo, wl.u_wall_hi],
        "delta": {2: "trilinear", 4: "peskin4"}[wl.delta],
        "parallelism": "replicas",
        "l2": "no flush: populations 2 x %.0f MB > 129 MB L2" % (19 * 4 * wl.n_nodes / 1e6),
    }


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The slowest rank's time: all-reduce MAX (identity on one rank)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of independent replicas: all ranks' units over
    the slowest rank's time."""
    return world * units_per_rank / seconds


def support_nodes(y, dims, width=2):
    """Number of distinct lattice nodes in the delta support (width 2:
    trilinear, 4: four-point) of y."""
    nx, ny, nz = dims
    b = np.floor(y).astype(np.int64) - (width // 2 - 1)
    keys = []
    r = range(width)
    for dz in r:
        for dy in r:
            for dx in r:
                X = (b[:, 0] + dx) % nx
                Y = b[:, 1] + dy
                Z = (b[:, 2] + dz) % nz
                keys.append(X + nx * (Y + ny * Z))
    return int(np.unique(np.concatenate(keys)).size)


def traffic_record(kernel, tag):
    """DRAM bytes per launch from a committed ncu summary of the workload
    `tag`, if it was taken on the current source of the stream-collide
    kernels (else None). profiles/<kernel>_<tag>.md holds one kernel;
    profiles/<tag>.md may hold several ("<kernel> dram_bytes_per_launch:")."""
    src = os.path.join(ROOT, "paper_2003_03130_gb300", "csrc", "lbm.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for path, pat in ((os.path.join(ROOT, "profiles", f"{kernel}_{tag}.md"), r"^dram_bytes_per_launch:"),
                      (os.path.join(ROOT, "profiles", f"{tag}.md"), rf"^{kernel} dram_bytes_per_launch:")):
        if not os.path.exists(path):
            continue
        text = open(path).read()
        m_sha = re.search(r"^source_sha256_16(?: lbm\.cu)?:\s*([0-9a-f]+)", text, re.M)
        m_b = re.search(pat + r"\s*([0-9.eE+]+)", text, re.M)
        if m_sha and m_b and m_sha.group(1) == sha:
            return float(m_b.group(1))
    return None


def _oracle_sample(job):
    """One oracle replica: whole coupled steps of workload `wl` until
    `seconds` of CPU work have passed (at most 200). Returns (steps, s)."""
    wl, seconds = job
    import oracle

    sim = oracle.Coupled(wl)
    sim.step(1)  # first touch
    t0 = time.perf_counter()
    n = 0
    while True:
        sim.step(1)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or n >= 200:
            return n, dt


def _host_replicas(n_nodes):
    """Oracle replicas that fit the host: one per usable core, at most as many
    as half the available memory holds (about 500 B per lattice node each)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    avail = None
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    if avail is None:
        return 1
    return max(1, min(cores, int(avail // 2 // (500 * n_nodes))))


def cpu_baseline(wl, seconds):
    """Oracle (FP64, as it stands) on the same workload: whole coupled steps
    until `seconds` of CPU work have passed, on one thread; then P independent
    replicas at once, one per host core (processes started with spawn), whose
    summed rate is the host's throughput."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    n, dt = _oracle_sample((wl, seconds))
    out = {"value": n / dt, "unit": "steps/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} whole coupled steps of the same {wl.nx}x{wl.ny}x{wl.nz} workload, FP64, 1 thread",
           "mlups": n * wl.n_nodes / dt / 1e6}
    procs = _host_replicas(wl.n_nodes)
    if procs > 1:
        # a worker that dies raises here instead of hanging the pool; the
        # wait is bounded as well
        from concurrent.futures import ProcessPoolExecutor

        try:
            with ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
                futs = [ex.submit(_oracle_sample, (wl, seconds)) for _ in range(procs)]
                res = [f.result(timeout=4 * seconds + 120) for f in futs]
        except Exception as e:  # reported, not fatal: the one-thread figure stands
            out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
            return out
        out["all_cores"] = {
            "value": sum(k / t for k, t in res), "unit": "steps/s", "cores": procs,
            "sample": f"{procs} independent replicas (one process each), {min(k for k, _ in res)}-"
                      f"{max(k for k, _ in res)} whole steps each, summed rates"}
    return out


def suspension_cpu_baseline():
    """The oracle (FP64, as it stands, one thread) on the 400-cell suspension:
    one untimed step, then whole steps for at least a second (one step takes
    ~18 s there)."""
    import oracle
    from workloads import configs

    oracle.build()
    n, dt = _oracle_sample((configs.batched_channel(), 1.0))
    return {"value": n / dt, "unit": "steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} whole coupled step(s) of the 400-cell suspension (512x256x256, 6.0 M tets) after one "
                      "untimed step, FP64, 1 thread"}


def precision_block(P, torch, dev, steps):
    """FP32, FP16 and BF16 population storage (round to nearest, and
    stochastic rounding: f16sr, bf16sr) on the pressure-driven channel
    (256 x 128 x 128, one R = 16 cell): steps/s of each, and the error of the
    16-bit runs against the FP32 run after the same steps from t = 0
    (norm-wise relative on the fluid velocity and the cell displacement;
    relative on the Taylor deformation D)."""
    from workloads import configs

    wl = configs.precision_channel(steps=steps)
    res = {}
    stream = torch.cuda.Stream(dev)
    for fmt in ("f32", "f16", "bf16", "f16sr", "bf16sr"):
        with torch.cuda.stream(stream):
            ctx = P.cf_create(dev, stream.cuda_stream)
            P.cf_set_population_format(ctx, fmt)
            (cid,) = P.load_workload(ctx, wl)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.cf_step_async(ctx, steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            P.cf_synchronize(ctx)
            ms = e0.elapsed_time(e1)
            y = P.cf_get_positions(ctx, cid)
            u = P.cf_get_velocity(ctx)
            D = P.cf_get_taylor(ctx, cid)["D"]
            P.cf_destroy(ctx)
        res[fmt] = {"steps_per_s": steps / (ms / 1e3), "mlups": wl.n_nodes * steps / (ms / 1e3) / 1e6,
                    "y": y, "u": u, "D": D}
    x0 = wl.cells[0].x_ref
    ref = res["f32"]
    out = {"workload": wl.name, "steps": steps, "D_f32": ref["D"]}
    for fmt in ("f32", "f16", "bf16", "f16sr", "bf16sr"):
        r = res[fmt]
        out[fmt] = {"steps_per_s": r["steps_per_s"], "mlups": r["mlups"], "D": r["D"]}
        if fmt != "f32":
            out[fmt]["rel_err_velocity_vs_f32"] = float(np.linalg.norm(r["u"] - ref["u"]) / np.linalg.norm(ref["u"]))
            out[fmt]["rel_err_displacement_vs_f32"] = float(
                np.linalg.norm(r["y"] - ref["y"]) / np.linalg.norm(ref["y"] - x0))
            out[fmt]["rel_err_D_vs_f32"] = float(abs(r["D"] - ref["D"]) / abs(ref["D"]))
    return out


def timed_regions(P, torch, ctx, stream, dev, K, repeats, world, barrier):
    """`repeats` timed regions of exactly K coupled steps, each bracketed by a
    barrier and a device synchronisation, timed with CUDA events on the
    launching stream; per region the slowest rank's time (ms)."""
    out = []
    for _ in range(max(1, repeats)):
        barrier()
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        P.cf_step_async(ctx, K)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        P.cf_synchronize(ctx)
        ms = ev0.elapsed_time(ev1)
        barrier()
        out.append(max_over_ranks(ms, world, device=f"cuda:{dev}"))
    return out


def region_stats(ms, K):
    return {"n": len(ms), "steps_per_region": K, "ms_per_step_median": statistics.median(ms) / K,
            "ms_per_step_min": min(ms) / K, "ms_per_step_max": max(ms) / K}


def stream_collide_roofline(wl, kms, near_nodes, y_now, pop_format, peak):
    """The stream-collide part with the longer mean launch time (far field:
    every node outside the force region, populations only; near field: the
    region's nodes with the force read and u(t) written, plus the zeroing of
    the consumed force on the spread's support): its algorithmic bytes over
    its CUDA-event launch time."""
    far_nodes = wl.n_nodes - near_nodes
    pop_b = POP_BYTES_PER_NODE // (1 if pop_format == "f32" else 2)  # 2-byte storage halves it
    n_sup = support_nodes(y_now, (wl.nx, wl.ny, wl.nz), wl.delta)
    if kms[2] >= kms[3]:
        dom, units, per_unit, dom_ms = "k_lbm_far", far_nodes, pop_b, kms[2]
        alg_bytes = per_unit * units
    else:
        near_b = pop_b + NEAR_BYTES_PER_NODE - POP_BYTES_PER_NODE
        dom, units, per_unit, dom_ms = "k_lbm_near", near_nodes, near_b, kms[3]
        alg_bytes = per_unit * units + CONSUME_BYTES_PER_SUPPORT_NODE * n_sup
    achieved = alg_bytes / (dom_ms / 1e3) / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "algorithmic_bytes_per_launch": alg_bytes, "units_per_launch": units,
            "bytes_per_unit": per_unit, "near_region_nodes": near_nodes, "support_nodes": n_sup}


def suspension_block(P, torch, dev, steps, peak):
    """The 400-cell suspension (512 x 256 x 256 channel, 1.26 M vertices,
    6.0 M tets, FP32): steps/s over three timed regions after the
    autotuner, MLUPS, tet forces/s, the stream-collide roofline and the cell
    kernels' roofline. GPU only (the oracle takes ~18 s per step here)."""
    from workloads import configs

    wl = configs.batched_channel()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        ctx = P.cf_create(dev, stream.cuda_stream)
        P.load_workload(ctx, wl)
        P.cf_step(ctx, 10)
        shape = P.cf_autotune(ctx, 20)
        P.cf_prepare_steps(ctx, steps)
        clocks = ClockSampler(dev)
        clocks.start()
        time.sleep(0.3)
        ms = timed_regions(P, torch, ctx, stream, dev, steps, 3, 1, lambda: None)
        clk = clocks.stop()
        kms, near_nodes = P.cf_step_profiled(ctx, 50)
        y_now = P.cf_get_positions(ctx, P.CF_ALL_CELLS)
        P.cf_destroy(ctx)
    med = statistics.median(ms) / 1e3
    roof = stream_collide_roofline(wl, kms, near_nodes, y_now, "f32", peak)
    return {"workload": wl.name, "lattice": [wl.nx, wl.ny, wl.nz], "n_cells": len(wl.cells),
            "n_verts": wl.n_verts, "n_tets": wl.n_tets, "steps_per_s": steps / med,
            "mlups": wl.n_nodes * steps / med / 1e6, "tet_forces_per_s": wl.n_tets * steps / med,
            "regions": region_stats(ms, steps), "launch_shape": shape,
            "kernel_ms": dict(zip(KERNELS, [float(x) for x in kms])),
            "roofline": roof, "cell_roofline": cell_roofline(wl, kms, peak),
            "step_roofline": step_roofline(wl, roof, "f32", med * 1e3 / steps, peak), "clocks": clk}


SWEEP_CA = (0.05, 0.2, 0.5)
SWEEP_W = (0.0, 0.5, 1.0)


PAPER_SWEEP_CA = (0.05, 0.1, 0.2, 0.3, 0.5)


def shear_sweep(P, torch, dev, steps, every, cases=None, make=None):
    """The production shear (128^3, R = 16, kappa = 50 mu) for every
    (Ca, w) in {0.05, 0.2, 0.5} x {0, 0.5, 1} (or the given cases and
    workload maker): `steps` coupled steps each, with the Taylor deformation
    D, its printed-expression variant, the inclination and the net cell
    strain (d_max - 2R) / 2R every `every` steps, and the steps/s of each
    run."""
    from workloads import configs

    out = []
    stream = torch.cuda.Stream(dev)
    cases = cases if cases is not None else [(ca, w) for ca in SWEEP_CA for w in SWEEP_W]
    make = make or (lambda ca, w: configs.production_shear(ca=ca, w=w))
    for ca, w in cases:
        wl = make(ca, w)
        with torch.cuda.stream(stream):
            ctx = P.cf_create(dev, stream.cuda_stream)
            (cid,) = P.load_workload(ctx, wl)
            P.cf_prepare_steps(ctx, every)
            rows, t_dev, done, error = [], 0.0, 0, None
            for k in range(0, steps, every):
                n = min(every, steps - k)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                P.cf_step_async(ctx, n)
                e1.record(stream)
                try:
                    P.cf_synchronize(ctx)
                except P.CellFSIError as e:  # e.g. a tet inverted: reported, the other cases still run
                    error = f"{e.name} within steps {k + 1}-{k + n}: {e}"
                    break
                t_dev += e0.elapsed_time(e1)
                done = k + n
                t = P.cf_get_taylor(ctx, cid)
                st = P.cf_get_cell_strain(ctx, cid, 2 * 16.0)
                rows.append([k + n, t["D"], t["D_literal"], t["inclination"], st["strain"]])
            P.cf_destroy(ctx)
        out.append({"ca": ca, "w": w, "mu": wl.cells[0].mu, "kappa": wl.cells[0].kappa,
                    "steps_done": done, "error": error,
                    "steps_per_s": done / (t_dev / 1e3) if t_dev > 0 else None,
                    "columns": ["step", "D", "D_literal", "inclination_deg", "cell_strain"], "rows": rows})
    return out


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch

    rank, world, local = dist_env()
    dev = local
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    import paper_2003_03130_gb300 as P
    from paper_2003_03130_gb300 import build as cbuild

    cbuild.build()
    wl = workload(args)
    stream = torch.cuda.Stream(dev)
    K, W = args.steps, args.warmup

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        ctx = P.cf_create(dev, stream.cuda_stream)
        P.cf_set_population_format(ctx, args.pop_format)
        P.cf_set_spread(ctx, args.spread)
        ids = P.load_workload(ctx, wl)
        if args.fused >= 0:
            P.cf_set_launch_shape(ctx, {"fused": args.fused})
        if args.tile:
            tx, ty, tz = (int(v) for v in args.tile.split(","))
            P.cf_set_launch_shape(ctx, {"tile_x": tx, "tile_y": ty, "tile_z": tz})
        P.cf_step(ctx, W)
        shape = P.cf_autotune(ctx, args.autotune_steps) if args.autotune_steps > 0 else P.cf_get_launch_shape(ctx)
        if args.shape:  # explicit knobs after the autotuner
            P.cf_set_launch_shape(ctx, {k: int(v) for k, v in (kv.split("=") for kv in args.shape.split(","))})
            shape = P.cf_get_launch_shape(ctx)
        P.cf_prepare_steps(ctx, K)  # graph instantiation stays out of the timed region
        clocks = ClockSampler(dev)
        clocks.start()
        time.sleep(0.3)
        region_ms = timed_regions(P, torch, ctx, stream, dev, K, args.repeats, world, barrier)
        clk = clocks.stop()
        ms = statistics.median(region_ms)

        # per-kernel durations: CUDA events around every launch, same stream
        kms, near_nodes = P.cf_step_profiled(ctx, args.profile_steps)

        # end to end through the public API with host buffers: per step the
        # positions go host -> device (pinned), one step, positions back, in
        # one call with one wait (two pinned buffers take turns)
        nv = P.cf_cell_verts(ctx, P.CF_ALL_CELLS)
        ybuf = [torch.empty((nv, 3), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
        P.cf_get_positions(ctx, P.CF_ALL_CELLS, out=ybuf[0])

        def e2e_step(k):
            P.cf_step_exchange(ctx, 1, ybuf[k & 1], out=ybuf[(k + 1) & 1])

        for k in range(6):  # warm-up: the one-step graphs of every parity and region phase
            e2e_step(k)
        barrier()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            e2e_step(k)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world, device=f"cuda:{dev}")
        barrier()
        y_now = P.cf_get_positions(ctx, P.CF_ALL_CELLS)
        mean_D = float(np.mean([P.cf_get_taylor(ctx, i)["D"] for i in ids])) if args.workload == "multicell" else None
        mean_strain = (float(np.mean([P.cf_get_cell_strain(ctx, i, 2 * MULTICELL_R)["strain"] for i in ids]))
                       if args.workload == "multicell" else None)
        P.cf_destroy(ctx)

    steps_per_s = job_rate(K, world, ms / 1e3)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("hbm_gbs", 6800.0))
    # dominant kernel: the stream-collide part that takes longer - the far
    # field in a single-cell box, the near field when the cells spread over
    # the whole lattice
    roof = stream_collide_roofline(wl, kms, near_nodes, y_now, args.pop_format, peak)
    dom = roof["kernel"]
    tag = (f"{wl.nx}cubed" if wl.nx == wl.ny == wl.nz else f"{wl.nx}x{wl.ny}x{wl.nz}") + (
        f"_{len(wl.cells)}cells" if args.workload == "suspension" else "")
    tag = ("suspension_" if args.workload == "suspension" else "") + tag
    # the ncu record of the same kernel form: the L2-normal form of the FP32 populations has its own
    traffic = (traffic_record(dom, tag + ("_l2" if shape.get("pop_l2") else ""))
               if wl.delta == 2 and args.pop_format == "f32" else None)
    step_ms_profiled = float(sum(kms))
    out = {
        "metric": METRIC,
        "value": steps_per_s,
        "unit": "steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32", "f16": "f16", "bf16": "bf16", "f16sr": "f16 (stochastic rounding)",
                  "bf16sr": "bf16 (stochastic rounding)"}[args.pop_format],
        "spread": args.spread,
        "data": "synthetic (seeded sphere mesh, fluid at rest at t=0)",
        "config": config_of(wl),
        "mlups": job_rate(wl.n_nodes * K, world, ms / 1e3) / 1e6,
        "tet_forces_per_s": job_rate(wl.n_tets * K, world, ms / 1e3),
        "gpu_launches": (4 if shape.get("fused") else 5) * K + 1,  # far, K5, K1 (+K23), near; mark + final K5
        "launch_shape": shape,
        "kernel_ms": dict(zip(KERNELS, [float(x) for x in kms])),
        "kernel_share": dict(zip(KERNELS, [float(x) / step_ms_profiled for x in kms])),
        "roofline": dict(roof, traffic=traffic,
                         peak_source="MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback"),
        "regions": region_stats(region_ms, K),
        # the tet forces and vertex sums + spread against the same HBM peak (FP32 corner forces
        # through HBM: the deterministic incidence-row gather)
        "cell_roofline": cell_roofline(wl, kms, peak) if wl.n_tets else None,
        "step_roofline": step_roofline(wl, roof, args.pop_format, ms / K, peak),
        "e2e": {
            "value": job_rate(args.e2e_steps, world, e2e_s),
            "unit": "steps/s",
            "h2d_bytes_per_step": int(nv * 3 * 8),
            "d2h_bytes_per_step": int(nv * 3 * 8),
            "api": "cf_step_exchange: all positions in, 1 step, all positions out, one wait; pinned host buffers",
        },
        "clocks": clk,
    }
    if mean_D is not None:  # Taylor deformation averaged over the cells, after warm-up + timed steps
        out["mean_taylor_D"] = mean_D
        out["mean_cell_strain"] = mean_strain  # (d_max - 2R) / 2R averaged over the cells
    if (rank == 0 and world == 1 and args.precision_steps > 0 and args.workload == "shear"
            and args.pop_format == "f32"):
        out["precision"] = precision_block(P, torch, dev, args.precision_steps)
    default_shear = (args.workload == "shear" and args.pop_format == "f32" and wl.delta == 2 and args.n == 128
                     and args.spread == "float")
    if rank == 0 and world == 1 and default_shear and args.suspension_steps > 0:
        out["suspension"] = suspension_block(P, torch, dev, args.suspension_steps, peak)
        if not args.no_cpu_baseline:
            out["suspension"]["cpu_baseline"] = suspension_cpu_baseline()
    if rank == 0 and world == 1 and default_shear and args.compression_iters > 0:
        m = compression_measure(args.compression_iters)
        out["compression"] = {k: m[k] for k in ("steps_per_s", "steps", "config", "tet_forces_per_s", "adjoint",
                                                "clocks")}
    if rank == 0 and world == 1 and default_shear and args.sweep_steps > 0:
        every = 100 if args.sweep else 1000
        sweep = shear_sweep(P, torch, dev, args.sweep_steps, every)
        out["shear_sweep"] = {"steps": args.sweep_steps, "every": every, "cases": sweep}
    if rank == 0 and world == 1 and args.paper_sweep_steps > 0:
        from workloads import configs

        cases = [(ca, 1.0) for ca in PAPER_SWEEP_CA]
        sweep = shear_sweep(P, torch, dev, args.paper_sweep_steps, 1000, cases,
                            lambda ca, w: configs.paper_box_shear(ca=ca, w=w))
        out["paper_box_sweep"] = {"workload": "paper_box_160x240x80_R16_neo-Hookean", "steps": args.paper_sweep_steps,
                                  "every": 1000, "cases": sweep}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "shear":
        out["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    """The FP64 oracle on the host cores. Each benchmark step processes a
    bounded sample: the fraction 1/m of one coupled step (a contiguous slice
    of the tets, of the vertices and of the lattice nodes, cycling through
    the slices), with m chosen so that the whole run takes about two
    minutes; the rate is scaled back to whole steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import ctypes

    import oracle

    oracle.build()
    L = oracle.lib()
    wl = workload(args)
    sim = oracle.Coupled(wl)
    mesh, fl = sim.mesh, sim.fluid
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))  # noqa: E731
    T, V, N = len(mesh.tets), len(mesh.x), wl.n_nodes
    fc = np.zeros((T, 4, 3))
    fv = np.zeros((V, 3))
    vel = np.zeros((V, 3))
    fout = np.empty_like(fl.f)
    cell = mesh.tmat  # material slot of each tet

    def sample(k, m):
        t0, t1 = k * T // m, (k + 1) * T // m
        v0, v1 = k * V // m, (k + 1) * V // m
        n0, n1 = k * N // m, (k + 1) * N // m
        u = sim.y - mesh.x
        L.ora_tet_force(t0, t1, ip(mesh.tets), dp(mesh.B), dp(mesh.V0), dp(u), ip(cell), dp(mesh.mu),
                        dp(mesh.kappa), dp(mesh.w), dp(fc), None)
        L.ora_gather(v0, v1, ip(mesh.ptr), ip(mesh.idx), dp(fc), dp(fv))
        L.ora_spread(v0, v1, dp(sim.y), dp(fv), wl.nx, wl.ny, wl.nz, wl.delta, dp(sim.Fn))
        L.ora_lbm_step(wl.nx, wl.ny, wl.nz, wl.tau, wl.u_wall_lo, wl.u_wall_hi, dp(fl.g), dp(fl.f), dp(sim.Fn),
                       dp(fout), dp(fl.rho), dp(fl.u), n0, n1)
        L.ora_interp(v0, v1, dp(sim.y), dp(fl.u), wl.nx, wl.ny, wl.nz, wl.delta, dp(vel))
        sim.y[v0:v1] += vel[v0:v1]

    t = time.perf_counter()
    sample(0, 16)
    est_full = 16 * (time.perf_counter() - t)
    budget = 120.0
    m = max(1, min(1024, int(np.ceil((args.steps + args.warmup) * est_full / budget))))
    for k in range(args.warmup):
        sample(k % m, m)
    t0 = time.perf_counter()
    for k in range(args.steps):
        sample((args.warmup + k) % m, m)
    dt = time.perf_counter() - t0
    steps_per_s = args.steps / m / dt
    desc = (f"each step = 1/{m} of a coupled step of {wl.name} (slices of tets, vertices and nodes); "
            f"FP64, 1 thread")
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": steps_per_s,
        "unit": "steps/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 / steps_per_s,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded sphere mesh, fluid at rest at t=0)",
        "config": config_of(wl),
        "mlups": N * steps_per_s / 1e6,
        "tet_forces_per_s": T * steps_per_s,
        "cpu_baseline": {"value": steps_per_s, "unit": "steps/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": steps_per_s, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- compression fit

def compression_measure(fit_iters):
    """Adjoint workload: 64 cells (R = 10, 8,256 tets each) compressed to 80 %
    strain in 8 levels of 2,000 damped steps; the moduli of every cell are
    fitted to force-strain curves generated from hidden moduli, with
    gradients from the hand-written adjoint. Returns the forward rate (one
    step = one relaxation step of all cells), the config and the adjoint's
    figures over `fit_iters` Adam iterations."""
    import torch

    import paper_2003_03130_gb300 as P
    from paper_2003_03130_gb300 import build as cbuild
    from paper_2003_03130_gb300.adjoint import Compression, CompressionCurve
    from workloads import configs

    cbuild.build()
    cs = configs.compression_set()
    ctx = P.cf_create(0)
    ids = P.cf_mesh_init_batch(ctx, [c.x_ref for c in cs.cells], [c.tets for c in cs.cells])
    y0 = np.concatenate([c.x_ref for c in cs.cells])
    z_lo = np.array([c.x_ref[:, 2].min() for c in cs.cells])
    radius = np.array([0.5 * (c.x_ref[:, 2].max() - c.x_ref[:, 2].min()) for c in cs.cells])
    run = Compression(ctx, ids, y0, z_lo, radius, cs.strains, cs.steps, cs.dt, cs.k_plate, cs.ramp, cs.damping)
    nsteps = len(cs.strains) * cs.steps
    target = run.run(cs.hidden_mu, cs.hidden_kappa, cs.hidden_w, record=False)  # warm-up and target curves
    clocks = ClockSampler(0)
    clocks.start()
    t0 = time.perf_counter()
    run.run(cs.hidden_mu, cs.hidden_kappa, cs.hidden_w, record=False)
    fwd_s = time.perf_counter() - t0
    clk = clocks.stop()
    th = torch.tensor(np.stack([np.zeros(len(ids)), np.log(np.full(len(ids), 20.0)), np.zeros(len(ids))], 1),
                      requires_grad=True)
    opt = torch.optim.Adam([th], lr=0.05)
    T = torch.as_tensor(target)
    norm = (T ** 2).sum(1)
    losses, bwd = [], []
    for _ in range(fit_iters):
        mu, ka, w = torch.exp(th[:, 0]), torch.exp(th[:, 1]), torch.sigmoid(th[:, 2])
        loss = (((CompressionCurve.apply(mu, ka, w, run) - T) ** 2).sum(1) / norm).sum()
        t1 = time.perf_counter()
        opt.zero_grad()
        loss.backward()
        bwd.append(time.perf_counter() - t1)
        opt.step()
        losses.append(loss.item())
    mu, ka, w = (torch.exp(th[:, 0]).detach().numpy(), torch.exp(th[:, 1]).detach().numpy(),
                 torch.sigmoid(th[:, 2]).detach().numpy())
    ntets = sum(len(c.tets) for c in cs.cells)
    P.cf_destroy(ctx)
    return {
        "steps_per_s": nsteps / fwd_s,
        "steps": nsteps,
        "forward_s": fwd_s,
        "config": {"workload": f"compression_{len(ids)}cells_R10", "n_tets": ntets, "levels": len(cs.strains),
                   "steps_per_level": cs.steps, "max_strain": cs.strains[-1], "parallelism": "replicas",
                   "l2": "working set ~30 MB, fits L2 (latency-bound relaxation)"},
        "tet_forces_per_s": ntets * nsteps / fwd_s,
        "gpu_launches": 3 * nsteps,
        "adjoint": {
            "backward_s": float(np.median(bwd)) if bwd else None,
            "forward_s": fwd_s,
            "grad_evals_per_s": 1.0 / (fwd_s + float(np.median(bwd))) if bwd else None,
            "fit_iters": fit_iters,
            "loss_first": losses[0] if losses else None,
            "loss_last": losses[-1] if losses else None,
            "median_rel_err_mu": float(np.median(np.abs(mu / cs.hidden_mu - 1))),
            "median_rel_err_kappa": float(np.median(np.abs(ka / cs.hidden_kappa - 1))),
            "median_abs_err_w": float(np.median(np.abs(w - cs.hidden_w))),
        },
        "clocks": clk,
    }


def run_compression(args):
    """The compression workload as the benchmark line: one step = one
    relaxation step of all 64 cells (forward); the adjoint and the fit are
    reported beside it."""
    m = compression_measure(args.fit_iters)
    out = {
        "metric": METRIC,
        "value": m["steps_per_s"],
        "unit": "steps/s",
        "n_gpus": 1,
        "steps": m["steps"],
        "warmup": m["steps"],
        "ms_per_step": 1e3 * m["forward_s"] / m["steps"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded spheres, hidden moduli)",
        "config": m["config"],
        "tet_forces_per_s": m["tet_forces_per_s"],
        "gpu_launches": m["gpu_launches"],
        "adjoint": m["adjoint"],
        "clocks": m["clocks"],
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.workload == "compression" and args.impl != "reference":
        return run_compression(args)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
