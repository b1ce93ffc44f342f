"""Benchmark: cells/s of the TPFA residual + Jacobian assembly on GB300s.

Workload (default): the paper-shaped grid, 512 x 512 x 256 cells (67.1 M),
10 links per cell (4 cardinal + 4 diagonal in-plane, 2 vertical), mixed
precision (FP32 fields and flux arithmetic, FP32 Kahan residual, FP64
accumulation term and FP64 residual/diagonal outputs), seeded synthetic
inputs.  One step = one fused residual + Jacobian assembly over all cells
with a new pressure vector (the repeated-application protocol of Section 3:
"a different pressure vector at every call"); 8 distinct pressure vectors
are cycled.  Inputs and outputs (~6.7 GB per step) exceed the 129 MB L2, so
no flush is needed between steps.

Multi-GPU (torchrun, N > 1): the grid is split into N z-slabs, one per rank;
every step exchanges one plane of pressure with each neighbouring slab (NCCL
point-to-point) and assembles the owned rows; value = the grid's cells /
max-over-ranks time (strong scaling).

--impl reference times the FP64 CPU oracle (the test oracle, unmodified) on
the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cells/s for TPFA residual+Jacobian (1 GB300) and % of HBM roofline, mixed vs FP64"
SHAPE = (512, 512, 256)
CONN = 10
WORKLOAD = "tpfa_residual_jacobian_512x512x256_10pt_mixed"
KERNEL_SOURCES = ["tpfa_assemble.cu", "tpfa_xmarch.cuh", "tpfa_ymarch.cuh", "tpfa_row.cuh", "tpfa_common.cuh",
                  "tpfa_grid.h"]
JVP_SOURCES = ["tpfa_jvp.cu", "tpfa_ymarch.cuh", "tpfa_row.cuh", "tpfa_common.cuh", "tpfa_grid.h"]
MESH_SOURCES = ["tpfa_mesh.cu", "tpfa_mesh.h", "tpfa_row.cuh", "tpfa_common.cuh", "tpfa_grid.h"]
FP64_SOURCES = ["tpfa_assemble.cu", "tpfa_ymarch.cuh", "tpfa_row.cuh", "tpfa_common.cuh", "tpfa_grid.h"]
VJP_SOURCES = ["tpfa_vjp.cu", "tpfa_ymarch.cuh", "tpfa_row.cuh", "tpfa_common.cuh", "tpfa_grid.h"]
# kernel names of the assembly variants, as the launch list shows them
VARIANT_KERNELS = {"tiled2": "k_assemble_xmarch<DIAG,!CRK,W>", "tiled": "k_assemble_ymarch<float,DIAG,!CR,JAC,W>",
                   "tiled_tma": "k_assemble_ymarch_tma<DIAG,!CR,JAC,W=4>", "naive": "k_assemble_naive<float,!CR,JAC>"}


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2304_11274_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# FP64 instruction throughput measured on this GPU (CUDA events, one FMA
# counted once): 604 G/s, 2.0 per clock per SM; a float-to-double conversion
# issues on the same pipe at the same rate
FP64_PEAK_TOPS = 0.604


def profile_values(summary: str, sources=KERNEL_SOURCES) -> dict:
    """The machine-readable lines (- `key`: `value`) of a committed ncu
    summary under profiles/, if it was taken on the current source of
    `sources` (else {}: a figure from another kernel source is not used)."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return {}
    vals = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.strip().startswith("- `"):
                key, _, v = line.strip()[3:].partition("`:")
                vals[key.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256_16") != kernel_source_hash(sources):
        return {}
    return vals


def profile_number(vals: dict, key: str):
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def scaled_traffic(vals: dict, cells: int):
    """DRAM bytes of one launch over `cells` cells, scaled from the summary's
    bytes per cell (the capture runs a smaller grid of the same kernel: the
    pool's rule keeps multi-metric captures to small cases), or None."""
    per_cell = profile_number(vals, "dram_bytes_per_cell")
    return None if per_cell is None else per_cell * cells


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_link_gbs(dev, nbytes=1 << 30, reps=3):
    """Copy bandwidth (GB/s) between pinned host memory and this GPU, each
    direction alone: one 1 GiB cudaMemcpyAsync, best of `reps`.  The
    end-to-end call copies its outputs back every step, so the device-to-host
    figure bounds it."""
    import torch

    n = nbytes // 4
    d = torch.ones(n, dtype=torch.float32, device=dev)
    h = torch.empty(n, dtype=torch.float32).pin_memory()
    out = {}
    for name, fn in (("d2h", lambda: h.copy_(d, non_blocking=True)), ("h2d", lambda: d.copy_(h, non_blocking=True))):
        fn()
        torch.cuda.synchronize(dev)
        best = float("inf")
        for _ in range(reps):
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize(dev)
            best = min(best, time.perf_counter() - t)
        out[name] = nbytes / best / 1e9
    del d, h
    return out


def algorithmic_bytes(n, nnz, precision, crk=False):
    """Bytes one assembly must move at least: each input field read once, each
    output written once (halo re-reads excluded: they are cache traffic)."""
    if precision == "mixed":
        reads = n * (4 + 4 + 8 + 5 * 4 + 4 + (4 if crk else 0))  # p, p^n, m^n, 5 owned T, depth (+phi0)
        writes = n * (8 + 8) + nnz * 4  # R, diag64, CSR values
    else:
        reads = n * (8 + 8 + 8 + 5 * 8 + 8 + (8 if crk else 0))
        writes = n * 8 + nnz * 8
    return reads + writes


# ---------------------------------------------------------------------- our arm


def run_sharded(args, rank, world, local):
    """N > 1 GPUs: the one grid split into z-slabs, one per rank (strong
    scaling: the total work is the 512 x 512 x 256 assembly whatever N).
    One step = the halo exchange (each rank sends its first and last owned
    planes of pressure to its neighbours and receives theirs, NCCL
    point-to-point) + the assembly of the owned rows; value = the grid's
    cells x steps / the slowest rank's time."""
    import torch
    import torch.distributed as dist

    from paper_2304_11274_gb300 import build as libbuild
    from paper_2304_11274_gb300 import synth
    from paper_2304_11274_gb300.api import Slab, slab_bounds
    from paper_2304_11274_gb300.distributed import slab_halo_exchange

    dev = torch.device("cuda", local)
    libbuild.build()
    nx, ny, nz = args.shape
    nxy = nx * ny
    k0, k1, e0, e1 = slab_bounds(nz, world, rank)
    prob = synth.make_problem(nx, ny, nz, synth.BASE_SEED + 1, connectivity=CONN)
    pres = [prob.p] + synth.pressure_sequence(prob, 7, seed=synth.BASE_SEED + 11)
    cut = lambda a: np.ascontiguousarray(a[e0 * nxy:e1 * nxy])
    g = Slab(nx, ny, nz, k0, k1, prob.phys, "mixed", cut(prob.perm), cut(prob.poro), cut(prob.depth), device=dev)
    p_dev = [torch.as_tensor(cut(x).astype(np.float32), device=dev) for x in pres]
    g.set_state(p_dev[0], torch.as_tensor(cut(prob.pn).astype(np.float32), device=dev))
    tiling = g.autotune(None)
    R, vals, diag = g.empty_outputs()
    stream = torch.cuda.current_stream(dev)

    def step(s):
        p = p_dev[s % len(p_dev)]
        slab_halo_exchange(p, nxy, k0, k1, e0, e1, rank, world)
        g.set_pressure(p)
        g.assemble_jacobian(R, vals, diag)

    for s in range(args.warmup):
        step(s)
    g.sync_status()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        step(s)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    clk = clocks.stop()
    g.sync_status()
    ms = torch.tensor([t0.elapsed_time(t1)], device=dev)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX)
    total_ms = float(ms.item())
    value = prob.n * args.steps / (total_ms * 1e-3)

    # end to end through the public API: pinned host pressure of the slab up,
    # halo exchange, assembly, the owned rows' R, values and diag64 down
    Ro, vo, do = g.owned(R, vals, diag)
    ph = [torch.as_tensor(cut(x).astype(np.float32)).pin_memory() for x in pres[:2]]
    Rh, vh, dh = (torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in (Ro, vo, do))
    e2e_steps = max(3, min(args.steps, 10))
    dist.barrier()
    torch.cuda.synchronize(dev)
    te = time.perf_counter()
    for s in range(e2e_steps):
        p = p_dev[0]
        p.copy_(ph[s % 2], non_blocking=True)
        slab_halo_exchange(p, nxy, k0, k1, e0, e1, rank, world)
        g.set_pressure(p)
        g.assemble_jacobian(R, vals, diag)
        Rh.copy_(Ro, non_blocking=True)
        vh.copy_(vo, non_blocking=True)
        dh.copy_(do, non_blocking=True)
        torch.cuda.synchronize(dev)
    es = torch.tensor([time.perf_counter() - te], device=dev)
    dist.all_reduce(es, op=dist.ReduceOp.MAX)
    e2e = {"value": prob.n * e2e_steps / float(es.item()), "unit": "cells/s",
           "h2d_bytes_per_step": prob.n * 4, "d2h_bytes_per_step": prob.n * 16 + 4 * g.lib.tpfa_nnz(nx, ny, nz, CONN),
           "steps": e2e_steps, "api": "Slab.assemble_jacobian with pinned host copies, all ranks"}
    nbytes = algorithmic_bytes(prob.n, g.lib.tpfa_nnz(nx, ny, nz, CONN), "mixed")
    peak, peak_kind = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded; log10 k ~ N(-13, 0.5), phi0 ~ U[0.1, 0.3], hydrostatic + U[-1e5, 1e5] Pa)",
        "config": {"workload": WORKLOAD if tuple(args.shape) == SHAPE else
                   "tpfa_residual_jacobian_%dx%dx%d_10pt_mixed" % tuple(args.shape), "grid": list(args.shape),
                   "cells": prob.n, "links_per_cell": CONN,
                   "parallelism": f"z-slabs x{world} (one plane of pressure exchanged each way per step, NCCL)",
                   "l2": "inputs+outputs 6.7 GB per step > 129 MB L2; no flush",
                   "tiling_rank0": {"rows_per_march": tiling[0], "warps_per_block": tiling[1]}},
        "roofline": {"bound": "hbm", "achieved": nbytes / (total_ms * 1e-3 / args.steps) / 1e9 / world,
                     "peak": peak, "unit": "GB/s per GPU", "peak_kind": peak_kind,
                     "frac": nbytes / (total_ms * 1e-3 / args.steps) / 1e9 / world / peak, "traffic": None,
                     "algorithmic_bytes_per_launch": nbytes / world,
                     "note": "whole-step time (exchange included) against each GPU's share of the bytes"},
        "clocks": clk, "e2e": e2e, "gpu_launches": args.steps,
        "ensemble": None if args.skip_ensemble else measure_ensemble(dev, stream, rank, world),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    dist.destroy_process_group()


def run_ours(args):
    import torch

    rank, world, local = env_rank()
    if world > 1 or args.slabs:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return run_sharded(args, rank, world, local)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2304_11274_gb300 import build as libbuild
    from paper_2304_11274_gb300 import synth
    from paper_2304_11274_gb300.api import Grid

    libbuild.build()
    nx, ny, nz = args.shape
    prob = synth.make_problem(nx, ny, nz, synth.BASE_SEED + 1 + 100 * rank, connectivity=CONN)
    pres = [prob.p] + synth.pressure_sequence(prob, 7, seed=synth.BASE_SEED + 11 + 100 * rank)
    g = Grid(nx, ny, nz, prob.phys, "mixed", prob.perm, prob.poro, prob.depth, device=dev)
    p_dev = [torch.as_tensor(x.astype(np.float32), device=dev) for x in pres]
    pn_dev = torch.as_tensor(prob.pn.astype(np.float32), device=dev)
    g.set_state(p_dev[0], pn_dev)
    tiling = g.autotune(None)  # rows per march, warps per block
    if args.tiling:  # a fixed tiling (profiling a small grid with the large grid's choice)
        g.set_tiling(*args.tiling)
        tiling = tuple(args.tiling)
    R, vals, diag = g.empty_outputs()
    stream = torch.cuda.current_stream(dev)

    def step(s):
        g.set_pressure(p_dev[s % len(p_dev)])
        g.assemble_jacobian(R, vals, diag, kernel=args.kernel)

    for s in range(args.warmup):
        step(s)
    g.sync_status()
    torch.cuda.synchronize(dev)

    # per-launch CUDA events on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        ev[s][0].record(stream)
        step(s)
        ev[s][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    g.sync_status()
    total_ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    ms = torch.tensor([total_ms], device=dev)
    if world > 1:
        torch.distributed.all_reduce(ms, op=torch.distributed.ReduceOp.MAX)
    total_ms = float(ms.item())
    ms_per_step = total_ms / args.steps
    cells = prob.n * world
    value = cells * args.steps / (total_ms * 1e-3)

    # roofline of the assembly kernel (the only kernel in the step)
    nbytes = algorithmic_bytes(prob.n, g.nnz, "mixed")
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    launch_stats = {"mean_ms": statistics.mean(launch_ms), "sd_ms": statistics.pstdev(launch_ms),
                    "min_ms": min(launch_ms), "max_ms": max(launch_ms)}
    peak, peak_kind = measured_peaks()
    achieved = nbytes / avg_launch_s / 1e9
    khash = kernel_source_hash()
    variant = g.kernel_in_use(args.kernel)
    # the kernel's ncu summary (a 256 x 256 x 128 capture of the same
    # variant): warp instructions and DRAM bytes per cell
    prof = profile_values("assemble_mixed_256x256x128_instmix.md")
    if prof.get("variant") != variant:
        prof = {}
    # instruction-issue bound of the same kernel: warp instructions per cell
    # x cells/s against 4 issue slots per SM per clock at the sampled SM clock
    ipc = profile_number(prof, "warp_instructions_per_cell")
    issue_roofline = None
    if ipc is not None:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = (clk or {}).get("sm_mhz") or 2070.0
        issue_peak = 4.0 * sms * mhz * 1e6
        issue_achieved = prob.n / (statistics.mean(launch_ms) * 1e-3) * ipc
        issue_roofline = {"bound": "issue", "warp_instructions_per_cell": ipc, "achieved": issue_achieved / 1e12,
                          "peak": issue_peak / 1e12, "unit": "T warp instructions/s", "frac": issue_achieved / issue_peak,
                          "source": "ncu count per cell in profiles/assemble_mixed_256x256x128_instmix.md"}
    kname = VARIANT_KERNELS[variant]
    traffic = scaled_traffic(prof, prob.n)

    # precision of the timed workload: every row of three planes (top,
    # middle, bottom) of the last timed step, against the oracle
    precision1 = None
    if rank == 0 and not args.skip_configs:
        from paper_2304_11274_gb300 import synth as _s
        last = _s.round_to_f32(_s.Problem(nx, ny, nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                          pres[(args.steps - 1) % len(pres)], prob.pn))
        precision1 = plane_errors(last, "mixed", [0, nz // 2, nz - 1], R, vals, diag)
        precision1["bar"] = 1e-6

    # end to end: host buffers through the C ABI (H2D of p, D2H of R, values, diag64)
    e2e = None
    if not args.no_e2e:
        ph = [torch.as_tensor(x.astype(np.float32)).pin_memory() for x in pres[:2]]
        Rh = torch.empty(prob.n, dtype=torch.float64).pin_memory()
        vh = torch.empty(g.nnz, dtype=torch.float32).pin_memory()
        dh = torch.empty(prob.n, dtype=torch.float64).pin_memory()
        g.assemble_jacobian_host(ph[0], Rh, vh, dh)
        e2e_steps = max(3, min(args.steps, 10))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        te = time.perf_counter()
        for s in range(e2e_steps):
            g.assemble_jacobian_host(ph[s % 2], Rh, vh, dh)
        e2e_s = time.perf_counter() - te
        es = torch.tensor([e2e_s], device=dev)
        if world > 1:
            torch.distributed.all_reduce(es, op=torch.distributed.ReduceOp.MAX)
        e2e = {"value": cells * e2e_steps / float(es.item()), "unit": "cells/s",
               "h2d_bytes_per_step": prob.n * 4, "d2h_bytes_per_step": prob.n * 8 + g.nnz * 4 + prob.n * 8,
               "steps": e2e_steps, "api": "tpfa_assemble_jacobian_host (pinned host buffers)"}
        del ph, Rh, vh, dh
        # the host link: the outputs' copy back bounds the call (the two
        # directions and the assembly overlap in its pipeline)
        link = host_link_gbs(dev)
        t_step = float(es.item()) / e2e_steps
        d2h = e2e["d2h_bytes_per_step"] / t_step / 1e9
        e2e["host_link"] = {"bound": "d2h", "achieved": d2h, "peak": link["d2h"], "unit": "GB/s",
                            "frac": d2h / link["d2h"], "h2d_peak": link["h2d"],
                            "ceiling_cells_per_s": cells / (e2e["d2h_bytes_per_step"] / (link["d2h"] * 1e9)),
                            "peak_measured": "this run: one 1 GiB pinned copy per direction, best of 3"}

    jvp = None if args.skip_jvp else measure_jvp(g, prob, dev, stream, peak)

    # the plain FP64 path on the same grid, for the mixed-vs-FP64 line
    fp64 = None
    if not args.skip_fp64:
        del R, vals, diag
        g.close()
        g64 = Grid(nx, ny, nz, prob.phys, "fp64", prob.perm, prob.poro, prob.depth, device=dev)
        p64 = [torch.as_tensor(x, device=dev) for x in pres[:2]]
        g64.set_state(p64[0], torch.as_tensor(prob.pn, device=dev))
        R64, v64, _ = g64.empty_outputs()
        for s in range(2):
            g64.set_pressure(p64[s % 2])
            g64.assemble_jacobian(R64, v64, None)
        torch.cuda.synchronize(dev)
        nf = 5
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for s in range(nf):
            g64.set_pressure(p64[s % 2])
            g64.assemble_jacobian(R64, v64, None)
        b.record(stream)
        torch.cuda.synchronize(dev)
        g64.sync_status()
        f_ms = a.elapsed_time(b) / nf
        b64 = algorithmic_bytes(prob.n, g64.nnz, "fp64")
        ops = profile_number(profile_values("assemble_fp64_256x256x128_ops.md", FP64_SOURCES), "fp64_ops_per_cell")
        rate = prob.n / (f_ms * 1e-3)
        fp64 = {"value": rate, "unit": "cells/s", "ms_per_step": f_ms,
                "hbm_GBps": b64 / (f_ms * 1e-3) / 1e9, "hbm_frac": b64 / (f_ms * 1e-3) / 1e9 / peak,
                "fp64_roofline": None if ops is None else {
                    "bound": "fp64", "ops_per_cell": ops, "achieved": rate * ops / 1e12, "peak": FP64_PEAK_TOPS,
                    "unit": "T FP64 instructions/s", "frac": rate * ops / 1e12 / FP64_PEAK_TOPS,
                    "peak_kind": "measured (FP64 FMA instructions/s on this GPU, CUDA events)",
                    "ops_source": "ncu count in profiles/assemble_fp64_256x256x128_ops.md"},
                "note": "plain FP64 path, same grid; bound by the FP64 pipe, not HBM"}
        g64.close()

    ensemble = None if args.skip_ensemble else measure_ensemble(dev, stream, rank, world)
    adjoint = None if (args.skip_adjoint or world > 1) else measure_adjoint(dev, stream)
    newton = None if (args.skip_newton or world > 1) else measure_newton(dev, stream)
    mesh = None if (args.skip_mesh or world > 1) else measure_mesh(dev, stream)

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "cells/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded; log10 k ~ N(-13, 0.5), phi0 ~ U[0.1, 0.3], hydrostatic + U[-1e5, 1e5] Pa)",
        "config": {"workload": WORKLOAD if tuple(args.shape) == SHAPE else
                   "tpfa_residual_jacobian_%dx%dx%d_10pt_mixed" % tuple(args.shape), "grid": list(args.shape), "cells": prob.n, "links_per_cell": CONN,
                   "nnz": g.nnz, "precision": "mixed: FP32 flux + Kahan residual, FP64 accumulation/diagonal/R",
                   "l2": "inputs+outputs 6.7 GB per step > 129 MB L2; no flush",
                   "pressure_vectors": len(pres), "parallelism": f"replicas x{world}",
                   "tiling": {"rows_per_march": tiling[0],
                              "warps_per_block": 4 if variant == "tiled_tma" else tiling[1]},
                   "kernel_variant": variant},
        "issue_roofline": issue_roofline,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": None if traffic is None else
                     "ncu DRAM bytes per cell at 256x256x128 (profiles/assemble_mixed_256x256x128_instmix.md) x cells",
                     "algorithmic_bytes_per_launch": nbytes, "peak_kind": peak_kind,
                     "kernel": kname, "kernel_source_sha256_16": khash},
        "launch_ms": launch_stats,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": args.steps,
        "fp64": fp64,
        "ensemble": ensemble,
        "adjoint": adjoint,
        "jvp": jvp,
        "newton": newton,
        "mesh": mesh,
    }
    if rank == 0 and world == 1 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_budget)
    if precision1 is not None:
        line["error_vs_oracle"] = precision1
    if rank == 0 and world == 1 and not args.skip_configs:
        line["configs"] = measure_configs(dev, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def measure_ensemble(dev, stream, rank=0, world=1, reps=10):
    """The 64-model uneven ensemble (nx, ny ~ U{64..256}, nz ~ U{32..128},
    10 links, mixed): one graph-captured persistent launch per step against
    sequential single-grid launches, both with autotuned tiling.  With
    several ranks the models are split by cell count (no collective on the
    data path); value = all models' cells / the slowest rank's time."""
    import torch

    from paper_2304_11274_gb300 import synth
    from paper_2304_11274_gb300.api import Ensemble, Grid
    from paper_2304_11274_gb300.distributed import aggregate, partition

    shapes = synth.ensemble_shapes()
    mine = partition([a * b * c for a, b, c in shapes], world, rank)
    grids, keep = [], []
    for m in mine:
        nx, ny, nz = shapes[m]
        prob = synth.make_problem(nx, ny, nz, synth.BASE_SEED + 1000 + m, connectivity=CONN)
        g = Grid(nx, ny, nz, prob.phys, "mixed", prob.perm, prob.poro, prob.depth, device=dev)
        p = torch.as_tensor(prob.p.astype(np.float32), device=dev)
        pn = torch.as_tensor(prob.pn.astype(np.float32), device=dev)
        g.set_state(p, pn)
        keep.append((p, pn))
        grids.append(g)
    cells = sum(g.n for g in grids)
    ens = Ensemble(grids)
    outs = ens.allocate_outputs()
    ens.autotune(None)
    for g in grids:
        g.autotune(None)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    batched_ms = timed(ens.assemble)

    def sequential():
        for m, g in enumerate(grids):
            R, vals, diag = outs[m]
            g.assemble_jacobian(R, vals, diag)

    seq_ms = timed(sequential)
    for g in grids:
        g.sync_status()
    info = ens.tiling()
    ens.close()
    for g in grids:
        g.close()
    nbytes = sum(algorithmic_bytes(g.n, g.nnz, "mixed") for g in grids)
    total, b_s = aggregate(cells, batched_ms * 1e-3, device=dev)
    _, s_s = aggregate(cells, seq_ms * 1e-3, device=dev)
    peak, peak_kind = measured_peaks()
    achieved = nbytes / (batched_ms * 1e-3) / 1e9
    return {"models": len(shapes), "cells": total, "unit": "cells/s", "ranks": world,
            "batched_value": total / b_s, "batched_ms": b_s * 1e3,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "algorithmic_bytes_per_launch": nbytes, "peak_kind": peak_kind,
                         "traffic": None, "kernel": "k_assemble_batch (this rank's models)"},
            "sequential_value": total / s_s, "sequential_ms": s_s * 1e3,
            "launches_per_step": {"batched": 1, "sequential": len(mine)},
            "tiling": info, "scaling": "strong (fixed 64 models split across ranks)",
            "note": "one CUDA-graph launch of the persistent kernel vs one launch per model"}


def measure_jvp(g, prob, dev, stream, peak, reps=10):
    """Matrix-free J w (the Krylov operator) on the headline grid, mixed:
    reads p, p^n, m^n, 5 owned T, depth and w; writes J w (56 B per cell)."""
    import torch

    from paper_2304_11274_gb300 import synth

    w = torch.as_tensor(synth.cotangent(prob.n, synth.BASE_SEED + 40), device=dev)
    Jw = torch.empty(prob.n, dtype=torch.float64, device=dev)
    for _ in range(3):
        g.jvp(w, out=Jw)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        g.jvp(w, out=Jw)
    b.record(stream)
    torch.cuda.synchronize(dev)
    g.sync_status()
    ms = a.elapsed_time(b) / reps
    nbytes = prob.n * (4 + 4 + 8 + 5 * 4 + 4 + 8 + 8)
    tiling = g.tiling()
    khash = kernel_source_hash(JVP_SOURCES)
    prof = profile_values("jvp_mixed_256x256x128.md", JVP_SOURCES)
    del w, Jw
    return {"grid": [prob.nx, prob.ny, prob.nz], "value": prob.n / (ms * 1e-3), "unit": "cells/s", "ms": ms,
            "roofline": {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": nbytes / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_launch": nbytes,
                         "traffic": scaled_traffic(prof, prob.n),
                         "traffic_source": "ncu DRAM bytes per cell at 256x256x128 (profiles/jvp_mixed_256x256x128.md) x cells",
                         "warp_instructions_per_cell": profile_number(prof, "warp_instructions_per_cell"),
                         "kernel_source_sha256_16": khash},
            "kernel": "k_jvp_ymarch<DIAG,!CR,W=%d>" % tiling[1],
            "tiling": {"rows_per_march": tiling[0], "warps_per_block": tiling[1]},
            "outputs": "J w (FP64)"}


def measure_mesh(dev, stream, reps=20):
    """Residual + Jacobian on a faulted corner-point-like mesh given as a
    connection list: 256 x 256 x 128 cells before 5 % pinch-outs, 10 links
    per cell plus the fault's non-neighbour connections, mixed."""
    import torch

    from paper_2304_11274_gb300 import synth
    from paper_2304_11274_gb300.api import Mesh

    m = synth.make_mesh(256, 256, 128, seed=synth.BASE_SEED + 5, connectivity=10)
    g = Mesh(m.n, m.ci, m.cj, m.T, m.V, m.poro, m.depth, m.phys, "mixed", device=dev)
    g.set_state(m.p.astype(np.float32), m.pn.astype(np.float32))
    R, vals, diag = g.empty_outputs()
    for _ in range(3):
        g.assemble(R, vals, diag)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        g.assemble(R, vals, diag)
    b.record(stream)
    torch.cuda.synchronize(dev)
    g.sync_status()
    ms = a.elapsed_time(b) / reps
    # per cell: row_ptr 8, p 4, p^n 4, m^n 8, depth 4 read, R 8 and diag64 8 written;
    # per entry: col_idx 4 read and the value 4 written; per off-diagonal entry: T 4 read
    nbytes = m.n * (8 + 4 + 4 + 8 + 4 + 8 + 8) + g.nnz * (4 + 4) + (g.nnz - m.n) * 4
    peak, _ = measured_peaks()
    khash = kernel_source_hash(MESH_SOURCES)
    out = {"cells": m.n, "connections": m.nc, "nnz": g.nnz, "value": m.n / (ms * 1e-3), "unit": "cells/s", "ms": ms,
           "roofline": {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": nbytes / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_launch": nbytes,
                        "traffic": profile_number(profile_values("mesh_mixed_256x256x128_faulted.md", MESH_SOURCES),
                                                  "dram_bytes_per_launch"),
                        "kernel_source_sha256_16": khash},
           "kernel": "k_mesh_assemble<float,!CR,JAC>",
           "workload": "faulted mesh 256x256x128, 10 links + fault NNCs, 5 % inactive, mixed"}
    del R, vals, diag
    g.close()
    return out


def measure_newton(dev, stream, reps=3):
    """One Newton step of Eq. vk (assemble, BiCGStab with the z-line
    preconditioner to rtol 1e-8, update) on 128^3, 10 links, mixed, from the
    synthetic state; each timed step restarts from the same p."""
    import torch

    from paper_2304_11274_gb300 import synth
    from paper_2304_11274_gb300.api import Grid

    prob = synth.config_problem(4)
    g = Grid(prob.nx, prob.ny, prob.nz, prob.phys, "mixed", prob.perm, prob.poro, prob.depth, device=dev)
    p0 = torch.as_tensor(prob.p.astype(np.float32), device=dev)
    g.set_state(p0, torch.as_tensor(prob.pn.astype(np.float32), device=dev))
    p = p0.clone()
    g.newton_step(p, rtol=1e-8, max_iters=5000)  # warm-up (allocates the workspace)
    times, iters = [], []
    for _ in range(reps):
        p.copy_(p0)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, _, _ = g.newton_step(p, rtol=1e-8, max_iters=5000)
        b.record(stream)
        torch.cuda.synchronize(dev)
        times.append(a.elapsed_time(b))
        iters.append(st["iterations"])
    g.sync_status()
    ms = statistics.median(times)
    it = statistics.median(iters)
    # two stencil SpMVs (FP32 values, 4 nnz + 32 N each), the FP64 vector
    # updates (120 N) and two z-line applications (64 N each)
    per_iter_bytes = 8 * g.nnz + 312 * prob.n
    ms_iter = ms / max(it, 1)
    g.close()
    peak, _ = measured_peaks()
    return {"grid": [prob.nx, prob.ny, prob.nz], "unit": "ms per Newton step", "ms": ms,
            "krylov_iterations": it, "ms_per_iteration": ms_iter, "rtol": 1e-8,
            "roofline_per_iteration": {"bound": "hbm", "algorithmic_bytes": per_iter_bytes,
                                       "achieved": per_iter_bytes / (ms_iter * 1e-3) / 1e9, "peak": peak,
                                       "unit": "GB/s", "frac": per_iter_bytes / (ms_iter * 1e-3) / 1e9 / peak},
            "preconditioner": "z-line (tridiagonal along z, per column)",
            "note": "includes one assembly and the update; 10 kernels per BiCGStab iteration, 8 iterations per CUDA-graph launch and host poll"}


def measure_adjoint(dev, stream, reps=20):
    """Adjoint (v^T dR/dp and v^T dR/d ln k) on 128^3, 10 links, mixed."""
    import torch

    from paper_2304_11274_gb300 import synth
    from paper_2304_11274_gb300.api import Grid

    prob = synth.config_problem(4)
    g = Grid(prob.nx, prob.ny, prob.nz, prob.phys, "mixed", prob.perm, prob.poro, prob.depth, device=dev)
    g.set_state(torch.as_tensor(prob.p.astype(np.float32), device=dev),
                torch.as_tensor(prob.pn.astype(np.float32), device=dev))
    v = torch.as_tensor(synth.cotangent(prob.n, synth.BASE_SEED + 4), device=dev)
    for _ in range(3):
        g.vjp(v)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        g.vjp(v)
    b.record(stream)
    torch.cuda.synchronize(dev)
    g.sync_status()
    ms = a.elapsed_time(b) / reps
    tiling = g.tiling()
    g.close()
    # reads p, p^n, depth, k (4 B each), 5 owned T (20 B), m^n and v (8 B each); writes g_p, g_lnk
    nbytes = prob.n * (4 * 4 + 5 * 4 + 8 + 8 + 16)
    peak, _ = measured_peaks()
    prof = profile_values("vjp_mixed_128x128x128.md", VJP_SOURCES)
    return {"grid": [prob.nx, prob.ny, prob.nz], "value": prob.n / (ms * 1e-3), "unit": "cells/s", "ms": ms,
            "roofline": {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": nbytes / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_launch": nbytes,
                         "timed": "per call: the cotangent split pre-pass and the march",
                         "traffic": profile_number(prof, "dram_bytes_per_launch"),
                         "warp_instructions_per_cell": profile_number(prof, "warp_instructions_per_cell"),
                         "kernel_source_sha256_16": kernel_source_hash(VJP_SOURCES)},
            "kernel": "k_vjp_ymarch<DIAG,!CR,W=%d>" % tiling[1],
            "tiling": {"rows_per_march": tiling[0], "warps_per_block": tiling[1]},
            "outputs": "g_p and g_lnk (FP64)"}


# ---------------------------------------------------------------------- precision statement
#
# The residual and Jacobian of each configuration against the FP64 oracle
# (normwise residual, row-normwise Jacobian, entrywise max / RMS; a link whose
# oracle dPhi lies within the path's rounding of zero may be upwinded either
# way).  Runs outside every timed region; the oracle is the test oracle.


def _plane_row_starts(nx, ny, nz, conn):
    """CSR offset of each plane's first row (nz + 1 values), from the closed
    form: a plane's rows hold its in-plane entries plus one entry per
    vertical link."""
    from paper_2304_11274_gb300 import _capi
    lib = _capi.load()
    inplane = lib.tpfa_nnz(nx, ny, 1, conn)
    counts = [inplane + nx * ny * ((k > 0) + (k < nz - 1)) for k in range(nz)]
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def _errors(R_gpu, J_gpu, ref, rows=None):
    """(residual, jacobian_row, entry_max, entry_rms) of GPU values against an
    oracle reference (oracle.compare.reference), optionally over a row range."""
    from oracle import compare as OC
    if rows is None:
        eR = OC.residual_error(R_gpu, ref)
        eJ = OC.jacobian_row_error(J_gpu, ref)
        emax, erms = OC.entry_stats(J_gpu, ref)
        return {"residual": eR, "jacobian_row": eJ, "entry_max": emax, "entry_rms": erms}
    r0, r1 = rows
    rp = ref["row_ptr"]
    e0, e1 = rp[r0], rp[r1]
    sub = {"R": ref["R"][r0:r1], "J": ref["J"][e0:e1], "row_ptr": rp[r0:r1 + 1] - e0,
           "R_alt": None if ref.get("R_alt") is None else ref["R_alt"][r0:r1],
           "J_alt": None if ref.get("J_alt") is None else ref["J_alt"][e0:e1]}
    return _errors(R_gpu, J_gpu, sub)


def plane_errors(prob, precision, planes, R, vals, diag):
    """Errors of the rows of the given z-planes (device outputs R, vals,
    diag64 of the whole grid) against the oracle run on the slab of the
    plane and its vertical neighbours (a row depends only on its cell and
    adj(K))."""
    import oracle
    from oracle import compare as OC
    from paper_2304_11274_gb300 import synth
    nx, ny, nz = prob.nx, prob.ny, prob.nz
    conn = prob.phys["connectivity"]
    nxy = nx * ny
    starts = _plane_row_starts(nx, ny, nz, conn)
    eps = OC.EPS32 if precision == "mixed" else OC.EPS64
    worst = {"residual": 0.0, "jacobian_row": 0.0, "entry_max": 0.0, "entry_rms2": 0.0}
    rows = 0
    for k in planes:
        k0, k1 = max(k - 1, 0), min(k + 2, nz)
        cut = lambda a: a.reshape(nz, nxy)[k0:k1].reshape(-1)
        sub = synth.Problem(nx, ny, k1 - k0, prob.phys, cut(prob.perm), cut(prob.poro), cut(prob.depth),
                            cut(prob.p), cut(prob.pn))
        ref = OC.reference(sub, eps)
        kk = k - k0
        Rg = R[k * nxy:(k + 1) * nxy].cpu().numpy()
        Jg = vals[int(starts[k]):int(starts[k + 1])].cpu().numpy().astype(np.float64)
        if diag is not None:  # the FP64 diagonal in place of its FP32 copy
            rp = ref["row_ptr"][kk * nxy:(kk + 1) * nxy + 1] - ref["row_ptr"][kk * nxy]
            cols = ref["col_idx"][ref["row_ptr"][kk * nxy]:ref["row_ptr"][(kk + 1) * nxy]]
            rowid = np.repeat(np.arange(kk * nxy, (kk + 1) * nxy), np.diff(rp))
            Jg[cols == rowid] = diag[k * nxy:(k + 1) * nxy].cpu().numpy()
        e = _errors(Rg, Jg, ref, rows=(kk * nxy, (kk + 1) * nxy))
        for key in ("residual", "jacobian_row", "entry_max"):
            worst[key] = max(worst[key], e[key])
        worst["entry_rms2"] += e["entry_rms"] ** 2 * nxy
        rows += nxy
    worst["entry_rms"] = float(np.sqrt(worst.pop("entry_rms2") / rows))
    worst["rows"] = f"every row of planes {list(planes)} ({rows} rows)"
    return worst


# Arm core names by the "CPU part" field of /proc/cpuinfo (implementer 0x41)
ARM_PARTS = {"0xd0c": "Arm Neoverse N1", "0xd40": "Arm Neoverse V1", "0xd49": "Arm Neoverse N2",
             "0xd4f": "Arm Neoverse V2"}


def host_info(cpuinfo="/proc/cpuinfo"):
    """Host threads and CPU model (x86: the model name; Arm, which has no
    model name line: the core named from its part number)."""
    fields = {}
    try:
        with open(cpuinfo) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip().lower(), v.strip())
    except OSError:
        pass
    cpu = fields.get("model name") or fields.get("hardware") or ""
    part = fields.get("cpu part", "")
    if not cpu and part:
        cpu = f"{ARM_PARTS.get(part.lower(), 'Arm core')} (CPU part {part})"
    return {"nproc": os.cpu_count(), "cpu_model": cpu or os.uname().machine, "machine": os.uname().machine}


def time_oracle(fn, min_reps=3, min_s=0.5):
    """Mean wall time of fn() over at least min_reps calls and min_s seconds."""
    fn()  # warm-up
    reps, t = 0, 0.0
    while reps < min_reps or t < min_s:
        t0 = time.perf_counter()
        fn()
        t += time.perf_counter() - t0
        reps += 1
    return t / reps, reps


def oracle_rates(prob, kind="assemble", v=None):
    """Oracle cells/s single-threaded and on every thread it may use."""
    import oracle
    allt = oracle.max_threads()
    pat = oracle.pattern(prob.nx, prob.ny, prob.nz, prob.phys["connectivity"])
    if kind == "assemble":
        fn = lambda: oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth,
                                     prob.p, prob.pn, pat=pat)
    else:
        fn = lambda: oracle.vjp(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth, prob.p,
                                prob.pn, v)
    out = {}
    for label, n in (("threads_1", 1), ("threads_all", allt)):
        oracle.set_threads(n)
        sec, reps = time_oracle(fn)
        out[label] = {"value": prob.n / sec, "unit": "cells/s", "threads": n, "reps": reps}
    oracle.set_threads(allt)
    out["sample"] = f"{prob.nx}x{prob.ny}x{prob.nz} ({prob.n} cells), {kind}"
    return out


def oracle_rates_sum(probs, sample):
    """Oracle cells/s over several grids (total cells / total time),
    single-threaded and on every thread."""
    import oracle
    allt = oracle.max_threads()
    out = {}
    for label, n in (("threads_1", 1), ("threads_all", allt)):
        oracle.set_threads(n)
        cells, sec = 0, 0.0
        for prob in probs:
            pat = oracle.pattern(prob.nx, prob.ny, prob.nz, prob.phys["connectivity"])
            t, _ = time_oracle(lambda: oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro,
                                                       prob.depth, prob.p, prob.pn, pat=pat), min_reps=1, min_s=0.2)
            cells += prob.n
            sec += t
        out[label] = {"value": cells / sec, "unit": "cells/s", "threads": n}
    oracle.set_threads(allt)
    out["sample"] = sample
    return out


def gpu_rate(g, p_dev, R, vals, diag, calls, stream, dev):
    """Cells/s of the fused assembly on a bound grid (CUDA events)."""
    import torch
    for _ in range(3):
        g.assemble_jacobian(R, vals, diag)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(calls):
        g.assemble_jacobian(R, vals, diag)
    b.record(stream)
    torch.cuda.synchronize(dev)
    g.sync_status()
    ms = a.elapsed_time(b) / calls
    return {"value": g.n / (ms * 1e-3), "unit": "cells/s", "ms": ms, "calls": calls}


def measure_configs(dev, stream, full=True):
    """Per-configuration precision and rates: config 0 (32^3, 6 links,
    FP64; every row), config 2 (256^3 layered, 10 links; mixed and FP64 GPU
    paths, every row), config 4 (128^3 adjoint; g_p and g_lnk), with the
    oracle timed on the host single-threaded and on every thread."""
    import torch

    import oracle
    from oracle import compare as OC
    from paper_2304_11274_gb300 import synth
    from paper_2304_11274_gb300.api import Grid

    oracle.build()
    out = {"host": host_info()}

    # config 0: FP64, 32^3, 6 links; L2-resident (16 MB per call)
    p0 = synth.config_problem(0)
    g = Grid(p0.nx, p0.ny, p0.nz, p0.phys, "fp64", p0.perm, p0.poro, p0.depth, device=dev)
    g.set_state(p0.p, p0.pn)
    R, vals, _ = g.empty_outputs()
    rate = gpu_rate(g, None, R, vals, None, 1000, stream, dev)
    ref = OC.reference(p0, OC.EPS64)
    err = _errors(R.cpu().numpy(), vals.cpu().numpy(), ref)
    g.close()
    out["config0_32x32x32_6pt_fp64"] = {
        "gpu": dict(rate, note="1000 calls, inputs and outputs L2-resident (16 MB), so no roofline"),
        "error_vs_oracle": dict(err, rows="every row", bar=1e-12), "oracle": oracle_rates(p0)}

    # config 2: the 256^3 layered precision study, both GPU paths, every row
    p2 = synth.config_problem(2)
    c2 = {"gpu": {}, "error_vs_oracle": {}}
    for precision in ("mixed", "fp64"):
        prob = synth.round_to_f32(p2) if precision == "mixed" else p2
        g = Grid(prob.nx, prob.ny, prob.nz, prob.phys, precision, prob.perm, prob.poro, prob.depth, device=dev)
        g.set_state(prob.p, prob.pn)
        R, vals, diag = g.empty_outputs()
        c2["gpu"][precision] = gpu_rate(g, None, R, vals, diag, 10 if precision == "fp64" else 20, stream, dev)
        if full:
            ref = OC.reference(prob, OC.EPS32 if precision == "mixed" else OC.EPS64)
            J = vals.cpu().numpy().astype(np.float64)
            if diag is not None:
                rows = np.repeat(np.arange(prob.n), np.diff(ref["row_ptr"]))
                J[ref["col_idx"] == rows] = diag.cpu().numpy()
            c2["error_vs_oracle"][precision] = dict(_errors(R.cpu().numpy(), J, ref), rows="every row",
                                                    bar=1e-6 if precision == "mixed" else 1e-12,
                                                    ambiguous_links=int(ref["ambiguous"].sum()))
            del ref, J
        del R, vals, diag
        g.close()
    c2["gpu"]["mixed_over_fp64"] = c2["gpu"]["mixed"]["value"] / c2["gpu"]["fp64"]["value"]
    c2["oracle"] = oracle_rates(synth.round_to_f32(synth.make_problem(
        256, 256, 16, synth.BASE_SEED + 2, connectivity=10, layered=True, layered_pressure=True)))
    out["config2_256x256x256_layered_10pt"] = c2

    # config 4: the adjoint on 128^3 (mixed), against the oracle's gradient
    p4 = synth.round_to_f32(synth.config_problem(4))
    p4.perm = p4.perm.astype(np.float32).astype(np.float64)  # the adjoint's k is stored in FP32
    v = synth.cotangent(p4.n, seed=synth.BASE_SEED + 4)
    g = Grid(p4.nx, p4.ny, p4.nz, p4.phys, "mixed", p4.perm, p4.poro, p4.depth, device=dev)
    g.set_state(p4.p.astype(np.float32), p4.pn.astype(np.float32))
    gp, gk = (x.cpu().numpy() for x in g.vjp(v))
    g.sync_status()
    g.close()
    gp_ref, gk_ref = oracle.vjp(p4.nx, p4.ny, p4.nz, p4.phys, p4.perm, p4.poro, p4.depth, p4.p, p4.pn, v)
    nw = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
    out["config4_128x128x128_adjoint_mixed"] = {
        "error_vs_oracle": {"g_p": nw(gp, gp_ref), "g_lnk": nw(gk, gk_ref), "norm": "normwise (inf)", "bar": 1e-6},
        "oracle": oracle_rates(synth.round_to_f32(synth.make_problem(128, 128, 16, synth.BASE_SEED + 4,
                                                                     connectivity=10)), kind="vjp",
                               v=synth.cotangent(128 * 128 * 16, seed=5))}
    # config 1 on the host: a 4-plane slab of the 512 x 512 x 256 workload
    out["config1_512x512x256_10pt_mixed"] = {
        "oracle": oracle_rates(synth.round_to_f32(synth.make_problem(512, 512, 4, synth.BASE_SEED + 1,
                                                                     connectivity=CONN)))}
    # config 3 on the host: the sum over a sample of the ensemble's models
    shapes = synth.ensemble_shapes()
    sample = [0, len(shapes) // 3, 2 * len(shapes) // 3, len(shapes) - 1]
    probs = [synth.round_to_f32(synth.make_problem(*shapes[m], synth.BASE_SEED + 1000 + m, connectivity=CONN))
             for m in sample]
    out["config3_ensemble"] = {"note": "each model's rows are bit-identical to its single-grid assembly "
                                       "(tests/test_gpu_ensemble.py), so its error is config 1's",
                               "oracle": oracle_rates_sum(probs, "models %s of the 64 (%d cells)" %
                                                          (sample, sum(q.n for q in probs)))}
    return out


# ---------------------------------------------------------------------- oracle on the host


def cpu_sample_problem():
    """A bounded slab of the same workload: 512 x 512 x 32 cells (8.4 M, one
    eighth of the grid), same distributions and physics, FP32-rounded inputs."""
    from paper_2304_11274_gb300 import synth
    return synth.round_to_f32(synth.make_problem(512, 512, 32, synth.BASE_SEED + 1, connectivity=CONN))


def cpu_baseline(budget_s=20.0):
    import oracle
    prob = cpu_sample_problem()
    pat = oracle.pattern(prob.nx, prob.ny, prob.nz, CONN)
    reps, t = 0, 0.0
    while t < budget_s and reps < 50:
        t0 = time.perf_counter()
        oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth, prob.p, prob.pn, pat=pat)
        t += time.perf_counter() - t0
        reps += 1
    return {"value": prob.n * reps / t, "unit": "cells/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{prob.nx}x{prob.ny}x{prob.nz} slab of the same workload, {reps} assemblies, {t:.1f} s"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    oracle.build()
    prob = cpu_sample_problem()
    pat = oracle.pattern(prob.nx, prob.ny, prob.nz, CONN)
    for _ in range(args.warmup):
        oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth, prob.p, prob.pn, pat=pat)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.assemble(prob.nx, prob.ny, prob.nz, prob.phys, prob.perm, prob.poro, prob.depth, prob.p, prob.pn, pat=pat)
    t = time.perf_counter() - t0
    value = prob.n * args.steps / t
    sample = f"{prob.nx}x{prob.ny}x{prob.nz} slab of the 512x512x256 workload per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cells/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)", "config": {"workload": WORKLOAD, "grid": list(SHAPE), "sample": sample},
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--skip-ensemble", action="store_true", help="skip the 64-model batched ensemble line")
    ap.add_argument("--skip-adjoint", action="store_true", help="skip the adjoint (VJP) line")
    ap.add_argument("--skip-jvp", action="store_true", help="skip the matrix-free J w line")
    ap.add_argument("--skip-newton", action="store_true", help="skip the Newton-step line")
    ap.add_argument("--skip-mesh", action="store_true", help="skip the general-mesh line")
    ap.add_argument("--slabs", action="store_true",
                    help="run the z-slab decomposition even on one rank (under torchrun; N > 1 always does)")
    ap.add_argument("--skip-configs", action="store_true",
                    help="skip the per-configuration precision statement and the config 0 / 2 / 4 lines")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tiled", "tiled2", "tiled_tma"],
                    help="assembly kernel variant of the timed step (auto = the library's choice)")
    ap.add_argument("--tiling", type=int, nargs=2, default=None, metavar=("ROWS", "WARPS"),
                    help="fixed tiling of the timed assembly instead of the autotuned one (profiling aid)")
    ap.add_argument("--shape", type=int, nargs=3, default=list(SHAPE),
                    help="grid size (default: the 512 x 512 x 256 workload; smaller shapes are for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
