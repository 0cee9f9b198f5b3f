#!/usr/bin/env python
"""Benchmark of the batched AMR ideal-MHD advance on GB300.

Workload: 3D periodic blast wave, 128^3 cells split into 512 patches of 16^3
(rho = 1, p = 0.1, p = 10 inside r < 0.1, uniform B = (1,1,1)/sqrt 3). A step
is one coarse step of the whole hot path: CFL reduction, the level advance
(MUSCL-Hancock + minmod, HLLD, constrained transport) of every patch, replayed
as one CUDA graph; the level tiles the periodic domain with equal patches, so
the advance reads its halo from the neighbour patches and no ghost fill runs.
The headline runs the mixed-precision path (FP32 stencil, FP64 primitive
recovery, registers, dt). Also reported: the FP64 path, the FP64
one-patch-per-launch baseline, the level advance alone against the HBM and
FP32 rooflines, end-to-end runs through the C ABI with the state exchanged with
pinned host memory every step (pipelined and serial), the CPU oracle on one
core and on every core, and the extra workloads (deep AMR clumps, shock clump,
the paper's cylinder, weak scaling over SM partitions, the adjoint).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MHD cell-updates/s on 1 GB300 (FP32 vs FP64) and achieved HBM GB/s vs peak"
UNIT = "cell-updates/s"
# Algorithmic FP operations of one 3D cell update (recovery, slopes, predictor,
# face states, 3 HLLD solves, reference and 3 GS edge EMFs, updates), counted
# by running the oracle's per-cell formulas with a counting scalar type
# (oracle/opcount.cpp, 2000 subsonic samples, seed 1; tests/test_oracle_opcount.py).
FLOPS_PER_CELL_UPDATE_3D = 1504.0
TILE_NAMES = {0: "16x16", 1: "16x16/512 threads", 2: "16x8", 3: "8x8", 4: "12x12"}
# DRAM bytes (read + write) of one launch of the fused advance (direct halo
# reads, 16x8 tile) on the 128^3 blast in 16^3 patches, mixed precision, from
# one ncu capture of that launch (profiles/k_advance3d_fused_blast3d_128.md)
FUSED_TRAFFIC_BYTES = 242.48e6  # 167.31 MB read + 75.17 MB written
# FP32 lanes per SM (the derived ALU peak: SMs x lanes x 2 (FMA) x max SM clock)
FP32_LANES = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=128)
    p.add_argument("--psize", type=int, default=16)
    p.add_argument("--skip-extras", action="store_true", help="headline only (no FP64/baseline/e2e/oracle legs)")
    p.add_argument("--leg", default=None,
                   choices=["adjoint", "deep", "shockclump", "error", "cylinder", "weakscale", "queue"],
                   help="run one extra leg alone and print its JSON (for profiling)")
    p.add_argument("--leg-steps", type=int, default=None, help="coarse steps of the --leg run")
    return p.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.t0 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v, device="cuda"):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms_local, device="cuda"):
    """Whole-job throughput of N replicas (weak scaling): the units all ranks
    processed over the slowest rank's time; returns (rate per second, max ms)."""
    ms_max = allmax(world, ms_local, device)
    return units_per_rank * world / (ms_max / 1e3), ms_max


def make_ctx(pb, precision, strict=False, baseline=False, graph=True):
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    stream = torch.cuda.Stream()
    ctx = A.context_for(pb, precision=precision, strict_fp64=strict, stream=stream.cuda_stream)
    if baseline:
        ctx.set_option(A.OPT_ADVANCE, 1)
    if not graph:
        ctx.set_option(A.OPT_GRAPH, 0)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    ctx.load_state(pb.state)
    torch.cuda.synchronize()
    return ctx, stream


def timed_steps(ctx, stream, k):
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    l0 = ctx.query(A.Q_KERNEL_LAUNCHES)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.step(k, want_dt=False)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), ctx.query(A.Q_KERNEL_LAUNCHES) - l0


def advance_alone(ctx, stream, reps):
    """CUDA-event times of the level-0 advance and of its ghost fill, each alone
    on the launching stream, averaged over reps calls: (advance ms, fill ms)."""
    import torch
    dt = ctx.cfl_dt()
    tot = tot_f = 0.0
    for _ in range(reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        ctx.fill_ghosts(0, 1)
        e[1].record(stream)
        e[1].synchronize()
        e[2].record(stream)
        ctx.advance_level(0, dt, 1)
        e[3].record(stream)
        e[3].synchronize()
        tot_f += e[0].elapsed_time(e[1])
        tot += e[2].elapsed_time(e[3])
    return tot / reps, tot_f / reps


def e2e_run(pb, precision, k):
    """Through the C ABI with host buffers: every step uploads the whole state
    from pinned host memory, advances one coarse step and reads the whole state
    back (amrmhd_set/get_state_all, in the stored element type: float for the
    mixed-precision context, double for FP64), timed with the host clock over k
    steps, in two ways:
    - serial: amrmhd_set_state_all / amrmhd_get_state_all with the pinned host
      buffers (the packing kernels read and write them over the host link), one
      step after the other;
    - pipelined (a stream of independent inputs): each step's input is copied
      from pinned host memory into one of two device staging buffers on an
      upload stream while the previous step computes, loaded with
      amrmhd_set_state_all from the device buffer, stepped (amrmhd_step_async:
      the host queues ahead), written with amrmhd_get_state_all into one of two
      device result buffers and copied to pinned host memory on a download
      stream while the next step computes; amrmhd_sync at the end.
    Returns (pipelined rate, serial rate, bytes per direction per step, host
    link rates)."""
    import numpy as np
    import torch
    import ctypes as C
    from paper_1110_1616_gb300 import amrmhd as A
    ctx, stream = make_ctx(pb, precision)
    ctx.autotune(3)
    f32 = precision == A.MIXED
    host = np.concatenate([ctx.pack(pb.state, f) for f in range(8)])
    host_in = torch.from_numpy(host.astype(np.float32) if f32 else host).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    lib = A.lib()
    set_all = lib.amrmhd_set_state_all_f32 if f32 else lib.amrmhd_set_state_all
    get_all = lib.amrmhd_get_state_all_f32 if f32 else lib.amrmhd_get_state_all

    def one():
        ctx._check(set_all(ctx.h, C.c_void_p(host_in.data_ptr()), 0), "set_all")
        ctx.step(1, want_dt=False)
        ctx._check(get_all(ctx.h, C.c_void_p(host_out.data_ptr()), 0), "get_all")

    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(k):
        one()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0

    # pipelined: double-buffered device staging, uploads and downloads on their
    # own streams, ordered against the context's stream by events
    up, dn = torch.cuda.Stream(), torch.cuda.Stream()
    dev_in = [torch.empty_like(host_in, device="cuda") for _ in range(2)]
    dev_out = [torch.empty_like(host_in, device="cuda") for _ in range(2)]
    outs = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    ev = {n: [torch.cuda.Event() for _ in range(2)] for n in ("in_ready", "in_free", "out_ready", "out_free")}

    def pipelined(n):
        for b in range(2):  # nothing outstanding on either buffer
            ev["in_free"][b].record(stream)
            ev["out_free"][b].record(dn)
        with torch.cuda.stream(up):
            dev_in[0].copy_(host_in, non_blocking=True)
            ev["in_ready"][0].record(up)
        for i in range(n):
            b, nb = i % 2, (i + 1) % 2
            if i + 1 < n:  # the next input uploads while this step computes
                up.wait_event(ev["in_free"][nb])
                with torch.cuda.stream(up):
                    dev_in[nb].copy_(host_in, non_blocking=True)
                    ev["in_ready"][nb].record(up)
            stream.wait_event(ev["in_ready"][b])
            ctx._check(set_all(ctx.h, C.c_void_p(dev_in[b].data_ptr()), 1), "set_all")
            ev["in_free"][b].record(stream)
            ctx.step_async(1)
            stream.wait_event(ev["out_free"][b])
            ctx._check(get_all(ctx.h, C.c_void_p(dev_out[b].data_ptr()), 1), "get_all")
            ev["out_ready"][b].record(stream)
            dn.wait_event(ev["out_ready"][b])
            with torch.cuda.stream(dn):
                outs[b].copy_(dev_out[b], non_blocking=True)
                ev["out_free"][b].record(dn)
        ctx.sync()  # device errors of the queued steps
        torch.cuda.synchronize()

    pipelined(2)
    t1 = time.perf_counter()
    pipelined(k)
    tp = time.perf_counter() - t1
    same = bool(torch.equal(outs[(k - 1) % 2], host_out))  # the same result as the serial path
    nbytes = host_in.numel() * host_in.element_size()
    cells = ctx.query(A.Q_CELL_UPDATES_PER_STEP)
    del ctx, dev_in, dev_out
    # the host link's own rate for these buffers: plain pinned copies of the
    # same bytes through the copy engine, timed with CUDA events
    dev = torch.empty_like(host_in, device="cuda")
    link = {}
    for name, dst, src in (("h2d_gbs", dev, host_in), ("d2h_gbs", host_out, dev)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        link[name] = 5 * nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9
    # both directions at once (an upload and a download on two streams)
    dev2 = torch.empty_like(host_in, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for _ in range(5):
        with torch.cuda.stream(s1):
            dev.copy_(host_in, non_blocking=True)
        with torch.cuda.stream(s2):
            host_out.copy_(dev2, non_blocking=True)
    torch.cuda.synchronize()
    link["both_ways_gbs_each"] = 5 * nbytes / (time.perf_counter() - t2) / 1e9
    del dev, dev2
    torch.cuda.empty_cache()
    link["pipelined_result_equals_serial"] = same
    return cells * k / tp, cells * k / t, nbytes, link


def queue_leg(steps=2, theta=0.1):
    """The deep clump hierarchy after one regrid, advanced through the device
    work queue with the coarser levels' tiles shared out by predicted work
    (balance 1) and in equal counts (balance 0): `steps` coarse steps each,
    CUDA events on the stream (the leg the idle-SM capture of the queue
    kernel runs)."""
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import inputs
    pb = inputs.clumps_3d()
    stream = torch.cuda.Stream()
    ctx = A.Context(A.make_config(3, pb.base, precision=A.MIXED, gamma=pb.gamma, cfl=pb.cfl), stream.cuda_stream)
    ctx.set_hierarchy(pb.patches)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    for f, a in enumerate(inputs.packed_clumps(pb)):
        ctx.set_field_packed(f, a)
    ctx.regrid(theta, pb.nlev)
    ctx.set_option(A.OPT_QUEUE, 1)
    out = {}
    for bal in (1, 0):
        ctx.set_option(A.OPT_QUEUE_BALANCE, bal)
        ctx.step(1, want_dt=False)
        ms, _ = timed_steps(ctx, stream, steps)
        out["balance_%d_ms_per_step" % bal] = ms / steps
    out["patches"] = ctx.query(A.Q_NPATCH)
    del ctx
    torch.cuda.empty_cache()
    return out


def deep_amr_leg(steps=20, regrid_every=2, theta=0.1):
    """The deep clump workload (3D, 32^3 base, 6 levels around 8 dense clumps):
    mixed precision, concurrent levels, autotuned tiles; a regrid every
    regrid_every coarse steps. Steps are timed with CUDA events on the
    launching stream; the regrid (clustering, map building and transfer on the
    device, the greedy merges of the block marks and the neighbour lists on the
    host) with the host clock."""
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import inputs
    pb = inputs.clumps_3d()
    stream = torch.cuda.Stream()
    ctx = A.Context(A.make_config(3, pb.base, precision=A.MIXED, gamma=pb.gamma, cfl=pb.cfl), stream.cuda_stream)
    ctx.set_hierarchy(pb.patches)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    for f, a in enumerate(inputs.packed_clumps(pb)):
        ctx.set_field_packed(f, a)
    ctx.regrid(theta, pb.nlev)
    tiles = ctx.autotune(3)
    ctx.step(1, want_dt=False)
    updates, leaves, t_steps, t_regrid, breakdown = 0, 0, 0.0, 0.0, [0, 0, 0, 0, 0, 0]
    nreg = 0
    for i in range(0, steps, regrid_every):
        k = min(regrid_every, steps - i)
        per = ctx.query(A.Q_CELL_UPDATES_PER_STEP)
        ms, _ = timed_steps(ctx, stream, k)
        t_steps += ms / 1e3
        updates += per * k
        leaves += leaf_updates(ctx.get_patches()) * k
        if i + k < steps:
            t0 = time.perf_counter()
            ctx.regrid(theta, pb.nlev)
            t_regrid += time.perf_counter() - t0
            nreg += 1
            for q in range(5):
                breakdown[q] += ctx.query(A.Q_REGRID_FLAG_US + q)
            breakdown[5] += ctx.query(A.Q_REGRID_TRANSFER_MAPS_US)
            ctx.autotune(2)
    # the final hierarchy in three schedules: finer levels on side streams (the
    # default), one stream in the recursive order, and the device work queue
    # (one persistent launch per finest sub-step, finest level first)
    ms_c, _ = timed_steps(ctx, stream, 2)
    ctx.set_option(A.OPT_CONCURRENT, 0)
    ctx.step(1, want_dt=False)
    ms_s, _ = timed_steps(ctx, stream, 2)
    ctx.set_option(A.OPT_CONCURRENT, 1)
    ctx.set_option(A.OPT_QUEUE, 1)
    ctx.step(1, want_dt=False)
    ms_q, _ = timed_steps(ctx, stream, 2)
    ctx.set_option(A.OPT_QUEUE_BALANCE, 0)
    ctx.step(1, want_dt=False)
    ms_q0, _ = timed_steps(ctx, stream, 2)
    ctx.set_option(A.OPT_QUEUE_BALANCE, 1)
    ctx.set_option(A.OPT_QUEUE, 0)
    cells = {}
    for (l, lo, hi) in ctx.get_patches():
        cells[l] = cells.get(l, 0) + (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    out = {"value": updates / t_steps, "unit": UNIT, "with_regrid": updates / (t_steps + t_regrid),
           "leaf_cell_updates_per_s": leaves / t_steps,
           "steps": steps, "regrid_every": regrid_every, "theta": theta, "regrids": nreg,
           "regrid_ms_mean": 1e3 * t_regrid / max(nreg, 1),
           "regrid_host_us_mean": {k: v / max(nreg, 1) for k, v in
                                   zip(("flag", "cluster", "build", "transfer", "build_maps", "transfer_maps"),
                                       breakdown)},
           "cells_per_level_final": [cells[l] for l in sorted(cells)], "patches_final": ctx.query(A.Q_NPATCH),
           "tiles": tiles, "tile_zchunk": launch_shapes(ctx), "concurrent_levels_speedup": ms_s / ms_c,
           "final_hierarchy_ms_per_step": {"side_streams": ms_c / 2, "serial": ms_s / 2, "device_queue": ms_q / 2,
                                           "device_queue_equal_shares": ms_q0 / 2},
           "workload": "clumps3d_32_6lev: 8 clumps rho 100 r 0.02, v (1,0,0), B (sqrt2,0,0); mixed precision"}
    del ctx
    torch.cuda.empty_cache()
    return out


def launch_shapes(ctx):
    """Per level, the fused advance's (tile variant, z planes per CTA) of its
    interior-only advance and of its advance with the extended ghost layers."""
    from paper_1110_1616_gb300 import amrmhd as A
    out = []
    for l in range(ctx.query(A.Q_NLEVEL)):
        out.append([list(ctx.tile_choice(l, 0)), list(ctx.tile_choice(l, 1)) if l > 0 else None])
    return out


def leaf_updates(patches, dim=3):
    """Cell updates per coarse step counting leaf cells only: per level, its
    cells minus those covered by the next level (each fine cell covers 2^-dim
    of a coarse cell), times 2^level."""
    cells = {}
    for (l, lo, hi) in patches:
        v = 1
        for d in range(dim):
            v *= hi[d] - lo[d]
        cells[l] = cells.get(l, 0) + v
    return sum((cells[l] - cells.get(l + 1, 0) // (1 << dim)) << l for l in cells)


def cylinder_leg(steps=20):
    """The paper's workload shape: an advected magnetized cylinder, 64^3 base in
    16^3 patches and one static refined level over 12.5 % of the volume, mixed
    precision, concurrent levels, autotuned tiles; coarse steps timed with CUDA
    events."""
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import inputs
    pb = inputs.cylinder_3d()
    ctx, stream = make_ctx(pb, A.MIXED)
    tiles = ctx.autotune(3)
    ctx.step(2, want_dt=False)
    per = ctx.query(A.Q_CELL_UPDATES_PER_STEP)
    ms, _ = timed_steps(ctx, stream, steps)
    leaf = leaf_updates(pb.patches)
    out = {"value": per * steps / (ms / 1e3), "unit": UNIT, "leaf_cell_updates_per_s": leaf * steps / (ms / 1e3),
           "ms_per_step": ms / steps, "steps": steps, "cell_updates_per_step": per, "tiles": tiles,
           "tile_zchunk": launch_shapes(ctx),
           "workload": "cylinder3d_64_2lev: magnetized cylinder (contrast 10, r 0.1) advected by v (1, 1/2, 0), "
                       "B (sqrt2,0,0), level 1 over 12.5 % of the volume; mixed precision"}
    del ctx
    torch.cuda.empty_cache()
    return out


def shock_clump_leg(steps=10, theta=0.1):
    """The shock-clump workload (3D, 64^3 base, 5 levels, Mach-10 shock into a
    lognormal fractal clump, inflow at x-low and outflow elsewhere), mixed
    precision: the state is generated per patch on the nested initial boxes,
    one regrid (theta) builds the flagged hierarchy (its host time reported),
    then `steps` coarse steps are timed with CUDA events."""
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import inputs
    pb = inputs.shock_clump_3d()
    fields = inputs.packed_shock_clump(pb)
    stream = torch.cuda.Stream()
    cfg = A.make_config(3, pb.base, precision=A.MIXED, gamma=pb.gamma, cfl=pb.cfl, bc=pb.bc, inflow=pb.inflow)
    ctx = A.Context(cfg, stream.cuda_stream)
    # floors of 1e-8 of the ambient density and pressure (both 1)
    ctx.set_floors(1e-8, 1e-8)
    ctx.set_hierarchy(pb.patches)
    ctx.alloc_arena()
    torch.cuda.synchronize()
    for f, a in enumerate(fields):
        ctx.set_field_packed(f, a)
    ctx.step(1, want_dt=False)
    t0 = time.perf_counter()
    ctx.regrid(theta, pb.nlev)
    t_regrid = time.perf_counter() - t0
    tiles = ctx.autotune(2)
    ctx.step(1, want_dt=False)
    per = ctx.query(A.Q_CELL_UPDATES_PER_STEP)
    ms, launches = timed_steps(ctx, stream, steps)
    cells = {}
    for (l, lo, hi) in ctx.get_patches():
        cells[l] = cells.get(l, 0) + (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
    out = {"value": per * steps / (ms / 1e3), "unit": UNIT,
           "leaf_cell_updates_per_s": leaf_updates(ctx.get_patches()) * steps / (ms / 1e3),
           "steps": steps, "ms_per_step": ms / steps,
           "cells_per_level": [cells[l] for l in sorted(cells)], "patches": ctx.query(A.Q_NPATCH),
           "arena_gb": ctx.query(A.Q_ARENA_BYTES) / 1e9, "regrid_s": t_regrid,
           "floors": {"rho": 1e-8, "p": 1e-8, "raises": ctx.query(A.Q_FLOOR_EVENTS)},
           "regrid_host_us": dict({k: ctx.query(A.Q_REGRID_FLAG_US + i)
                                   for i, k in enumerate(("flag", "cluster", "build", "transfer", "build_maps"))},
                                  transfer_maps=ctx.query(A.Q_REGRID_TRANSFER_MAPS_US)),
           "tiles": tiles, "tile_zchunk": launch_shapes(ctx),
           "workload": "shock_clump3d_64_5lev: Mach-10 shock into a lognormal (sigma 1, slope -11/3, contrast 10) "
                       "clump r 0.15; B (sqrt2,0,0); inflow x-low, outflow elsewhere; mixed precision"}
    del ctx
    torch.cuda.empty_cache()
    return out


def weak_scale_leg(steps=10, unit_sms=16):
    """The paper's weak-scaling experiment (Sec. 6: the advected magnetized
    cylinder with one refined level at 12.5 % filling, 64^3 base cells per
    processor) on SM partitions of one GPU: P = 1, 2, 4, 8 work units (unit
    cubes, each with its cylinder and refined level) advanced on a partition
    of P x unit_sms SMs (a green context, amrmhd_sm_partition_create), mixed
    precision, one stream, CUDA events on the partition's stream. Efficiency
    = time per coarse step at P = 1 / time at P (work and SMs both grow P-fold)."""
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import inputs
    out = {"unit": "64^3 base + refined central eighth (12.5 %)", "unit_sms": unit_sms, "runs": []}
    t1 = None
    for P, reps in ((1, (1, 1, 1)), (2, (2, 1, 1)), (4, (2, 2, 1)), (8, (2, 2, 2))):
        pb = inputs.cylinder_3d_tiled(reps, 64, 16)
        part = A.SmPartition(P * unit_sms)
        ext = torch.cuda.ExternalStream(part.stream)
        ctx = A.context_for(pb, precision=A.MIXED, stream=part.stream)
        ctx.set_option(A.OPT_CONCURRENT, 0)
        ctx.alloc_arena()
        torch.cuda.synchronize()
        ctx.load_state(pb.state)
        ctx.autotune(2)
        ctx.step(2, want_dt=False)
        per = ctx.query(A.Q_CELL_UPDATES_PER_STEP)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ext)
        ctx.step(steps, want_dt=False)
        e1.record(ext)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        t1 = ms if t1 is None else t1
        out["runs"].append({"units": P, "sms": part.sms, "ms_per_step": ms, "cell_updates_per_s": per / (ms / 1e3),
                            "per_sm": per / (ms / 1e3) / part.sms, "efficiency": t1 / ms})
        del ctx
        torch.cuda.synchronize()
        part.close()
        torch.cuda.empty_cache()
    return out


def adjoint_leg(steps=200, ckpt=20):
    """The adjoint workload (2D, 256^2 base in 32^2 patches + refined quadrant):
    forward amrmhd_step_dt and amrmhd_backward with checkpoints every ckpt
    coarse steps for a fixed dt sequence, FP64 and mixed precision, and the
    recorded pair (amrmhd_step_dt_ckpt, amrmhd_backward_recorded); the seed is
    the derivative of 0.5 sum (rho - rho_target)^2 over the level-0 cells with
    rho_target the final density of a second seed's forward run."""
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import inputs
    pb = inputs.adjoint_2d(seed=4)
    pt = inputs.adjoint_2d(seed=5)
    out = {"workload": "adjoint_2d_256_q: 256^2 base + refined quadrant, Alfven wave + smooth dv, %d steps, "
                       "checkpoint every %d" % (steps, ckpt)}
    for name, prec in (("fp64", A.FP64), ("mixed", A.MIXED)):
        stream = torch.cuda.Stream()
        ctx = A.context_for(pb, precision=prec, strict_fp64=False, stream=stream.cuda_stream)
        ctx.alloc_arena()
        torch.cuda.synchronize()
        ctx.load_state(pb.state)
        dts = [0.8 * ctx.cfl_dt()] * steps
        n0 = sum((hi[0] - lo[0]) * (hi[1] - lo[1]) for (l, lo, hi) in pb.patches if l == 0)
        tgt = A.context_for(pt, precision=prec, strict_fp64=False, stream=stream.cuda_stream)
        tgt.alloc_arena()
        torch.cuda.synchronize()
        tgt.load_state(pt.state)
        tgt.step_dt(dts)
        rho_t = tgt.get_field_packed(0)[:n0]
        del tgt
        import numpy as np
        u0 = torch.tensor(np.concatenate([ctx.pack(pb.state, f) for f in range(8)]), dtype=torch.float64,
                          device="cuda")
        ctx.step_dt(dts)  # warm-up: the context's first forward carries one-time costs
        ctx.load_packed_all(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.step_dt(dts)
        t_fwd = time.perf_counter() - t0
        uf = torch.empty_like(u0)
        ctx.read_packed_all(uf)
        torch.cuda.synchronize()
        g = torch.zeros_like(u0)
        g[:n0] = uf[:n0] - torch.tensor(rho_t, dtype=torch.float64, device="cuda")
        ctx.load_packed_all(u0)
        g0 = torch.empty_like(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.backward(dts, g, g0, ckpt)
        t_bwd = time.perf_counter() - t0
        per = pb.cells_per_coarse_step()
        # the recorded forward (checkpoints kept by the forward, as the autograd
        # path runs it) and its backward without a second forward pass
        ctx.load_packed_all(u0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.step_dt_ckpt(dts, ckpt)
        t_fwd_rec = time.perf_counter() - t0
        g0r = torch.empty_like(u0)
        t0 = time.perf_counter()
        ok = ctx.backward_recorded(g, g0r)
        t_bwd_rec = time.perf_counter() - t0
        assert ok
        # the configuration's control: the gradient with respect to the initial
        # velocity (rho, p and B held), from dL/dU0
        from paper_1110_1616_gb300.autograd import velocity_gradient
        gv = velocity_gradient(u0, g0, ctx.packed_size(0))
        out[name] = {"forward_cell_updates_per_s": per * steps / t_fwd, "forward_s": t_fwd, "backward_s": t_bwd,
                     "backward_over_forward": t_bwd / t_fwd, "grad_norm": float(g0.norm()),
                     "grad_v0_norm": float(gv.norm()),
                     "recorded": {"forward_s": t_fwd_rec, "backward_s": t_bwd_rec,
                                  "backward_over_forward": t_bwd_rec / t_fwd,
                                  "grad_max_rel_diff": float((g0 - g0r).abs().max() / g0.abs().max())}}
        del ctx
        torch.cuda.empty_cache()
    return out


def mixed_error_leg():
    """Relative L1 error per field of the mixed path against the strict FP64
    path (which matches the oracle to 1e-12), per config, with the same dt
    sequence: Orszag-Tang (config-1 hierarchy, 50 coarse steps), the 3D blast at
    64^3 (20 steps), the finite-amplitude Alfven wave (40 steps)."""
    import numpy as np
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import inputs
    names = ["rho", "mx", "my", "mz", "E", "bx", "by", "bz"]
    cases = [("orszag_tang_64_amr", inputs.orszag_tang(64, 16, refine=True, noise=1e-3, seed=1), 50),
             ("blast3d_64", inputs.blast_3d(64, 16), 20),
             ("alfven_2d_64_amp0.1", inputs.alfven_2d(64, 16, amp=1e-1), 40)]
    out = {}
    for name, pb, steps in cases:
        res = {}
        ref, dts = None, None
        for prec in (A.FP64, A.MIXED):
            stream = torch.cuda.Stream()
            ctx = A.context_for(pb, precision=prec, strict_fp64=True, stream=stream.cuda_stream)
            ctx.alloc_arena()
            torch.cuda.synchronize()
            ctx.load_state(pb.state)
            if dts is None:
                dts = list(ctx.step(steps))
            else:
                ctx.step_dt(dts)
            st = [ctx.get_field_packed(f) for f in range(8)]
            if ref is None:
                ref = st
            else:
                for f in range(8):
                    den = np.abs(ref[f]).sum()
                    res[names[f]] = float(np.abs(st[f] - ref[f]).sum() / den) if den > 0 else float(np.abs(st[f]).sum())
            del ctx
            torch.cuda.empty_cache()
        out[name] = res
    return out


def cpu_oracle_rate(pb, steps=1):
    from oracle import OracleSim
    s = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, gamma=pb.gamma, cfl=pb.cfl)
    s.set_state(pb.state)
    c0 = s.cell_updates()
    t0 = time.perf_counter()
    for _ in range(steps):
        s.step()
    t = time.perf_counter() - t0
    return (s.cell_updates() - c0) / t, t


def _oracle_one_step(n_psize):
    """One oracle coarse step of the n^3 blast in psize^3 patches, in a process
    of its own: (cell updates, seconds of the step)."""
    from paper_1110_1616_gb300 import inputs
    from oracle import OracleSim
    n, psize = n_psize
    pb = inputs.blast_3d(n, psize)
    s = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, gamma=pb.gamma, cfl=pb.cfl)
    s.set_state(pb.state)
    c0 = s.cell_updates()
    t0 = time.perf_counter()
    s.step()
    return s.cell_updates() - c0, time.perf_counter() - t0


def cpu_oracle_rate_all_cores(n, psize):
    """The oracle as it stands on every host core this process may use: one
    process per core (spawned, so none inherits the GPU context), each taking
    one coarse step of its own copy of the workload at once; the rate is the
    cell updates of all of them over the longest step."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_one_step, [(n, psize)] * cores)
    return sum(c for c, _ in res) / max(t for _, t in res), cores, max(t for _, t in res)


def run_reference(args, world, rank):
    """The oracle, as it stands, on the host cores: each step is one coarse step
    of a bounded sample of the workload (the same blast physics and 16^3 patches
    at 64^3 = 1/8 of the cells)."""
    if rank != 0:
        return
    from paper_1110_1616_gb300 import inputs
    from oracle import OracleSim
    n = max(args.n // 2, 32)
    pb = inputs.blast_3d(n, args.psize)
    s = OracleSim(pb.dim, pb.base, pb.patches, pb.nlev, gamma=pb.gamma, cfl=pb.cfl)
    s.set_state(pb.state)
    for _ in range(args.warmup):
        s.step()
    c0 = s.cell_updates()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step()
    t = time.perf_counter() - t0
    v = (s.cell_updates() - c0) / t
    sample = "blast %d^3 in %d^3 patches (1/%d of the %d^3 workload), %d coarse steps" % (
        n, args.psize, (args.n // n) ** 3, args.n, args.steps)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "blast3d_%d_p%d" % (args.n, args.psize), "global_batch": 1,
                       "cells": args.n ** 3, "patches": (args.n // args.psize) ** 3, "parallelism": "replicas" if world > 1 else "single"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args) if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    from paper_1110_1616_gb300 import amrmhd as A
    from paper_1110_1616_gb300 import build as B
    from paper_1110_1616_gb300 import inputs
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    barrier(world)
    if args.leg:
        kw = {} if args.leg_steps is None else {"steps": args.leg_steps}
        if args.leg == "adjoint" and args.leg_steps is not None:
            kw["ckpt"] = max(1, args.leg_steps // 2)
        fn = {"adjoint": adjoint_leg, "deep": deep_amr_leg, "shockclump": shock_clump_leg,
              "error": mixed_error_leg, "cylinder": cylinder_leg, "weakscale": weak_scale_leg,
              "queue": queue_leg}[args.leg]
        if rank == 0:
            print(json.dumps({"leg": args.leg, "result": fn(**kw) if args.leg != "error" else fn()}), flush=True)
        return
    pb = inputs.blast_3d(args.n, args.psize)
    cells_step = pb.cells_per_coarse_step()
    pk = peaks()
    hbm_peak = pk.get("hbm_gbs", 6800.0)

    ctx, stream = make_ctx(pb, A.MIXED)
    tile = ctx.autotune(3)[0]  # the library's autotuner picks the fused tile (state unchanged)
    clocks = Clocks(local)
    clocks.start()
    ctx.step(args.warmup, want_dt=False)
    torch.cuda.synchronize()
    barrier(world)
    ms, launches = timed_steps(ctx, stream, args.steps)
    clk = clocks.stop()
    value, ms_max = whole_job_rate(world, cells_step * args.steps, ms)

    # level advance alone, against the HBM roofline (algorithmic bytes: the 8
    # stored fields read and written once per cell update, 16 x 4 B in FP32)
    t_adv, t_fill = advance_alone(ctx, stream, 20)
    alg_bytes = 16 * 4 * cells_step
    achieved = alg_bytes / (t_adv / 1e3) / 1e9
    arena_gb = ctx.query(A.Q_ARENA_BYTES) / 1e9
    sm_max = pk.get("sm_max_mhz", 2070.0)
    # ALU peaks: derived from the unit counts and the clock, and measured by the
    # library's multiply-add probe (FP32 and FP64) on this device
    fp32_meas, sms = A.alu_peak(False)
    fp64_meas, _ = A.alu_peak(True)
    fp32_peak = sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    flops_achieved = FLOPS_PER_CELL_UPDATE_3D * cells_step / (t_adv / 1e3) / 1e12
    del ctx
    torch.cuda.empty_cache()

    extras = {"alu_peaks": {"fp32_tflops": fp32_meas / 1e12, "fp64_tflops": fp64_meas / 1e12, "sms": sms,
                            "how": "amrmhd_alu_peak: 8 independent multiply-add chains per thread, 8 x 256 "
                                   "threads per SM, best of 5 launches, CUDA events"}}
    if not args.skip_extras:
        # FP64: the staged kernels (the default) and the fused kernel (option 3)
        k64 = max(5, args.steps // 5)
        fp64 = {}
        for name, opt in (("staged", None), ("fused", 3)):
            ctx64, s64 = make_ctx(pb, A.FP64)
            if opt is not None:
                ctx64.set_option(A.OPT_ADVANCE, opt)
            ctx64.step(2, want_dt=False)
            ms64, _ = timed_steps(ctx64, s64, k64)
            rate = cells_step * k64 / (ms64 / 1e3)
            fp64[name] = {"value": rate, "unit": UNIT, "ms_per_step": ms64 / k64, "steps": k64,
                          "alu_frac_of_measured_fp64": FLOPS_PER_CELL_UPDATE_3D * rate / fp64_meas,
                          "hbm_frac": 16 * 8 * rate / 1e9 / hbm_peak}
            del ctx64
            torch.cuda.empty_cache()
        extras["fp64"] = dict(fp64["staged"], fused=fp64["fused"])

        ctxb, sb = make_ctx(pb, A.FP64, baseline=True, graph=False)
        ctxb.step(1, want_dt=False)
        kb = max(3, args.steps // 20)
        msb, _ = timed_steps(ctxb, sb, kb)
        vb = cells_step * kb / (msb / 1e3)
        extras["baseline_fp64_one_patch_per_launch"] = {"value": vb, "unit": UNIT, "ms_per_step": msb / kb,
                                                        "steps": kb}
        extras["speedup_vs_fp64_one_patch_per_launch"] = value / world / vb
        del ctxb
        torch.cuda.empty_cache()
        extras["mixed_rel_l1_vs_fp64"] = mixed_error_leg()
        extras["deep_amr_clumps3d"] = deep_amr_leg()
        extras["adjoint_2d"] = adjoint_leg()
        extras["shock_clump3d"] = shock_clump_leg()
        extras["cylinder3d_paper_shape"] = cylinder_leg()
        extras["weak_scaling_sm_partitions"] = weak_scale_leg()
    e2e = None
    if not args.skip_extras:
        ke = max(10, args.steps // 4)
        ve, vs, nbytes, link = e2e_run(pb, A.MIXED, ke)
        e2e = {"value": ve * world, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "how": "pipelined: step n+1's input uploads and step n-1's result downloads (pinned host "
                      "memory, double-buffered device staging, own streams) overlap step n's "
                      "amrmhd_set_state_all + amrmhd_step_async + amrmhd_get_state_all, amrmhd_sync at the end; "
                      "host clock over %d steps" % ke,
               "serial": {"value": vs * world, "how": "amrmhd_set/get_state_all on the pinned host buffers, "
                                                      "one step after the other"},
               "host_link_measured": link}
    cpu = None
    if rank == 0 and not args.skip_extras:
        rate, t = cpu_oracle_rate(pb, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "1 coarse step of the same %d^3 blast, single-threaded FP64 (%.1f s)" % (args.n, t)}
        rate_all, cores, t_all = cpu_oracle_rate_all_cores(args.n, args.psize)
        cpu["all_cores"] = {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "one process per host core, each 1 coarse step of its own copy of the "
                                      "%d^3 blast (FP64, the longest step %.1f s)" % (args.n, t_all)}
    barrier(world)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "blast3d_%d_p%d" % (args.n, args.psize), "global_batch": world,
                   "cells": args.n ** 3, "patches": (args.n // args.psize) ** 3, "precision": "mixed",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (arena %.2f GB: ping-pong state and stage scratch)" % arena_gb},
        "roofline": {"bound": "alu",
                     "kernel": "k_advance3d_fused<float,%s> (one launch per level advance, autotuned tile; "
                               "halo read from the neighbour patches)" % TILE_NAMES.get(tile, str(tile)),
                     "achieved": flops_achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": flops_achieved / fp32_peak,
                     "peak_kind": "derived: %d SMs x %d FP32 lanes x 2 x %.0f MHz" % (sms, FP32_LANES, sm_max),
                     "measured_peak": fp32_meas / 1e12, "frac_of_measured": flops_achieved / (fp32_meas / 1e12),
                     "traffic": FUSED_TRAFFIC_BYTES if args.n == 128 and args.psize == 16 and tile == 2 else None,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of "
                                       "this kernel on this workload (profiles/k_advance3d_fused_blast3d_128.md)",
                     "flops_per_cell_update": FLOPS_PER_CELL_UPDATE_3D,
                     "ms_per_launch": t_adv,
                     "fill_ms_per_launch": t_fill, "fill_in_step": False},
        "hbm": {"achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_kind": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in pk else "fallback",
                "alg_bytes_per_launch": alg_bytes},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
