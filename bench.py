#!/usr/bin/env python3
"""Benchmark of the Minimod acoustic-isotropic step on GB300.

Workload (one shot): 512^3 grid, 8-layer velocity model drawn from a seed,
20-cell Cerjan sponge, 20 Hz Ricker source at a seeded cell, 64 receivers
on the first plane below the top sponge, FP32, 1000 steps.  A benchmark
"step" is one leapfrog step of the whole grid through the fused kernel
(stencil, sponge, source, receivers, FP64 norm partials; every 25 steps the
norm reduction).  The metric is Gpoint-updates per second.

  value      device-resident: K timed steps of a shot whose model is already
             in HBM, CUDA events on the launching stream, per-launch events
             around every step kernel for the roofline.
  e2e        the same metric through the C ABI with host buffers: domain
             creation, velocity model from pinned host memory, source,
             receivers, K steps (graph-replayed chunks) and the traces back
             to pinned host memory, all inside the timed region.
  roofline   the step kernel's algorithmic 16 B per point (read u_n, read
             u_{n-1}, write u_{n+1}, read coef) per launch / its average
             launch time, against the measured HBM copy bandwidth.
  cpu_baseline  the FP64 oracle as it stands on the host cores, on a
             bounded slab of the same workload.

--impl reference times that oracle (the only reference implementation of
this method; the paper ships no code) on the same workload, one bounded
slab per step.  With N > 1 (torchrun) every rank runs an independent
replica on its own GPU ("replicas only": the path has no data exchange
between GPUs); value = all ranks' point-updates / the slowest rank's time.
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
sys.path.insert(0, ROOT)

N_GRID = 512
ALG_BYTES_PER_POINT = 16          # FP32 3-level: u_n, u_{n-1}, coef in; u_{n+1} out
METRIC = "stencil Gpts/s & % HBM roofline, FP32 vs BF16/FP16-store; shot p50/p99 latency"
UNIT = "Gpts/s"
# the step kernel and the work-item planning that decides what one launch
# reads (tiles, planes per item, schedule): a DRAM-traffic record taken on
# other sources no longer describes the kernel
KERNEL_SOURCES = ["paper_2506_02486_gb300/csrc/stencil.cuh",
                  "paper_2506_02486_gb300/csrc/stencil_inst.cu",
                  "paper_2506_02486_gb300/csrc/stencil_dispatch.cpp",
                  "paper_2506_02486_gb300/csrc/ptx.cuh",
                  "paper_2506_02486_gb300/csrc/gw_device.h",
                  "paper_2506_02486_gb300/csrc/domain.cpp"]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peak() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_peak_tensor() -> tuple[float, str]:
    """Dense BF16 TFLOP/s (cuBLAS burst) measured on this machine's GPUs."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def recorded_traffic() -> float | None:
    """Per-launch DRAM bytes of the step kernel from the committed ncu
    summary, if it was taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic_step_kernel.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("kernel_hash") != kernel_hash():
        return None
    return float(rec["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}",
                 f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend=None):
    """One process per GPU (torchrun env): replicas of the whole workload,
    joined only by a host-side barrier and a max-over-ranks of the timing
    (no collective on the data path).  NCCL on GPU machines, gloo otherwise."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
        else:
            dist.init_process_group("gloo")
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def replica_rate(pg, world: int, units_per_rank: float, ms: float):
    """(slowest rank's ms, whole-job rate in units per second): every rank
    processed units_per_rank; the job took as long as its slowest rank."""
    ms_max = max_over_ranks(pg, ms)
    return ms_max, world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------------ oracle

def _oracle_slab(shot, nthreads: int, target_s: float):
    """A z-slab of the workload around the source sized so that one oracle
    step over it takes about target_s (calibrated on 8 planes)."""
    import oracle
    oracle.build()
    n = N_GRID
    dt = oracle.time_step(shot.h, float(shot.vel.max()))
    z0 = max(0, shot.src[2] - 4)
    probe = np.ascontiguousarray(shot.vel[z0:z0 + 8])
    oracle.run(probe, shot.h, 1, dt=dt, nthreads=nthreads)       # page in
    t = time.perf_counter()
    oracle.run(probe, shot.h, 3, dt=dt, nthreads=nthreads)
    per_pt_step = (time.perf_counter() - t) / 3 / probe.size
    nz = int(max(8, min(n, target_s / (per_pt_step * n * n))))
    z0 = max(0, min(n - nz, shot.src[2] - nz // 2))
    slab = np.ascontiguousarray(shot.vel[z0:z0 + nz])
    src = (shot.src[0], shot.src[1], shot.src[2] - z0)
    return slab, src, dt, per_pt_step


def cpu_oracle_rate(shot, target_s: float, nthreads: int) -> tuple[float, str]:
    """Oracle Gpts/s on a slab of the workload: one run of several steps
    (set-up included once), sized to ~target_s."""
    import oracle
    slab, src, dt, per = _oracle_slab(shot, nthreads, target_s / 8)
    steps = int(max(2, min(2000, round(target_s / (per * slab.size)))))
    t = time.perf_counter()
    oracle.run(slab, shot.h, steps, dt=dt, src=src, f_peak=shot.f_peak,
               sponge=shot.sponge, nthreads=nthreads)
    el = time.perf_counter() - t
    n = N_GRID
    return (slab.size * steps / el / 1e9,
            f"{n}x{n}x{slab.shape[0]} slab of the 512^3 layered model, one oracle run "
            f"of {steps} steps, {el:.1f} s, {nthreads} thread(s)")


def bench_config(shot) -> dict:
    """The workload both arms report (launch details of our kernel are in
    the line's `launch` object, not here)."""
    n = N_GRID
    return {"workload": "layered_512cubed", "grid": [n, n, n],
            "model": "8 layers, velocities U[1500, 4500] m/s, seed 2506",
            "sponge": shot.sponge, "source_hz": shot.f_peak,
            "receivers": int(shot.receivers.shape[0]),
            "l2": "inputs larger than L2: 3 fields x 571 MB streamed per step"}


def run_reference(args, world, rank, pg):
    """The FP64 oracle, as it stands, on the host cores.  One call runs the
    warm-up and the K timed steps (the state stays inside it); a second
    call runs the warm-up steps alone.  Both pay the same set-up (arrays,
    coefficients, sponge tables), so K steps over the difference of the two
    times is the oracle's stepping rate.  The grid is a z-slab of the 512^3
    workload around the source, the whole grid when K steps of it take
    under a minute."""
    import workloads
    if rank != 0:
        return 0
    import oracle
    shot = workloads.layered_cube(N_GRID)
    cores = os.cpu_count() or 1
    slab, src, dt, _ = _oracle_slab(shot, cores, 60.0 / max(1, args.steps))

    def timed(k):
        t = time.perf_counter()
        oracle.run(slab, shot.h, k, dt=dt, src=src, f_peak=shot.f_peak,
                   sponge=shot.sponge, nthreads=cores)
        return time.perf_counter() - t

    t_all = timed(args.warmup + args.steps)
    t_warm = timed(args.warmup)
    el = max(t_all - t_warm, 1e-9)
    value = slab.size * args.steps / el / 1e9
    n = N_GRID
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / max(1, args.steps) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": bench_config(shot),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                         "kind": "oracle",
                         "sample": f"{n}x{n}x{slab.shape[0]} slab of the 512^3 layered "
                                   f"model: one call of {args.warmup}+{args.steps} steps "
                                   f"({t_all:.1f} s) minus one of {args.warmup} "
                                   f"({t_warm:.1f} s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours

def seg_bytes(nx, ny, nz, dtype, px=1, py=1, pz=1):
    from paper_2506_02486_gb300.runtime import padded_bytes
    nsub = px * py * pz
    sub = padded_bytes(-(-nx // px), -(-ny // py), -(-nz // pz), dtype)
    return nsub * (4 * sub + (320 << 20))


def run_shot_device(seg, shot, steps, warmup, dtype="f32", px=1, py=1, pz=1,
                    timing=True, stream=None, sampler=None, halo_mode=0,
                    timing_steps=None, tile=0):
    """Device-resident timing; returns (elapsed_ms, kernel_stats, info,
    clocks, norms).  The wall time covers `steps` steps launched as the
    library does by default (graph-replayed chunks); kernel statistics come
    from a separate pass of per-launch CUDA events (timing_steps, default
    min(steps, 100)).  The clock sampler, if any, runs from the warm-up to
    the end of the timed steps."""
    import torch
    from paper_2506_02486_gb300 import gbwave as gw
    from paper_2506_02486_gb300.runtime import Shot
    n = N_GRID
    tsteps = (timing_steps or min(steps, 100)) if timing else 0
    with Shot(seg, n, n, n, px=px, py=py, pz=pz,
              nsteps=steps + warmup + tsteps, dtype=dtype,
              sponge=shot.sponge, halo_mode=halo_mode, tile=tile) as s:
        s.set_model(shot.vel)
        s.add_ricker(shot.src, shot.f_peak)
        s.set_receivers(shot.receivers)
        st = stream or torch.cuda.current_stream()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        s.step(warmup, st)
        gw.gw_barrier(s.dom, st, True)
        stats = None
        if timing:
            gw.gw_kernel_timing(s.dom, True)
            gw.gw_kernel_stats_get(s.dom)        # reset
            s.step(tsteps, st)
            gw.gw_barrier(s.dom, st, True)
            stats = gw.gw_kernel_stats_get(s.dom)
            gw.gw_kernel_timing(s.dom, False)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        s.step(steps, st)
        e1.record(st)
        torch.cuda.synchronize()
        clocks = sampler.stop() if sampler else None
        ms = e0.elapsed_time(e1)
        info = s.info
        norms = s.norms(min(steps + warmup, 50))
    return ms, stats, info, clocks, norms


def run_e2e(seg, shot, steps):
    """The user's call sequence with host buffers, timed end to end."""
    import torch
    from paper_2506_02486_gb300 import gbwave as gw
    n = N_GRID
    # the workload's velocity model is FP32: it goes in through the FP32 call
    vel_pinned = torch.empty(shot.vel.shape, dtype=torch.float32,
                             pin_memory=True)
    vel_pinned.numpy()[...] = shot.vel
    traces = torch.empty((shot.receivers.shape[0], steps), dtype=torch.float32,
                         pin_memory=True)
    rec = np.ascontiguousarray(shot.receivers, dtype=np.int32)
    torch.cuda.synchronize()
    t = time.perf_counter()
    desc = gw.shot_desc(n, n, n, nsteps=steps, sponge=shot.sponge)
    dom = gw.gw_domain_create(seg.ctx, desc)
    try:
        gw.gw_set_model_f32(dom, vel_pinned.numpy())
        gw.gw_inject_ricker(dom, *shot.src, shot.f_peak)
        gw.gw_set_receivers(dom, rec)
        gw.gw_step(dom, steps, torch.cuda.current_stream())
        gw.gw_read_receivers(dom, rec.shape[0], steps, out=traces.numpy())
    finally:
        gw.gw_domain_destroy(dom)
    el = time.perf_counter() - t
    h2d = vel_pinned.numel() * 4 + rec.nbytes
    d2h = traces.numel() * 4
    return el, h2d, d2h


BATCH_SEED = 2508
BATCH_STEPS = 300
BATCH_CHUNK = 25


def run_batch(dtype="f32", *, seed=BATCH_SEED, steps=BATCH_STEPS,
              chunk=BATCH_CHUNK, autotune=True, persistent=False,
              sequential=False, warmup=BATCH_CHUNK, tile=0, margin=0.0,
              tiles_by="plan"):
    """64 independent cubic shots (sides drawn from {96..256} step 16, each
    with its own layered model and source, 20-cell sponge, 20 Hz) advanced
    together: tiles per grid side from the autotuner, one launch per tile
    group per step with the groups side by side, K-step chunks replayed
    from one CUDA graph (or, persistent, one cooperative launch per group
    per chunk).  Returns a dict of aggregate Gpts/s and the schedule."""
    import torch
    import workloads
    from paper_2506_02486_gb300 import gbwave as gw
    from paper_2506_02486_gb300.runtime import Batch, Segment, Shot, shot_bytes
    plan = workloads.batch_shots(seed, n=64, nsteps=steps)
    total = sum(shot_bytes(b.side, b.side, b.side, dtype, steps + warmup, 16)
                for b in plan)
    pts = sum(b.side ** 3 for b in plan)
    out = {"shots": len(plan), "points": pts, "steps": steps, "chunk": chunk,
           "seed": seed, "dtype": dtype, "persistent": persistent}
    with Segment(total + (2 << 30)) as seg:
        tiles = {}
        t0 = time.perf_counter()
        if autotune and tiles_by == "model":
            for b in plan:
                tiles[b.side] = gw.gw_pick_tile(dtype, b.side, b.side)
        elif autotune:
            descs = [gw.shot_desc(b.side, b.side, b.side, nsteps=steps,
                                  dtype=dtype, sponge=b.sponge) for b in plan]
            for b, t in zip(plan, gw.gw_plan_tiles(seg.ctx, descs, 20, margin)):
                tiles[b.side] = t
        out["autotune_s"] = time.perf_counter() - t0
        out["tiles"] = {str(k): v for k, v in tiles.items()}
        shots = []
        try:
            for b in plan:
                s = Shot(seg, b.side, b.side, b.side, nsteps=steps + warmup,
                         dtype=dtype, sponge=b.sponge,
                         tile=tiles.get(b.side, tile))
                shots.append(s)
                s.set_model(b.model())
                s.add_ricker(b.source, 20.0)
                s.set_receivers(workloads.lattice_receivers(
                    b.side, b.side, b.sponge, n=4, margin=b.sponge))
            st = torch.cuda.current_stream()
            if sequential:
                # the same shots one after the other, each its own launches
                for s in shots:
                    s.step(warmup, st)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                for s in shots:
                    s.step(steps, st)
                e1.record(st)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
            else:
                with Batch(seg, shots, chunk=chunk,
                           persistent=persistent) as bt:
                    out.update(bt.info)
                    bt.step(warmup, st)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    bt.step(steps, st)
                    e1.record(st)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1)
            out["ms"] = ms
            out["gpts"] = pts * steps / (ms * 1e-3) / 1e9
            out["check_norm2"] = [float(shots[i].check()[0]) for i in (0, -1)]
        finally:
            for s in shots:
                s.close()
    return out


def _variant_line(npts, vms, vs, vstats, bpp):
    kavg = vstats["total_ms"] / max(1, vstats["launches"])
    return {
        "gpts": npts * vs / (vms * 1e-3) / 1e9,
        "kernel_ms": kavg,
        "halo_kernel_ms": vstats["halo_ms"] / max(1, vstats["launches"]),
        "alg_bytes_per_point": bpp,
        "roofline_frac": bpp * npts / (kavg * 1e-3) / 1e9 / measured_peak()[0],
        "steps": vs,
    }


def run_ours(args, world, rank, local, pg):
    import torch
    import workloads
    from paper_2506_02486_gb300 import buildlib
    from paper_2506_02486_gb300.runtime import Segment

    buildlib.build()
    torch.cuda.set_device(local)
    shot = workloads.layered_cube(N_GRID)
    n = N_GRID
    npts = n ** 3
    seg1 = Segment(seg_bytes(n, n, n, "f32"), nranks=1, device=local)
    try:
        sampler = ClockSampler(local) if rank == 0 else None
        barrier(pg)
        # per-launch timing over >= 1500 steps (~0.6 s), so that the clock
        # samples of the window see the kernel under load
        ms, stats, info, clocks, norms = run_shot_device(
            seg1, shot, args.steps, args.warmup, sampler=sampler,
            timing_steps=max(args.steps, 1500))
        ms_max, rate = replica_rate(pg, world, npts * args.steps, ms)
        value = rate / 1e9
        # e2e through the public API with host buffers
        barrier(pg)
        # the median of three runs of the whole call sequence (one run can
        # meet a stall of the host), after one untimed run (the first use of
        # the FP32 model path's kernels in the process loads them)
        run_e2e(seg1, shot, args.steps)
        e2e_runs = []
        for _ in range(3):
            e2e_s, h2d, d2h = run_e2e(seg1, shot, args.steps)
            e2e_runs.append(e2e_s)
        e2e_s = max_over_ranks(pg, statistics.median(e2e_runs))
        e2e_value = world * npts * args.steps / e2e_s / 1e9
        variants = {}
        if args.variants:
            vs = max(100, args.steps // 5)
            for name, kw in (("f16s_delta", dict(dtype="f16s")),
                             ("bf16_delta", dict(dtype="bf16"))):
                vms, vstats, _, _, _ = run_shot_device(seg1, shot, vs, args.warmup, **kw)
                variants[name] = _variant_line(npts, vms, vs, vstats, 10)
    finally:
        seg1.close()
    if args.variants:
        # decompositions inside one HBM: 2 x 2 x 2 cubes and the paper's
        # 1-D x slabs (Listing 1), halos put by the step kernel or copied by
        # a separate kernel after it
        from paper_2506_02486_gb300 import gbwave as gw
        for dec in ((2, 2, 2), (8, 1, 1)):
            tag = "x".join(map(str, dec))
            with Segment(seg_bytes(n, n, n, "f32", *dec), nranks=8, device=local) as seg:
                for mode, hm in (("fused_halo", 0), ("separate_halo", 1)):
                    # the kernel tile the library's autotuner picks for the
                    # subdomain shape
                    tile, _ = gw.gw_autotune(
                        seg.ctx, gw.shot_desc(n, n, n, nsteps=16, sponge=shot.sponge,
                                              halo_mode=hm), *dec, steps=6)
                    vms, vstats, vinfo, _, _ = run_shot_device(
                        seg, shot, vs, args.warmup, px=dec[0], py=dec[1], pz=dec[2],
                        halo_mode=hm, tile=tile)
                    variants[f"f32_{tag}_{mode}"] = dict(
                        _variant_line(npts, vms, vs, vstats, 16), tile=vinfo["tile"])
        variants[f"cannon_{CANNON_N}_p{CANNON_P}"] = run_cannon(device=local)
        variants[f"f32_{MINIMOD_N}cubed"] = run_minimod_size(device=local)
        for dt in ("f32", "bf16"):
            # persistent: one tile for every shot (the autotuner's best
            # uniform choice), so that one cooperative launch per 25-step
            # chunk advances all 64 shots
            for suffix, kw in (("", {}), ("_persistent", dict(persistent=True, margin=1.0))):
                r = run_batch(dt, **kw)
                variants[f"batch64_{dt}{suffix}"] = {
                    k: r[k] for k in ("gpts", "ms", "steps", "chunk",
                                      "points", "groups", "ctas", "seed",
                                      "autotune_s", "persistent")}
    precision = None
    if args.variants and args.precision_check:
        precision = precision_results(500, device=local)
    serving = None
    if args.serving and args.variants:
        # the serving stream (2000 Poisson requests, real time, ~2.5 min) at
        # 0.7 of the 64-shot FP32 batch throughput measured above: p50/p99
        # latency beside the throughput numbers
        srv = run_serve(args.serve_requests, device=local,
                        capacity_gpts=variants["batch64_f32"]["gpts"])
        serving = {k: srv[k] for k in (
            "requests", "rate_per_s", "offered_load", "capacity_gpts_assumed",
            "failed", "p50_latency_s", "p99_latency_s", "aggregate_gpts",
            "busy_gpts", "makespan_s", "max_active", "budget_bytes")}
    if rank != 0:
        return 0
    peak, peak_kind = measured_peak()
    kavg_ms = stats["total_ms"] / max(1, stats["launches"])
    achieved = ALG_BYTES_PER_POINT * npts / (kavg_ms * 1e-3) / 1e9
    traffic = recorded_traffic()
    cpu = None
    cores = os.cpu_count() or 1
    if args.cpu_baseline:
        rate, sample = cpu_oracle_rate(shot, 20.0, cores)
        rate1, sample1 = cpu_oracle_rate(shot, 8.0, 1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": sample,
               "one_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": sample1}}
    # the timed region: one step kernel per step, one norm reduction per
    # 25-step chunk
    gpu_launches = args.steps + -(-args.steps // 25)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": bench_config(shot),
        "launch": {
            "decomposition": "1x1x1", "halo": "fused",
            "parallelism": f"replicas{world}",
            "tile": info["tile"], "ctas": info["ctas"], "items": info["items"],
            "timing": "CUDA events on the launching stream; roofline from "
                      "per-launch events over a separate pass of "
                      f"{max(args.steps, 1500)} steps",
        },
        "roofline": {
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_kind": peak_kind,
            "alg_bytes_per_launch": ALG_BYTES_PER_POINT * npts,
            "alg_bytes_per_point": ALG_BYTES_PER_POINT,
            "dram_bytes_per_point": (traffic / npts) if traffic else None,
            "kernel_ms": kavg_ms,
        },
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": d2h / args.steps,
                "scope": "domain create + set_model_f32 (pinned FP32 model) + "
                         "source + receivers + K graph-chunked steps + traces D2H; "
                         "median of 3 runs after one untimed run",
                "runs_ms": [round(t * 1e3, 3) for t in e2e_runs]},
        "gpu_launches": gpu_launches,
        "clocks": clocks,
        "variants": variants,
        "precision": precision,
        "serving": serving,
        "kernel_hash": kernel_hash(),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


SERVE_SEED = 2509
SERVE_BUDGET = 150 << 30
SERVE_LOAD = 0.7


def run_serve(n=2000, *, seed=SERVE_SEED, load=SERVE_LOAD, slots=64,
              budget=SERVE_BUDGET, chunk=BATCH_CHUNK, device=0,
              capacity_gpts=None):
    """Replay a Poisson stream of shot requests in real time through the
    continuous-batching server; latency is arrival -> traces on the host.
    The arrival rate is set so that the offered work is `load` times the
    batched FP32 capacity (capacity_gpts: measured in the same run, else
    measured here first)."""
    import torch
    import workloads
    from paper_2506_02486_gb300.runtime import Segment, Server
    if capacity_gpts is None:
        capacity_gpts = run_batch("f32")["gpts"]
    reqs = workloads.arrival_stream(seed, n=n, rate_per_s=1.0)
    work = [r.nx * r.ny * r.nz * r.nsteps for r in reqs]
    lam = load * capacity_gpts * 1e9 / (sum(work) / len(work))
    # same draws, rescaled inter-arrival times
    arrivals = [r.arrival_s / lam for r in reqs]
    torch.cuda.empty_cache()          # earlier segments' blocks
    seg = Segment(budget + (8 << 30), device=device)
    try:
        srv = Server(seg, budget, max_slots=slots, chunk=chunk)
        try:
            tickets = []
            t0 = time.perf_counter()
            s0 = srv.now()
            for r, a in zip(reqs, arrivals):
                wait = a - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                vz = workloads.layered_profile(r.nz, r.model_seed)
                rec = workloads.lattice_receivers(r.nx, r.ny, r.sponge, n=8,
                                                  margin=r.sponge)
                tickets.append(srv.submit(
                    r.nx, r.ny, r.nz, r.nsteps, src=r.source, f_peak=20.0,
                    vz=vz, receivers=rec, dtype=r.dtype, sponge=r.sponge))
            results = [srv.wait(t) for t in tickets]
            st = srv.stats()
        finally:
            srv.close()
    finally:
        seg.close()
    bad = [r["status"] for r in results if r["status"] != 0]
    lat = np.array([r["done_s"] - r["submit_s"] for r in results])
    qwait = np.array([r["admit_s"] - r["submit_s"] for r in results])
    t_first = min(r["submit_s"] for r in results)
    t_last = max(r["done_s"] for r in results)
    pu = sum(r["points"] * r["steps"] for r in results)
    by_dtype = {}
    for q, r in zip(reqs, results):
        by_dtype.setdefault(q.dtype, []).append(r["done_s"] - r["submit_s"])
    return {
        "requests": n, "seed": seed, "rate_per_s": lam, "offered_load": load,
        "capacity_gpts_assumed": capacity_gpts,
        "budget_bytes": budget, "slots": slots, "chunk": chunk,
        "failed": len(bad),
        "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(lat.mean()),
        "p99_queue_wait_s": float(np.percentile(qwait, 99)),
        "latency_by_dtype_p50_s": {k: float(np.percentile(v, 50))
                                   for k, v in by_dtype.items()},
        "makespan_s": t_last - t_first,
        "aggregate_gpts": pu / (t_last - t_first) / 1e9,
        "busy_gpts": st["point_updates"] / max(st["busy_s"], 1e-9) / 1e9,
        "point_updates": pu,
        "max_active": st["max_active"], "chunks": st["chunks"],
        "rebuilds": st["rebuilds"], "peak_bytes": st["peak_bytes"],
    }


CANNON_N, CANNON_P = 30240, 4     # the paper's matrix size; 4 ring ranks
MINIMOD_N = 1200                  # the paper's Minimod grid (section 4.5)


def run_minimod_size(steps=100, warmup=5, seed=2506, device=0):
    """FP32 Gpts/s on the paper's own Minimod grid, 1200^3 (8-layer model
    set per plane, 20-cell sponge, 20 Hz source, 64 receivers): fields
    3 x 7 GB, device-resident, per-launch CUDA events, kernel tile chosen
    by the library's autotuner for this shape."""
    import torch
    import workloads
    from paper_2506_02486_gb300 import gbwave as gw
    from paper_2506_02486_gb300.runtime import Segment, Shot
    n = MINIMOD_N
    vz = workloads.layered_profile(n, seed)
    src = workloads.source_position(seed + 1, n, n, n, margin=20)
    rec = workloads.lattice_receivers(n, n, 20, n=8, margin=20)
    with Segment(seg_bytes(n, n, n, "f32"), device=device) as seg:
        t0 = time.perf_counter()
        tile, _, times = gw.gw_autotune(
            seg.ctx, gw.shot_desc(n, n, n, nsteps=16, sponge=20), steps=6,
            all_times=True)
        tune_s = time.perf_counter() - t0
        with Shot(seg, n, n, n, nsteps=steps + warmup, sponge=20, tile=tile) as s:
            gw.gw_set_model_layered(s.dom, vz)
            s.add_ricker(src, 20.0)
            s.set_receivers(rec)
            st = torch.cuda.current_stream()
            s.step(warmup, st)
            gw.gw_barrier(s.dom, st, True)
            gw.gw_kernel_timing(s.dom, True)
            gw.gw_kernel_stats_get(s.dom)
            s.step(steps, st)
            gw.gw_barrier(s.dom, st, True)
            k = gw.gw_kernel_stats_get(s.dom)
            gw.gw_kernel_timing(s.dom, False)
            info = s.info
    kms = k["total_ms"] / max(1, k["launches"])
    npts = n ** 3
    return {"grid": [n, n, n], "steps": steps, "gpts": npts / (kms * 1e-3) / 1e9,
            "kernel_ms": kms, "alg_bytes_per_point": ALG_BYTES_PER_POINT,
            "roofline_frac": ALG_BYTES_PER_POINT * npts / (kms * 1e-3) / 1e9 /
                             measured_peak()[0],
            "tile": info["tile"], "items": info["items"],
            "autotune_ms_per_tile": times, "autotune_s": tune_s}


def run_cannon(n=CANNON_N, p=CANNON_P, runs=3, tile_m=256, group=4,
               seed=2506, device=0):
    """Cannon's ring exchange (section 5) on dyadic BF16 inputs: TFLOP/s of
    whole runs (P ring steps each, puts overlapped) and of the block-product
    kernel alone (per-launch CUDA events in a separate run)."""
    import torch
    from paper_2506_02486_gb300 import gbwave as gw
    from paper_2506_02486_gb300.runtime import Segment
    from workloads import matmul as mm
    a_bits = mm.dyadic_bits(mm.dyadic_codes(n, n, seed))
    bt_bits = mm.dyadic_bits(mm.dyadic_codes(n, n, seed + 1))
    per = gw.gw_cannon_bytes(n, p)
    flops = 2.0 * n ** 3
    with Segment(p * (per + (1 << 20)), nranks=p, device=device) as seg:
        cn = gw.gw_cannon_create(seg.ctx, n, p)
        try:
            gw.gw_cannon_schedule(cn, tile_m, group)
            gw.gw_cannon_set(cn, a_bits, bt_bits)
            del a_bits, bt_bits
            st = torch.cuda.current_stream()
            gw.gw_cannon_run(cn, st)                  # warm-up
            gw.gw_cannon_sync(cn)
            gw.gw_cannon_timing(cn, True)
            gw.gw_cannon_run(cn, st)
            gw.gw_cannon_sync(cn)
            k = gw.gw_cannon_stats(cn)
            gw.gw_cannon_timing(cn, False)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(runs):
                gw.gw_cannon_run(cn, st)
            e1.record(st)
            gw.gw_cannon_sync(cn)
            ms = e0.elapsed_time(e1) / runs
            pool = gw.gw_pool_stats_get(seg.ctx)
        finally:
            gw.gw_cannon_destroy(cn)
    peak = measured_peak_tensor()
    kms = k["gemm_ms"] / max(1, k["launches"])
    kflops = flops / p                            # one ring step
    return {
        "n": n, "p": p, "tile_m": tile_m, "group": group, "runs": runs,
        "inputs": "dyadic bf16",
        "ms_per_run": ms, "tflops": flops / (ms * 1e-3) / 1e12,
        "kernel_ms": kms, "kernel_launches_per_run": p, "grid": k["grid"],
        "roofline": {"bound": "tensor", "achieved": kflops / (kms * 1e-3) / 1e12,
                     "peak": peak[0], "peak_kind": peak[1], "unit": "TFLOP/s",
                     "frac": kflops / (kms * 1e-3) / 1e12 / peak[0]},
        "puts_per_run": p * (p - 1),
        "pool_peak_active": pool["peak_active"],
    }


def run_batch_modes(args):
    """The 64-shot workload under each schedule, one JSON line each."""
    import torch
    from paper_2506_02486_gb300 import buildlib
    buildlib.build()
    torch.cuda.set_device(0)
    for dt in ("f32", "bf16"):
        for name, kw in (("batch_graphs_tuned_side_by_side", {}),
                         ("batch_persistent_tuned", dict(persistent=True)),
                         ("batch_persistent_uniform_tile", dict(persistent=True, margin=1.0)),
                         ("batch_graphs_uniform_tile", dict(margin=1.0)),
                         ("batch_graphs_tile_model", dict(tiles_by="model")),
                         ("batch_graphs_default_tile", dict(autotune=False)),
                         ("sequential_shots_tuned", dict(sequential=True))):
            r = run_batch(dt, **kw)
            r["schedule"] = name
            print(json.dumps(r), flush=True)
    return 0


def run_case(args):
    """One plain shot of an N^3 layered model (no timing extras): the
    workload the ncu captures profile.  --split PX,PY,PZ decomposes it into
    subdomains with halos put by the step kernel (--halo fused) or copied by
    the separate kernel (--halo separate)."""
    import workloads
    from paper_2506_02486_gb300 import buildlib
    from paper_2506_02486_gb300.runtime import Segment, Shot
    buildlib.build()
    n = args.case
    px, py, pz = (int(v) for v in args.split.split(","))
    shot = workloads.layered_cube(n)
    with Segment(seg_bytes(n, n, n, args.dtype, px, py, pz), nranks=px * py * pz) as seg:
        with Shot(seg, n, n, n, px=px, py=py, pz=pz, nsteps=args.steps,
                  sponge=shot.sponge, dtype=args.dtype, chunk=-1, tile=args.tile,
                  halo_mode=0 if args.halo == "fused" else 1) as s:
            s.set_model(shot.vel)
            s.add_ricker(shot.src, shot.f_peak)
            s.set_receivers(shot.receivers)
            s.step(args.steps)
            s.sync()
            info = s.info
    print(json.dumps({"case": n, "dtype": args.dtype, "steps": args.steps,
                      "split": [px, py, pz], "halo": args.halo,
                      "tile": info["tile"], "ctas": info["ctas"],
                      "items": info["items"]}), flush=True)
    return 0


def precision_results(steps=500, device=0):
    """Storage types on the 1024 x 1024 x 512 perturbed layered model:
    Gpts/s of each and its error against the FP64 GPU path (whose agreement
    with the oracle is pinned on a 128^3 crop by the tests), the same run of
    `steps` steps for every type."""
    import torch
    import workloads
    from paper_2506_02486_gb300 import gbwave as gw
    from paper_2506_02486_gb300.runtime import Segment, Shot, padded_bytes
    shot = workloads.perturbed_box()
    nz, ny, nx = shot.vel.shape
    # receivers on the source plane: within reach of the wave after 500
    # steps (the z = 20 lattice is ~250 cells away and records nothing)
    rec = workloads.lattice_receivers(nx, ny, int(shot.src[2]), n=16,
                                      margin=shot.sponge)
    npts = nx * ny * nz
    vel32 = np.ascontiguousarray(shot.vel, dtype=np.float32)
    res, ref = {}, None
    for dt in ("f64", "f32", "f16s", "bf16"):
        nf = 4 if dt in ("f16s", "bf16") else 3
        with Segment(nf * padded_bytes(nx, ny, nz, dt) + (1 << 30), device=device) as seg:
            with Shot(seg, nx, ny, nz, nsteps=steps, dtype=dt,
                      sponge=shot.sponge) as s:
                gw.gw_set_model_f32(s.dom, vel32)
                s.add_ricker(shot.src, shot.f_peak)
                s.set_receivers(rec)
                s.sync()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                s.step(steps)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                u = s.u(f64=True)
                tr = s.traces(steps).astype(np.float64)
                info = s.info
        r = {"gpts": npts * steps / (ms * 1e-3) / 1e9, "ms": ms,
             "scale_u": info["scale_u"]}
        if ref is None:
            ref = (u, tr)
        else:
            d = u - ref[0]
            r["rel_l2"] = float(np.linalg.norm(d) / np.linalg.norm(ref[0]))
            r["max_abs"] = float(np.abs(d).max())
            r["traces_rel_l2"] = float(np.linalg.norm(tr - ref[1]) /
                                       np.linalg.norm(ref[1]))
        res[dt] = r
        del u
    res["max_abs_u"] = float(np.abs(ref[0]).max())
    for dt in ("f16s", "bf16"):
        res[dt]["speedup_vs_f32"] = res[dt]["gpts"] / res["f32"]["gpts"]
    return {"workload": shot.name, "grid": [nx, ny, nz], "steps": steps,
            "sponge": shot.sponge, "reference": "FP64 GPU path",
            "results": res}


def run_precision(args):
    from paper_2506_02486_gb300 import buildlib
    buildlib.build()
    steps = args.steps if args.steps != 1000 else 500
    print(json.dumps({"precision": precision_results(steps)}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=25)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-variants", dest="variants", action="store_false")
    ap.add_argument("--no-serving", dest="serving", action="store_false",
                    help="skip the serving replay of the default run")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the default run's serving replay")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline",
                    action="store_false")
    ap.add_argument("--no-precision", dest="precision_check", action="store_false",
                    help="skip the storage-type errors of the default run")
    ap.add_argument("--case", type=int, default=0,
                    help="run one plain N^3 shot for --steps steps (profiling)")
    ap.add_argument("--dtype", default="f32", help="storage type for --case")
    ap.add_argument("--tile", type=int, default=0, help="kernel tile for --case")
    ap.add_argument("--split", default="1,1,1", help="subdomains PX,PY,PZ for --case")
    ap.add_argument("--halo", choices=["fused", "separate"], default="fused",
                    help="halo mode of a decomposed --case")
    ap.add_argument("--precision", action="store_true",
                    help="storage types vs FP64 on the 1024x1024x512 model")
    ap.add_argument("--serve", type=int, default=0, metavar="N",
                    help="replay N Poisson shot requests through the server")
    ap.add_argument("--batch", action="store_true",
                    help="64-shot batched workload: schedules compared")
    ap.add_argument("--cannon", type=int, default=0, metavar="N",
                    help="Cannon ring-exchange product of two N x N matrices")
    ap.add_argument("--cannon-p", type=int, default=CANNON_P, help="ring ranks")
    ap.add_argument("--cannon-tile-m", type=int, default=256,
                    help="rows of a CTA's output tile (128 or 256)")
    ap.add_argument("--cannon-group", type=int, default=4,
                    help="tile rows per raster group")
    args = ap.parse_args()
    if args.cannon:
        from paper_2506_02486_gb300 import buildlib
        buildlib.build()
        print(json.dumps({"cannon": run_cannon(args.cannon, args.cannon_p,
                                               runs=max(1, args.steps if args.steps != 1000 else 3),
                                               tile_m=args.cannon_tile_m,
                                               group=args.cannon_group)}), flush=True)
        return 0
    if args.batch:
        return run_batch_modes(args)
    if args.serve:
        from paper_2506_02486_gb300 import buildlib
        buildlib.build()
        print(json.dumps({"serving": run_serve(args.serve)}), flush=True)
        return 0
    if args.case:
        return run_case(args)
    if args.precision:
        return run_precision(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; no GPU, no collective
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        return run_reference(args, world, rank, None)
    world, rank, local, pg = dist_setup()
    try:
        return run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
