#!/usr/bin/env python3
"""Throughput of the MUSCL-Hancock + Roe patch-group hydro step on GB300.

Workload (default): a uniform periodic level of 16^3 patch groups = 4096
groups, 256^3 cells, FP32, gamma = 5/3, rho = 1 + 0.1 * (8 seeded Fourier
modes, |k| <= 8), p = 1, smooth Gaussian velocity of rms 0.3 c_s; every step
advances all groups, each kernel CTA gathering its group's ghost zones from
the neighbours' interiors, and reduces the next shared dt in FP64.  Synthetic
data (seed 1007).

One step = hydro step (ghost gather fused in) + dt reduction over the level.
value = cells updated per second over the timed steps (max time over ranks;
each rank runs its own level: weak scaling).  e2e = the same groups through
the host-buffer pipeline entry point, host<->device copies included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--mode f32|mixed|f64]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell updates/s per GB300"
UNIT = "cell updates/s"
GAMMA = 5.0 / 3.0
CFL = 0.5
SEED = 1007
NCELLS = 256          # level edge in cells
GROUP_CELLS = 4096
# algorithmic HBM bytes of one group update by the fused level kernel: its
# 16^3x5 interior read once (neighbours' ghost cells are re-reads served by
# L2), 16^3x5 out and 6x5x16^2 face flux written (element size), dt, dh
# (8 B each), status (4 B), partials (48 B)
def group_bytes(esz):
    return (20480 + 20480 + 7680) * esz + 16 + 4 + 48


# DRAM traffic of one launch of the FP32 fused level kernel on this workload
# (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of
# `python -m paper_1007_3818_gb300.profile_case --path both --groups 16 16 16
# --ctas 3`), valid for the kernel sources it was taken on only: reported as
# null once any of them changes.
KERNEL_SOURCES = ["paper_1007_3818_gb300/csrc/hydro_kernel.cuh",
                  "paper_1007_3818_gb300/csrc/device_util.cuh",
                  "paper_1007_3818_gb300/csrc/hydro_launch.cuh",
                  "paper_1007_3818_gb300/csrc/hydro_f32.cu"]
NCU_TRAFFIC = {"mode": "f32", "groups": 4096, "ctas_per_sm": 3, "bytes": 773214976,
               "sources_sha256": "9d4da8196f69f2b3748d17d1bcca88c83b4643a291cec13dd3b28103a9e72ca6"}


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(mode, groups, ctas_per_sm):
    t = NCU_TRAFFIC
    if (mode, groups, ctas_per_sm) != (t["mode"], t["groups"], t["ctas_per_sm"]):
        return None
    try:
        return t["bytes"] if kernel_sources_sha256() == t["sources_sha256"] else None
    except OSError:
        return None


SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12  # 80.5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["f32", "mixed", "f64", "ff"], default="f32")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", choices=["uniform256", "streamed1024"], default="uniform256",
                    help="uniform256: device-resident 256^3 level (default); streamed1024: "
                         "1024^3 level in pinned host memory streamed through the GPU")
    ap.add_argument("--batch", type=int, default=32768,
                    help="streamed slab size in groups (a multiple of a 4096-group layer)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (every 200 ms) during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
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
        self.thread.join(timeout=5)
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------------
def make_level():
    from paper_1007_3818_gb300 import workloads as wl
    U = wl.fourier_level(n=NCELLS, seed=SEED, gamma=GAMMA)
    return wl.level_to_groups(U)  # float64 [4096][5][16][16][16]


def cpu_baseline(tiles_f64, seconds):
    """The FP64 oracle, as it stands, on this host's cores, over a bounded
    sample of the benchmark's groups; returns (cells/s, cores, sample text,
    algorithmic flops per cell from the oracle's counting scalar)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    dt, dh = 1e-3, 1.0 / NCELLS
    probe = tiles_f64[:cores]
    t0 = time.perf_counter()
    oracle.advance_groups(probe, dt, dh, gamma=GAMMA, nthreads=cores)
    t_probe = time.perf_counter() - t0
    # as many groups as the budget allows, repeated steps if the whole level is quicker
    n = int(min(len(tiles_f64), max(cores, cores * round(seconds / max(t_probe, 1e-3)))))
    reps = max(1, int(round(seconds / max(t_probe * n / cores, 1e-3))))
    sample = tiles_f64[:n]
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.advance_groups(sample, dt, dh, gamma=GAMMA, nthreads=cores)
    el = time.perf_counter() - t0
    counts = oracle.count_ops_group(tiles_f64[0], dt, dh, gamma=GAMMA)
    flops = (counts["add"] + counts["mul"] + counts["div"] + counts["sqrt"]) / counts["cells"]
    return n * GROUP_CELLS * reps / el, cores, \
        f"{n} of the {len(tiles_f64)} groups x {reps} step(s), {el:.1f} s on {cores} threads " \
        f"(OpenMP over groups)", flops


def reference_arm(args):
    """--impl reference: the oracle timed on the host cores on this workload."""
    rank, world, _ = __import__("paper_1007_3818_gb300.dist", fromlist=["x"]).env_world()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    level = make_level()
    tiles = oracle.fill_ghosts_uniform(level, 16, 16, 16, 0)
    if args.mode != "f64":
        tiles = tiles.astype(np.float32).astype(np.float64)
    cores = os.cpu_count() or 1
    oracle.build()
    # size one step's sample so the whole run takes a few minutes at most
    t0 = time.perf_counter()
    oracle.advance_groups(tiles[:cores], 1e-3, 1.0 / NCELLS, gamma=GAMMA, nthreads=cores)
    t1 = time.perf_counter() - t0
    budget = 150.0 / max(1, args.steps + args.warmup)
    n = int(min(len(tiles), max(cores, cores * int(budget / max(t1, 1e-3)))))
    sample = tiles[:n]
    for _ in range(args.warmup):
        oracle.advance_groups(sample, 1e-3, 1.0 / NCELLS, gamma=GAMMA, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.advance_groups(sample, 1e-3, 1.0 / NCELLS, gamma=GAMMA, nthreads=cores)
    el = time.perf_counter() - t0
    v = n * GROUP_CELLS * args.steps / el
    desc = f"{n} of the 4096 groups per step, {cores} threads (OpenMP over groups)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "uniform periodic level, 4096 patch groups (256^3 cells), "
                               "Fourier-mode density, gamma 5/3", "mode": args.mode},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


# --------------------------------------------------------------------------
def streamed_main(args):
    """1024^3 level (262,144 groups) in pinned host memory; every step streams
    z-slabs of the interiors to a device copy of the level, where the ghost
    zones are gathered, and the results back, on three streams, one step's
    copies overlapping the next one's (gamer_pipeline_level_run_host)."""
    import numpy as np
    import torch
    from paper_1007_3818_gb300 import native
    from paper_1007_3818_gb300 import workloads as wl
    torch.cuda.set_device(0)
    mode = {"f32": native.GAMER_MODE_F32, "mixed": native.GAMER_MODE_MIXED,
            "f64": native.GAMER_MODE_F64, "ff": native.GAMER_MODE_FF}[args.mode]
    T = torch.float64 if mode == native.GAMER_MODE_F64 else torch.float32
    base = wl.level_to_groups(wl.lognormal_base(256, SEED + 2, gamma=GAMMA,
                                                sigma_ln=np.log(1e4) / 8, clip=4.0, vel_rms=1.0))
    gx = 64
    G = gx ** 3
    gid = np.arange(G)
    src = (((gid // (gx * gx)) % 16) * 16 + ((gid // gx) % gx) % 16) * 16 + (gid % gx) % 16
    lv = [torch.empty((G, 5, 16, 16, 16), dtype=T, pin_memory=True) for _ in range(2)]
    torch.index_select(torch.from_numpy(base).to(T), 0, torch.from_numpy(src), out=lv[0])
    part = torch.zeros((G, 6), dtype=torch.float64, pin_memory=True)
    st = torch.zeros(G, dtype=torch.int32, pin_memory=True)
    dh = 1.0 / 1024
    params = native.make_params(GAMMA, cfl=CFL)
    pl = native.Pipeline(mode, args.batch, with_flux=False)
    pl.set_timeout(600.0)
    pl.set_level_mode(2)   # slab windows for the partials of U^0 (no device copy held)
    pl.level_step_host(lv[0], lv[1], gx, gx, gx, 0, 0.0, dh, st, part, params)
    dt0 = CFL * dh / float(part[:, 0].max())              # FP64 reduction of the partials
    dts = torch.zeros(args.steps, dtype=torch.float64, pin_memory=True)
    # the clock sampler starts before the allocating call, so that its own
    # start-up is over before the timed region
    clocks = ClockSampler(0)
    clocks.start()
    pl.level_run_host(lv[0], lv[1], gx, gx, gx, 0, 1, dt0, dh, CFL, params)  # allocation
    time.sleep(1.0)
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("streamed level run")
    pl.level_run_host(lv[0], lv[1], gx, gx, gx, 0, args.steps, dt0, dh, CFL, params, dts, st,
                      part)
    torch.cuda.nvtx.range_pop()
    el = time.perf_counter() - t0
    clk = clocks.stop()
    h2d, d2h = pl.last_bytes()
    h2d, d2h = h2d // args.steps, d2h // args.steps
    pl.close()
    cells = G * GROUP_CELLS
    v = cells * args.steps / el
    print(json.dumps({
        "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": 1, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.mode, "data": "synthetic",
        "config": {"workload": "streamed 1024^3 level: 262,144 patch groups in pinned host "
                               "memory, advanced by gamer_pipeline_level_run_host: every step "
                               "copies the interiors in and the new state out in z-slabs "
                               "through a device copy of the level, ghost gather on the device, "
                               "the next step's copies in overlapping this step's copies out, "
                               "dt from the previous step's partials on the device; lognormal "
                               "density contrast 1e4, gamma 5/3",
                   "slab_groups": args.batch},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clk, "status_or": int(np.bitwise_or.reduce(st.numpy())),
    }), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.workload == "streamed1024":
        return streamed_main(args)
    import numpy as np
    import torch
    from paper_1007_3818_gb300 import dist, native

    rank, world, local = dist.env_world()
    torch.cuda.set_device(local)
    dist.init("nccl")
    dev = torch.device("cuda", local)
    rc = native.gamer_device_check()
    if rc != 0:
        raise SystemExit(f"device check failed: {native.strerror(rc)}")
    mode = {"f32": native.GAMER_MODE_F32, "mixed": native.GAMER_MODE_MIXED,
            "f64": native.GAMER_MODE_F64, "ff": native.GAMER_MODE_FF}[args.mode]
    T = torch.float64 if mode == native.GAMER_MODE_F64 else torch.float32
    esz = 8 if T == torch.float64 else 4
    gx = gy = gz = NCELLS // 16
    G = gx * gy * gz
    dh = 1.0 / NCELLS
    params = native.make_params(GAMMA, cfl=CFL)

    level_h = make_level()
    level_a = torch.from_numpy(level_h).to(dev, T)
    level_b = torch.empty_like(level_a)
    tiles = torch.empty((G, 5, 20, 20, 20), device=dev, dtype=T)
    ff = torch.empty((G, 6, 5, 16, 16), device=dev, dtype=T)
    dt_g = torch.zeros(G, device=dev, dtype=torch.float64)
    dh_g = torch.full((G,), dh, device=dev, dtype=torch.float64)
    status = torch.zeros(G, device=dev, dtype=torch.int32)
    partials = torch.zeros((G, 6), device=dev, dtype=torch.float64)
    dh_level = torch.tensor([dh], device=dev, dtype=torch.float64)
    dt_level = torch.zeros(1, device=dev, dtype=torch.float64)
    totals = torch.zeros(5, device=dev, dtype=torch.float64)
    ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(G, 1), device=dev, dtype=torch.uint8)
    fill = (native.gamer_fill_ghosts_uniform_f64 if T == torch.float64
            else native.gamer_fill_ghosts_uniform_f32)
    stream = torch.cuda.current_stream(dev)

    # initial dt: a zero-length step gives the partials of the initial state
    fill(level_a, tiles, gx, gy, gz, 0)
    native.hydro_advance(mode, tiles, level_b, None, dt_g, dh_g, None, partials, params)
    native.gamer_hydro_dt(partials, None, dh_level, CFL, dt_level, totals, dt_g, ws)
    torch.cuda.synchronize()
    tiles_host0 = tiles.double().cpu().numpy() if (rank == 0 and not args.no_cpu_baseline) else None
    tot0 = totals.cpu().numpy().copy()

    # autotuned launch shape (register/smem variant and CTAs per SM) on this batch
    from paper_1007_3818_gb300 import tune
    tuned = tune.tune_hydro(mode, tiles, level_b, ff, dt_g, dh_g, status, partials, params)
    tuned_level = tune.tune_hydro_level(mode, level_a, level_b, ff, gx, gy, gz, 0, dt_g, dh_g,
                                        status, partials, params)

    cur, nxt = [level_a, level_b], 0
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def step(i=None):
        # one level step: hydro step with the ghost gather fused in, then the
        # FP64 dt / conservation reduction that feeds the next step's dt
        nonlocal nxt
        src, dst = cur[nxt], cur[1 - nxt]
        torch.cuda.nvtx.range_push("level step")
        if i is not None:
            ev_a[i].record(stream)
        native.hydro_advance_level(mode, src, dst, ff, gx, gy, gz, 0, dt_g, dh_g, status,
                                   partials, params)
        if i is not None:
            ev_b[i].record(stream)
        native.gamer_hydro_dt(partials, None, dh_level, CFL, dt_level, totals, dt_g, ws)
        torch.cuda.nvtx.range_pop()
        nxt = 1 - nxt

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    el_local = e0.elapsed_time(e1) / 1e3
    el = dist.max_over_ranks(el_local, device=dev)
    adv_ms = statistics.mean(ev_a[i].elapsed_time(ev_b[i]) for i in range(args.steps))
    st = status.cpu().numpy()
    tot = totals.cpu().numpy()
    cells_per_step = G * GROUP_CELLS
    value = world * cells_per_step * args.steps / el

    # CUDA-graph replay of the same step (A -> B, B -> A alternating)
    graphs = [native.LevelGraph(mode, cur[0], cur[1], None, ff, dt_g, dh_g, status, partials,
                                gx, gy, gz, 0, params, dh_level, dt_level, totals, ws),
              native.LevelGraph(mode, cur[1], cur[0], None, ff, dt_g, dh_g, status, partials,
                                gx, gy, gz, 0, params, dh_level, dt_level, totals, ws)]
    nsteps_done = args.warmup + args.steps  # parity of the buffer holding the state
    gi = nsteps_done % 2
    for _ in range(4):
        graphs[gi].launch(stream)
        gi ^= 1
    torch.cuda.synchronize()
    dist.barrier()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(args.steps):
        graphs[gi].launch(stream)
        gi ^= 1
    g1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    el_graph = dist.max_over_ranks(g0.elapsed_time(g1) / 1e3, device=dev)
    for g in graphs:
        g.close()

    # end to end: the same level held in pinned HOST memory, advanced through
    # the public multi-step call (gamer_pipeline_level_run_host): every step
    # copies the level's interiors in and the new state out (z-slabs through a
    # device copy of the level, ghost zones gathered on the device), the next
    # step's copies in overlapping this step's copies out; the dt of each step
    # after the first is the FP64 CFL reduction of the previous step's
    # partials on the device (the first from the partials of U^0)
    e2e = None
    if not args.no_e2e:
        h_lv = [torch.from_numpy(level_h).to(T).pin_memory(),
                torch.empty((G, 5, 16, 16, 16), dtype=T).pin_memory()]
        h_st = torch.empty(G, dtype=torch.int32).pin_memory()
        h_part = torch.empty((G, 6), dtype=torch.float64).pin_memory()
        h_dt = torch.empty(max(args.steps, 50), dtype=torch.float64).pin_memory()
        pre = native.Pipeline(mode, G, with_flux=False)
        pre.level_step_host(h_lv[0], h_lv[1], gx, gy, gz, 0, 0.0, dh, h_st, h_part, params)
        pre.close()
        dt0 = CFL * dh / float(h_part[:, 0].max())
        timing = {}
        for batch in (256, 512, 1024, 2048):             # slabs of 1, 2, 4, 8 layers
            pl = native.Pipeline(mode, batch, with_flux=False)
            pl.level_run_host(h_lv[0], h_lv[1], gx, gy, gz, 0, 2, dt0, dh, CFL, params)
            t0 = time.perf_counter()
            pl.level_run_host(h_lv[0], h_lv[1], gx, gy, gz, 0, 4, dt0, dh, CFL, params)
            timing[batch] = time.perf_counter() - t0
            pl.close()
        batch = min(timing, key=timing.get)
        pipe = native.Pipeline(mode, batch, with_flux=False)
        pipe.level_run_host(h_lv[0], h_lv[1], gx, gy, gz, 0, 2, dt0, dh, CFL, params)
        n_e2e = max(3, min(args.steps, 50))
        dist.barrier()
        t0 = time.perf_counter()
        pipe.level_run_host(h_lv[0], h_lv[1], gx, gy, gz, 0, n_e2e, dt0, dh, CFL, params,
                            h_dt[:n_e2e], h_st, h_part)
        el_e2e = dist.max_over_ranks(time.perf_counter() - t0, device=dev)
        h2d, d2h = pipe.last_bytes()
        pipe.close()
        e2e = {"value": world * cells_per_step * n_e2e / el_e2e, "unit": UNIT,
               "h2d_bytes_per_step": h2d // n_e2e, "d2h_bytes_per_step": d2h // n_e2e,
               "steps": n_e2e, "slab_groups": batch,
               "api": "gamer_pipeline_level_run_host (%d steps of the pinned host level in one "
                      "call; each step copies the interiors in and the new state out in z-slabs "
                      "of %d layers through a device copy of the level, ghost gather on the "
                      "device, the next step's copies in overlapping this step's copies out; "
                      "dt per step from the previous step's partials on the device; status and "
                      "last partials back at the end)" % (n_e2e, batch // (gx * gy))}

    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6702.2)
    adv_s = adv_ms / 1e3
    cpu = None
    flops_per_cell = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        v, cores, desc, flops_per_cell = cpu_baseline(tiles_host0, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    roofline = None
    traffic = measured_traffic(args.mode, G, tuned_level["ctas_per_sm"])
    roofline_hbm = {
        "bound": "hbm", "achieved": G * group_bytes(esz) / adv_s / 1e9, "peak": hbm_peak,
        "unit": "GB/s", "frac": G * group_bytes(esz) / adv_s / 1e9 / hbm_peak,
        "traffic": traffic, "algorithmic_bytes": G * group_bytes(esz),
        "note": "algorithmic bytes of the fused hydro kernel (level in, state and face "
                "fluxes out) vs measured HBM copy"}
    if flops_per_cell is not None:
        ach = flops_per_cell * cells_per_step / adv_s / 1e12
        roofline = {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS, "traffic": traffic,
                    "kernel": "hydro_step_kernel", "flops_per_cell": flops_per_cell,
                    "peak_basis": "152 SM x 128 FP32 lanes x 2 flop x 2070 MHz"}
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"f32": "f32", "mixed": "f32+f64", "f64": "f64", "ff": "f32"}[args.mode],
            "data": "synthetic",
            "config": {"workload": "uniform periodic level, 4096 patch groups of 16^3 cells "
                                   "(256^3), MUSCL-Hancock/Roe step with the ghost gather "
                                   "fused in + FP64 dt reduction per step",
                       "mode": args.mode, "groups": G, "cells_per_step": cells_per_step,
                       "gamma": GAMMA, "cfl": CFL, "seed": SEED,
                       "l2": "inputs larger than L2 (level %.0f MB read, %.0f MB written "
                             "per step)" % (G * 20480 * esz / 1e6, G * 28160 * esz / 1e6),
                       "parallelism": f"{world} independent levels (weak scaling)"},
            "roofline": roofline, "roofline_hbm": roofline_hbm, "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clk,
            "gpu_launches": 4 * args.steps,
            "kernel_ms": {"hydro_step": adv_ms},
            "tuned": {"ctas_per_sm": tuned_level["ctas_per_sm"],
                      "variant": tuned_level["variant"], "candidates_ms": tuned_level["all"],
                      "tiles_kernel": {"ctas_per_sm": tuned["ctas_per_sm"],
                                       "variant": tuned["variant"],
                                       "candidates_ms": tuned["all"]}},
            "graph": {"ms_per_step": el_graph / args.steps * 1e3,
                      "value": world * cells_per_step * args.steps / el_graph},
            "status_or": int(np.bitwise_or.reduce(st)),
            "conservation_rel": [float(abs(a - b) / max(abs(b), 1e-300))
                                 for a, b in zip(tot, tot0)],
        }
        print(json.dumps(out), flush=True)
    dist.finalize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
