#!/usr/bin/env python3
"""Throughput of the MUSCL-Hancock + Roe patch-group hydro step on GB300.

Headline workload (default; the largest configuration that fits one GPU): a
periodic 1024^3 level, 64^3 = 262,144 patch groups of 16^3 cells, FP32,
gamma 5/3, lognormal density of contrast 1e4 (ln rho = sigma clip(g, -4, 4),
sigma = ln(1e4)/8, on a periodic 256^3 field that the level repeats 4 times
per axis), p = rho^gamma / gamma, smooth Gaussian velocities of rms 1 c_s.
Synthetic data, seed 1007.  One step = the hydro step of every group, each
CTA gathering its group's ghost zones from the neighbours' interiors, then
the FP64 dt reduction that sets the next step's dt.

  value  cells updated per second, the level resident in HBM when the timed
         region starts (CUDA events; max over ranks; each rank its own level:
         weak scaling);
  e2e    the same level held in pinned HOST memory and advanced through the
         public multi-step call gamer_pipeline_level_run_host: every step
         copies the interiors in and the new state out.

Sub-records (rank 0, one GPU): per_config.uniform256 (config 2: 4,096 groups,
roofline, CPU baseline, CUDA-graph replay, e2e), per_config.amr54000 (config
4: 54,000 tiles of three levels through the captured batch graph), modes (f32,
mixed, ff, f64 on the 256^3 level: kernel time, roofline fraction, and the
rel-L1 error against the FP64 oracle on the precision-study problems).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--mode f32|mixed|ff|f64] [--workload level1024|uniform256]
                  [--no-extras] [--no-cpu-baseline] [--no-e2e]
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
GROUP_CELLS = 4096
MODES = {"f32": 0, "mixed": 1, "f64": 2, "ff": 3}
DTYPE = {"f32": "f32", "mixed": "f32+f64", "f64": "f64", "ff": "f32"}


# algorithmic HBM bytes of one group update by the fused level kernel: its
# 16^3x5 interior read once (neighbours' ghost cells are re-reads served by
# L2), 16^3x5 out and 6x5x16^2 face flux written (element size), dt, dh
# (8 B each), status (4 B), partials (48 B)
def group_bytes(esz, with_flux=True):
    return (20480 + 20480 + (7680 if with_flux else 0)) * esz + 16 + 4 + 48


# DRAM traffic of one launch of the FP32 fused level kernel (dram__bytes_read.sum
# + dram__bytes_write.sum, one ncu capture of `python -m
# paper_1007_3818_gb300.profile_case --path level --groups 16 16 16`, 4,096
# groups), valid for the kernel sources it was taken on only: reported as null
# once any of them changes.  Traffic grows with the groups processed, so a
# launch over G groups is reported as bytes * G / groups.
KERNEL_SOURCES = ["paper_1007_3818_gb300/csrc/hydro_kernel.cuh",
                  "paper_1007_3818_gb300/csrc/device_util.cuh",
                  "paper_1007_3818_gb300/csrc/hydro_launch.cuh",
                  "paper_1007_3818_gb300/csrc/hydro_f32.cu"]
NCU_TRAFFIC = {"mode": "f32", "groups": 4096, "bytes": 360896768 + 417231360,
               "sources_sha256": "3cdb04ec70a56c5ce37fa636b4849cd318902bc1956cef420fb89a67427163b6"}


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(mode, groups):
    t = NCU_TRAFFIC
    if mode != t["mode"] or t["bytes"] is None:
        return None
    try:
        if kernel_sources_sha256() != t["sources_sha256"]:
            return None
    except OSError:
        return None
    return t["bytes"] * groups / t["groups"]


FP32_LANES_PER_SM = 128      # FP32 FMA lanes per SM (Blackwell)
FP64_FMA_PER_SM_CLK = 2      # GB300: 1.25 TFLOP/s nominal FP64 = 152 SM x 2 FMA x 2 x ~2.06 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=list(MODES), default="f32")
    ap.add_argument("--workload", choices=["level1024", "uniform256"], default="level1024",
                    help="level1024: the 262,144-group 1024^3 level (default); uniform256: the "
                         "4,096-group 256^3 level as the headline (quicker)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of each oracle baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: no per-config, mode or precision sub-records")
    ap.add_argument("--host-alloc", choices=["library", "torch"], default="library",
                    help="host levels of the end-to-end legs from gamer_host_alloc (huge-page "
                         "backed, default) or from torch's pinned allocator")
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


def alu_peaks(dev, clk):
    """FP32 and FP64 peaks (TFLOP/s) from this device's SM count and the SM
    clock nvidia-smi reported as maximum during the run (2070 MHz if none)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    med = (clk or {}).get("sm_mhz") or mhz
    f32 = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    f64 = sms * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e12
    basis = f"{sms} SM x {{}} x 2 flop x {mhz:.0f} MHz (clocks.max.sm)"
    return {"f32": f32, "f64": f64, "sms": sms, "mhz": mhz,
            "f32_at_median_clock": f32 * med / mhz, "f64_at_median_clock": f64 * med / mhz,
            "basis_f32": basis.format(f"{FP32_LANES_PER_SM} FP32 lanes"),
            "basis_f64": basis.format(f"{FP64_FMA_PER_SM_CLK} FP64 FMA units")}


# --------------------------------------------------------------------------
# workloads (seeded, synthetic; generators in paper_1007_3818_gb300/workloads.py)
def level1024_base():
    """Config 5 field: the periodic 256^3 lognormal base (4,096 groups) that
    the 1024^3 level repeats 4 x 4 x 4 times."""
    import numpy as np
    from paper_1007_3818_gb300 import workloads as wl
    return wl.level_to_groups(wl.lognormal_base(256, SEED + 2, gamma=GAMMA,
                                                sigma_ln=np.log(1e4) / 8, clip=4.0, vel_rms=1.0))


def tiled_sources(gx, gb):
    """Group g of a gx^3 level that repeats a periodic gb^3-group field: the
    field's group index of g."""
    import numpy as np
    gid = np.arange(gx ** 3)
    bx, by, bz = gid % gx, (gid // gx) % gx, gid // (gx * gx)
    return ((bz % gb) * gb + (by % gb)) * gb + (bx % gb)


def periodic_tiles(groups, gx, out=None):
    """The 20^3 ghost-padded input of every group of a periodic gx^3-group
    level (the level's own cells, wrapped), sliced group by group out of the
    padded level -- plain indexing, independent of the CUDA path.  `out`
    (reused between steps) avoids faulting in a new array every time."""
    import numpy as np
    from paper_1007_3818_gb300 import workloads as wl
    box = wl.groups_to_level(groups, gx, gx, gx)                        # [5][n][n][n]
    pad = np.pad(box, ((0, 0), (2, 2), (2, 2), (2, 2)), mode="wrap")
    if out is None:
        out = np.empty((gx ** 3, 5, 20, 20, 20), dtype=groups.dtype)
    for g in range(gx ** 3):
        bz, by, bx = g // (gx * gx), (g // gx) % gx, g % gx
        out[g] = pad[:, 16 * bz:16 * bz + 20, 16 * by:16 * by + 20, 16 * bx:16 * bx + 20]
    return out


def uniform256_level():
    from paper_1007_3818_gb300 import workloads as wl
    return wl.level_to_groups(wl.fourier_level(n=256, seed=SEED, gamma=GAMMA))


# --------------------------------------------------------------------------
# CPU baseline leg: the FP64 oracle, as it stands, on this host's cores.
# Besides the timed samples it runs the precision-study problems whose states
# serve as the reference of the modes' rel-L1 figures.
def oracle_rate(tiles_f64, dt, dh, seconds):
    """Oracle throughput on a bounded sample of the given tiles: (cells/s,
    cores, sample text)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.build()
    probe = tiles_f64[:4 * cores]
    oracle.advance_groups(probe[:cores], dt, dh, gamma=GAMMA, nthreads=cores)  # first-call costs
    t0 = time.perf_counter()
    oracle.advance_groups(probe, dt, dh, gamma=GAMMA, nthreads=cores, want_flux=True)
    t_probe = (time.perf_counter() - t0) / 4   # one group per core
    n = int(min(len(tiles_f64), max(cores, cores * round(seconds / max(t_probe, 1e-3)))))
    reps = max(1, int(round(seconds / max(t_probe * n / cores, 1e-3))))
    sample = tiles_f64[:n]
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.advance_groups(sample, dt, dh, gamma=GAMMA, nthreads=cores, want_flux=True)
    el = time.perf_counter() - t0
    return n * GROUP_CELLS * reps / el, cores, \
        f"{n} groups x {reps} step(s), {el:.1f} s on {cores} threads (OpenMP over groups)"


def oracle_flops_per_cell(tile_f64, dt, dh):
    import oracle
    c = oracle.count_ops_group(tile_f64, dt, dh, gamma=GAMMA)
    return (c["add"] + c["mul"] + c["div"] + c["sqrt"]) / c["cells"]


def oracle_precision_reference(problem, n, steps, cfl):
    """The oracle's run of a precision-study problem (periodic box, its own
    dt sequence): (initial groups, dt list, final groups, oracle seconds)."""
    import numpy as np
    import oracle
    from paper_1007_3818_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    gx, dh = n // 16, 1.0 / n
    U = wl.sedov_level(n, gamma=GAMMA) if problem == "sedov" else wl.kh_level(n, gamma=GAMMA)
    G0 = wl.level_to_groups(U).astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    ref, dts = G0, []
    tiles = periodic_tiles(ref, gx)
    _, _, _, part = oracle.advance_groups(tiles, 0.0, dh, gamma=GAMMA, nthreads=cores,
                                          want_flux=False)
    for _ in range(steps):
        dt = oracle.hydro_dt(part, [dh], cfl)[0][0]
        ref, _, _, part = oracle.advance_groups(tiles, dt, dh, gamma=GAMMA, nthreads=cores,
                                                want_flux=False)
        tiles = periodic_tiles(ref, gx, out=tiles)
        dts.append(dt)
    return G0, dts, ref, time.perf_counter() - t0


# --------------------------------------------------------------------------
def reference_arm(args):
    """--impl reference: the oracle timed on the host cores on a bounded sample
    of the same workload, per step."""
    rank, world, _ = __import__("paper_1007_3818_gb300.dist", fromlist=["x"]).env_world()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    base = level1024_base() if args.workload == "level1024" else uniform256_level()
    tiles = oracle.fill_ghosts_uniform(base, 16, 16, 16, 0)
    if args.mode != "f64":
        tiles = tiles.astype(np.float32).astype(np.float64)
    cores = os.cpu_count() or 1
    dh = 1.0 / (1024 if args.workload == "level1024" else 256)
    oracle.build()
    t0 = time.perf_counter()
    oracle.advance_groups(tiles[:cores], 1e-4, dh, gamma=GAMMA, nthreads=cores)
    t1 = time.perf_counter() - t0
    budget = 120.0 / max(1, args.steps + args.warmup)
    n = int(min(len(tiles), max(cores, cores * int(budget / max(t1, 1e-3)))))
    sample = tiles[:n]
    for _ in range(args.warmup):
        oracle.advance_groups(sample, 1e-4, dh, gamma=GAMMA, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.advance_groups(sample, 1e-4, dh, gamma=GAMMA, nthreads=cores)
    el = time.perf_counter() - t0
    v = n * GROUP_CELLS * args.steps / el
    desc = (f"{n} of the level's groups per step (the {len(tiles)} distinct ghost-padded "
            f"groups of its periodic field), {cores} threads (OpenMP over groups)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.workload), "mode": args.mode},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def workload_name(w):
    if w == "level1024":
        return ("periodic 1024^3 level: 262,144 patch groups of 16^3 cells, lognormal density "
                "contrast 1e4 (a periodic 256^3 field repeated 4^3 times), velocity rms 1 c_s, "
                "gamma 5/3; MUSCL-Hancock/Roe step with the ghost gather fused in + FP64 dt "
                "reduction per step")
    return ("uniform periodic 256^3 level: 4,096 patch groups of 16^3 cells, density 1 + 0.1 x "
            "8 Fourier modes, p = 1, velocity rms 0.3 c_s, gamma 5/3; MUSCL-Hancock/Roe step "
            "with the ghost gather fused in + FP64 dt reduction per step")


# --------------------------------------------------------------------------
class LevelRun:
    """A device-resident uniform level stepped by the fused level kernel and
    the dt reduction (the benchmark's step)."""

    def __init__(self, native, mode, groups_dev, gx, dh, with_flux=True):
        import torch
        self.native, self.mode, self.gx, self.dh = native, mode, gx, dh
        G = gx ** 3
        self.G = G
        dev = groups_dev.device
        T = groups_dev.dtype
        self.cur = [groups_dev, torch.empty_like(groups_dev)]
        self.nxt = 0
        self.ff = torch.empty((G, 6, 5, 16, 16), device=dev, dtype=T) if with_flux else None
        self.dt_g = torch.zeros(G, device=dev, dtype=torch.float64)
        self.dh_g = torch.full((G,), dh, device=dev, dtype=torch.float64)
        self.status = torch.zeros(G, device=dev, dtype=torch.int32)
        self.partials = torch.zeros((G, 6), device=dev, dtype=torch.float64)
        self.dh_level = torch.tensor([dh], device=dev, dtype=torch.float64)
        self.dt_level = torch.zeros(1, device=dev, dtype=torch.float64)
        self.totals = torch.zeros(5, device=dev, dtype=torch.float64)
        self.ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(G, 1), device=dev,
                              dtype=torch.uint8)
        self.params = native.make_params(GAMMA, cfl=CFL)
        # dt of the first step: a zero-length step gives the partials of U^0
        native.hydro_advance_level(mode, self.cur[0], self.cur[1], None, gx, gx, gx, 0,
                                   self.dt_g, self.dh_g, None, self.partials, self.params)
        native.gamer_hydro_dt(self.partials, None, self.dh_level, CFL, self.dt_level,
                              self.totals, self.dt_g, self.ws)
        torch.cuda.synchronize()
        self.tot0 = self.totals.cpu().numpy().copy()
        self.dt0 = float(self.dt_level.item())

    def step(self, ev=None):
        import torch
        n = self.native
        src, dst = self.cur[self.nxt], self.cur[1 - self.nxt]
        torch.cuda.nvtx.range_push("level step")
        if ev is not None:
            ev[0].record()
        n.hydro_advance_level(self.mode, src, dst, self.ff, self.gx, self.gx, self.gx, 0,
                              self.dt_g, self.dh_g, self.status, self.partials, self.params)
        if ev is not None:
            ev[1].record()
        n.gamer_hydro_dt(self.partials, None, self.dh_level, CFL, self.dt_level, self.totals,
                         self.dt_g, self.ws)
        torch.cuda.nvtx.range_pop()
        self.nxt = 1 - self.nxt

    def timed(self, steps, warmup, dist, dev, clocks=None):
        """W untimed steps, then K steps between barriers and syncs; returns
        (max-over-ranks seconds, mean hydro-kernel ms, clock record)."""
        import torch
        for _ in range(warmup):
            self.step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        if clocks:
            clocks.start()
            time.sleep(0.3)
        dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            self.step(ev[i])
        e1.record()
        torch.cuda.synchronize()
        dist.barrier()
        clk = clocks.stop() if clocks else None
        el = dist.max_over_ranks(e0.elapsed_time(e1) / 1e3, device=dev)
        kms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        return el, kms, clk

    def conservation(self):
        tot = self.totals.cpu().numpy()
        return [float(abs(a - b) / max(abs(b), 1e-300)) for a, b in zip(tot, self.tot0)]


def tuned_record(t):
    return {"ctas_per_sm": t["ctas_per_sm"], "variant": t["variant"],
            "threads_per_group": t["threads_per_group"],
            "candidates_ms (ctas x variant)": t["all"]}


def tune_level(native, run):
    from paper_1007_3818_gb300 import tune
    return tune.tune_hydro_level(run.mode, run.cur[0], run.cur[1], run.ff, run.gx, run.gx,
                                 run.gx, 0, run.dt_g, run.dh_g, run.status, run.partials,
                                 run.params)


def rooflines(flops_per_cell, cells, kernel_ms, esz, peaks, hbm_peak, traffic, mode, kernel,
              with_flux=True):
    """ALU (or FP64-pipe) and HBM roofline records of one kernel launch."""
    s = kernel_ms / 1e3
    out = {}
    if flops_per_cell is not None:
        fp64 = mode == "f64"
        peak = peaks["f64"] if fp64 else peaks["f32"]
        ach = flops_per_cell * cells / s / 1e12
        out["alu"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                      "frac": ach / peak, "traffic": traffic, "kernel": kernel,
                      "flops_per_cell": flops_per_cell,
                      "peak_basis": peaks["basis_f64" if fp64 else "basis_f32"],
                      "frac_at_median_clock":
                          ach / peaks["f64_at_median_clock" if fp64 else "f32_at_median_clock"],
                      # the counted operations are adds, muls, divides and
                      # square roots, one each: against one operation per
                      # lane per clock (an FMA counted once) the same rate is
                      "frac_of_lane_op_peak": 2 * ach / peak}
    nbytes = cells / GROUP_CELLS * group_bytes(esz, with_flux)
    out["hbm"] = {"bound": "hbm", "achieved": nbytes / s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                  "frac": nbytes / s / 1e9 / hbm_peak, "traffic": traffic,
                  "algorithmic_bytes": nbytes, "kernel": kernel,
                  "peak_basis": "measured HBM copy (MEASURED_PEAKS.json hbm_gbs)"}
    return out


# --------------------------------------------------------------------------
def headline(args, native, dist, dev, world, rank):
    """The headline level on the device: returns (record, state kept for the
    other legs)."""
    import numpy as np
    import torch
    mode = MODES[args.mode]
    T = torch.float64 if args.mode == "f64" else torch.float32
    if args.workload == "level1024":
        base = level1024_base()
        gx = 64
        src = torch.as_tensor(tiled_sources(gx, 16), device=dev)
        base_dev = torch.from_numpy(base).to(dev, T)
        groups = torch.index_select(base_dev, 0, src)
        del src
    else:
        base = uniform256_level()
        gx = 16
        base_dev = torch.from_numpy(base).to(dev, T)
        groups = base_dev.clone()
    run = LevelRun(native, mode, groups, gx, 1.0 / (16 * gx))
    u0_host = None
    if not args.no_e2e:   # the initial state, for the end-to-end leg
        u0_host = host_level(args, groups.shape, T)
        u0_host[0].copy_(groups)
    tuned = tune_level(native, run)
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    el, kms, clk = run.timed(args.steps, args.warmup, dist, dev, clocks)
    cells = run.G * GROUP_CELLS
    rec = {"value": world * cells * args.steps / el, "ms_per_step": el / args.steps * 1e3,
           "kernel_ms": kms, "clocks": clk, "groups": run.G, "cells_per_step": cells,
           "tuned": tuned_record(tuned),
           "status_or": int(np.bitwise_or.reduce(run.status.cpu().numpy())),
           "conservation_rel": run.conservation(), "dt0": run.dt0}
    keep = {"base": base, "base_dev": base_dev, "gx": gx, "u0_host": u0_host}
    del run, groups
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return rec, keep


def link_peak(h_lv, dev):
    """Host-link bandwidth each way with both directions busy: up to 4 GB of
    the first host level copied in while as much of the second is copied out,
    on two streams (GB/s, the slower direction)."""
    import torch
    n = min(h_lv[0].numel(), (4 << 30) // h_lv[0].element_size())
    src, dst = h_lv[0].view(-1)[:n], h_lv[1].view(-1)[:n]
    d_in = torch.empty(n, dtype=h_lv[0].dtype, device=dev)
    d_out = torch.zeros(n, dtype=h_lv[0].dtype, device=dev)
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    best = 0.0
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s1):
            d_in.copy_(src, non_blocking=True)
        with torch.cuda.stream(s2):
            dst.copy_(d_out, non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, n * h_lv[0].element_size() / (time.perf_counter() - t0) / 1e9)
    del d_in, d_out
    return best


def host_room(world, level_bytes):
    """Whether the host's available memory holds two copies of a level per
    rank with 20 % to spare."""
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024 >= 2.4 * world * level_bytes
    except OSError:
        pass
    return world == 1


def uniform256_e2e(args, native, dist, dev, world):
    import torch
    T = torch.float64 if args.mode == "f64" else torch.float32
    u0 = host_level(args, (4096, 5, 16, 16, 16), T)
    u0[0].copy_(torch.from_numpy(uniform256_level()).to(T))
    run = LevelRun(native, MODES[args.mode], u0[0].to(dev), 16, 1 / 256, with_flux=False)
    dt0 = run.dt0
    del run
    rec = end_to_end(args, native, dist, dev, world, {"gx": 16, "u0_host": u0}, dt0)
    rec["workload"] = "the 256^3 level (host memory too small for every rank's 1024^3 level)"
    return rec


def host_level(args, shape, dtype):
    """(tensor, owner) of page-locked host memory for one host-resident level."""
    import torch
    from paper_1007_3818_gb300 import native
    if args.host_alloc == "torch":
        t = torch.empty(shape, dtype=dtype, pin_memory=True)
        return t, None
    hb = native.HostBuffer(shape, dtype)
    return hb.tensor, hb


def end_to_end(args, native, dist, dev, world, keep, dt0):
    """The headline level from pinned host memory through the public
    multi-step call; every step copies its input in and its result out."""
    import torch
    mode = MODES[args.mode]
    gx = keep["gx"]
    G = gx ** 3
    dh = 1.0 / (16 * gx)
    first = keep["u0_host"]
    second = host_level(args, first[0].shape, first[0].dtype)
    h_lv = [first[0], second[0]]
    h_st = torch.zeros(G, dtype=torch.int32).pin_memory()
    h_part = torch.zeros((G, 6), dtype=torch.float64).pin_memory()
    n_e2e = max(3, args.steps)
    h_dt = torch.zeros(n_e2e, dtype=torch.float64).pin_memory()
    params = native.make_params(GAMMA, cfl=CFL)
    # slab size: 8 z-layers of groups (a few GB per copy) for the 1024^3 level,
    # picked by a short trial among 1..8 layers for the 256^3 one
    layer = gx * gx
    if gx >= 64:
        batch = 8 * layer
    else:
        trial = {}
        for nl in (1, 2, 4, 8):
            pl = native.Pipeline(mode, nl * layer, with_flux=False)
            pl.level_run_host(h_lv[0], h_lv[1], gx, gx, gx, 0, 2, dt0, dh, CFL, params)
            t0 = time.perf_counter()
            pl.level_run_host(h_lv[0], h_lv[1], gx, gx, gx, 0, 4, dt0, dh, CFL, params)
            trial[nl] = time.perf_counter() - t0
            pl.close()
        batch = min(trial, key=trial.get) * layer
    link = link_peak(h_lv, dev)
    pipe = native.Pipeline(mode, batch, with_flux=False)
    pipe.set_timeout(600.0)
    pipe.level_run_host(h_lv[0], h_lv[1], gx, gx, gx, 0, 1, dt0, dh, CFL, params)  # allocation
    dist.barrier()
    t0 = time.perf_counter()
    pipe.level_run_host(h_lv[0], h_lv[1], gx, gx, gx, 0, n_e2e, dt0, dh, CFL, params, h_dt,
                        h_st, h_part)
    el = dist.max_over_ranks(time.perf_counter() - t0, device=dev)
    h2d, d2h = pipe.last_bytes()
    pipe.close()
    del h_lv
    for owner in (first[1], second[1]):
        if owner is not None:
            owner.close()
    each_way = max(h2d, d2h) / n_e2e / (el / n_e2e) / 1e9
    return {"value": world * G * GROUP_CELLS * n_e2e / el, "unit": UNIT,
            "roofline": {"bound": "host link", "achieved": each_way, "peak": link,
                         "unit": "GB/s each way", "frac": each_way / link,
                         "peak_basis": "measured in this run: the same host levels copied "
                                       "in and out at once on two streams"},
            "host_memory": ("gamer_host_alloc (huge-page backed, page-locked)"
                            if args.host_alloc == "library" else "torch pinned (cudaHostAlloc)"),
            "h2d_bytes_per_step": h2d // n_e2e, "d2h_bytes_per_step": d2h // n_e2e,
            "steps": n_e2e, "ms_per_step": el / n_e2e * 1e3, "slab_groups": batch,
            "api": "gamer_pipeline_level_run_host (%d steps of the pinned host level in one "
                   "call; each step copies the interiors in and the new state out in z-slabs of "
                   "%d layers through a device copy of the level, ghost gather on the device, "
                   "the next step's copies in overlapping this step's copies out; dt per step "
                   "from the previous step's partials on the device; status and last partials "
                   "back at the end)" % (n_e2e, batch // layer)}


def uniform256_record(args, native, dev, peaks, hbm_peak, flops, cpu):
    """Config 2: the 256^3 level (4,096 groups) on the device, its CUDA-graph
    replay, rooflines and CPU baseline."""
    import torch
    from paper_1007_3818_gb300 import dist
    mode = MODES[args.mode]
    T = torch.float64 if args.mode == "f64" else torch.float32
    run = LevelRun(native, mode, torch.from_numpy(uniform256_level()).to(dev, T), 16, 1 / 256)
    tuned = tune_level(native, run)
    el, kms, _ = run.timed(args.steps, args.warmup, dist, dev)
    cells = run.G * GROUP_CELLS
    graphs = [native.LevelGraph(mode, run.cur[i], run.cur[1 - i], None, run.ff, run.dt_g,
                                run.dh_g, run.status, run.partials, 16, 16, 16, 0, run.params,
                                run.dh_level, run.dt_level, run.totals, run.ws) for i in (0, 1)]
    gi = run.nxt
    for _ in range(4):
        graphs[gi].launch()
        gi ^= 1
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record()
    for _ in range(args.steps):
        graphs[gi].launch()
        gi ^= 1
    g1.record()
    torch.cuda.synchronize()
    el_graph = g0.elapsed_time(g1) / 1e3
    for g in graphs:
        g.close()
    esz = 8 if args.mode == "f64" else 4
    traffic = measured_traffic(args.mode, run.G)
    rl = rooflines(flops, cells, kms, esz, peaks, hbm_peak, traffic, args.mode,
                   "hydro_step_kernel (fused level)")
    rec = {"workload": workload_name("uniform256"), "groups": run.G, "value": cells * args.steps / el,
           "ms_per_step": el / args.steps * 1e3, "kernel_ms": kms,
           "graph": {"ms_per_step": el_graph / args.steps * 1e3,
                     "value": cells * args.steps / el_graph},
           "roofline": rl.get("alu"), "roofline_hbm": rl["hbm"], "cpu_baseline": cpu,
           "tuned": tuned_record(tuned),
           "conservation_rel": run.conservation()}
    u0 = None
    if not args.no_e2e:
        u0 = host_level(args, run.cur[0].shape, T)
        u0[0].copy_(torch.from_numpy(uniform256_level()).to(T))
    dt0 = run.dt0
    del run
    torch.cuda.empty_cache()
    if u0 is not None:
        rec["e2e"] = end_to_end(args, native, dist, dev, 1, {"gx": 16, "u0_host": u0}, dt0)
    return rec


def amr_record(args, native, dev):
    """Config 4: 54,000 tiles of three AMR levels (2,000 / 12,000 / 40,000 at dh
    1/256, 1/512, 1/1024), shuffled, one persistent launch per step under the
    captured batch graph (dt per level from the previous partials, scatter,
    step)."""
    import torch
    from paper_1007_3818_gb300 import tune
    from paper_1007_3818_gb300 import workloads as wl
    mode = MODES[args.mode]
    T = torch.float64 if args.mode == "f64" else torch.float32
    base, origins, level, dh_level = wl.amr_batch_parts()
    N = len(level)
    tiles = wl.window_tiles_torch(base, origins, dev).to(T)
    d_level = torch.as_tensor(level, device=dev)
    d_dhl = torch.as_tensor(dh_level, device=dev)
    d_dh = d_dhl[d_level.long()].contiguous()
    params = native.make_params(GAMMA, cfl=CFL)
    out = torch.empty((N, 5, 16, 16, 16), device=dev, dtype=T)
    ff = torch.empty((N, 6, 5, 16, 16), device=dev, dtype=T)
    dt_g = torch.zeros(N, device=dev, dtype=torch.float64)
    st = torch.zeros(N, device=dev, dtype=torch.int32)
    part = torch.empty((N, 6), device=dev, dtype=torch.float64)
    dtl = torch.zeros(3, device=dev, dtype=torch.float64)
    tot = torch.zeros(5, device=dev, dtype=torch.float64)
    ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(N, 3), device=dev, dtype=torch.uint8)
    native.hydro_advance(mode, tiles, out, None, dt_g, d_dh, None, part, params)
    tuned = tune.tune_hydro(mode, tiles, out, ff, dt_g, d_dh, st, part, params)
    native.hydro_advance(mode, tiles, out, None, torch.zeros_like(dt_g), d_dh, None, part,
                         params)
    graph = native.BatchGraph(mode, tiles, out, ff, dt_g, d_dh, d_level, 3, st, part, params,
                              d_dhl, dtl, tot, ws)
    for _ in range(args.warmup):
        graph.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        graph.launch()
    e1.record()
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    graph.close()
    cells = N * GROUP_CELLS
    return {"workload": "AMR-shaped batch: 2,000 / 12,000 / 40,000 ghost-padded 20^3 tiles of "
                        "three levels (dh 1/256, 1/512, 1/1024; lognormal sigma_ln 1.5, "
                        "p = rho^gamma/gamma, v rms 1), shuffled; per step one captured graph: "
                        "FP64 dt per level from the previous partials, scatter, one persistent "
                        "launch over all groups, face fluxes on",
            "groups": N, "value": cells * args.steps / el, "ms_per_step": el / args.steps * 1e3,
            "dt_level": dtl.cpu().numpy().tolist(),
            "tuned": tuned_record(tuned)}


def modes_record(args, native, dev, peaks, hbm_peak, flops, refs):
    """f32, mixed, ff and f64 on the 256^3 level: fused-kernel time, rate,
    roofline fraction; and the rel-L1 error of each against the oracle on the
    precision-study problems (same initial state rounded to FP32, the oracle's
    dt sequence)."""
    import numpy as np
    import torch
    from paper_1007_3818_gb300 import dist
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    out = {}
    lv = uniform256_level()
    for name, mode in (("f32", 0), ("mixed", 1), ("ff", 3), ("f64", 2)):
        T = torch.float64 if mode == 2 else torch.float32
        run = LevelRun(native, mode, torch.from_numpy(lv).to(dev, T), 16, 1 / 256)
        tuned = tune_level(native, run)
        steps = max(3, min(args.steps, 10))
        el, kms, _ = run.timed(steps, 2, dist, dev)
        cells = run.G * GROUP_CELLS
        rl = rooflines(flops, cells, kms, 8 if mode == 2 else 4, peaks, hbm_peak, None, name,
                       "hydro_step_kernel (fused level)")
        rec = {"kernel_ms": kms, "value": cells / (kms / 1e3),
               "step_value": cells * steps / el, "tuned": tuned_record(tuned),
               "roofline": rl.get("alu"), "roofline_hbm_frac": rl["hbm"]["frac"]}
        del run
        for key, (G0, dts, ref, _) in refs.items():
            gx = round(len(G0) ** (1 / 3))
            cur = torch.from_numpy(G0).to(dev, T)
            nxt = torch.empty_like(cur)
            Gn = gx ** 3
            dh_t = torch.full((Gn,), 1.0 / (16 * gx), device=dev, dtype=torch.float64)
            st = torch.zeros(Gn, device=dev, dtype=torch.int32)
            params = native.make_params(GAMMA)
            for dt in dts:
                dt_t = torch.full((Gn,), dt, device=dev, dtype=torch.float64)
                native.hydro_advance_level(mode, cur, nxt, None, gx, gx, gx, 0, dt_t, dh_t, st,
                                           None, params)
                cur, nxt = nxt, cur
            torch.cuda.synchronize()
            got = cur.double().cpu().numpy()
            rec[key] = precision_entry(got, ref)
            del cur, nxt
        out[name] = rec
        torch.cuda.empty_cache()
    return out


def precision_entry(got, ref):
    import numpy as np
    from gpu_util import rel_l1_fields, rel_l1_per_field
    fin = bool(np.isfinite(got).all())
    return {"rel_l1": rel_l1_fields(got, ref) if fin else None,
            "rel_l1_per_field": rel_l1_per_field(got, ref).tolist() if fin else None,
            "finite": fin}


# --------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
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
    t_start = time.perf_counter()
    head, keep = headline(args, native, dist, dev, world, rank)
    e2e = None
    if not args.no_e2e:
        if keep["gx"] == 64 and not host_room(world, keep["u0_host"][0].numel() *
                                              keep["u0_host"][0].element_size()):
            # N ranks of one node would hold N x 2 host copies of the 21.5 GB
            # level: where the host cannot, every rank streams the 256^3 level
            e2e = uniform256_e2e(args, native, dist, dev, world)
        else:
            e2e = end_to_end(args, native, dist, dev, world, keep, head["dt0"])
    keep.pop("u0_host", None)
    clk = head["clocks"]
    peaks = alu_peaks(dev, clk)
    hbm_peak = measured_peaks().get("hbm_gbs", 6702.2)
    esz = 8 if args.mode == "f64" else 4
    extras = rank == 0 and world == 1 and not args.no_extras
    cpu = cpu256 = flops = None
    refs = {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # CPU baseline leg: the oracle on bounded samples of the headline and
        # config-2 workloads, its flop count, and the precision-study runs
        # whose states are the reference of the modes' rel-L1 figures
        base = keep["base"]
        if args.mode != "f64":
            base = base.astype(np.float32).astype(np.float64)
        tiles = periodic_tiles(base, 16)   # the level's 4,096 distinct 20^3 inputs
        dh = 1.0 / (16 * keep["gx"])
        v, cores, desc = oracle_rate(tiles, head["dt0"], dh, args.cpu_seconds)
        flops = oracle_flops_per_cell(tiles[0], head["dt0"], dh)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": desc + (" of the level's 4,096 distinct ghost-padded groups"
                                 if keep["gx"] == 64 else "")}
        if extras:
            import oracle
            lv = uniform256_level().astype(np.float32).astype(np.float64)
            v2, c2, d2 = oracle_rate(periodic_tiles(lv, 16), 1e-3, 1 / 256, args.cpu_seconds)
            cpu256 = {"value": v2, "unit": UNIT, "cores": c2, "kind": "oracle", "sample": d2}
            refs["kh128_cfl0.5_100steps"] = oracle_precision_reference("kh", 128, 100, 0.5)
            refs["sedov128_cfl0.3_100steps"] = oracle_precision_reference("sedov", 128, 100, 0.3)
    traffic = measured_traffic(args.mode, head["groups"])
    rl = rooflines(flops, head["cells_per_step"], head["kernel_ms"], esz, peaks, hbm_peak,
                   traffic, args.mode, "hydro_step_kernel (fused level)")
    per_config, modes = {}, None
    if extras:
        if args.workload == "level1024":
            per_config["uniform256"] = uniform256_record(args, native, dev, peaks, hbm_peak,
                                                         flops, cpu256)
        per_config["amr54000"] = amr_record(args, native, dev)
        if refs:
            modes = modes_record(args, native, dev, peaks, hbm_peak, flops, refs)
            modes["reference"] = {k: {"oracle_s": r[3], "steps": len(r[1]),
                                      "t_end": float(sum(r[1]))} for k, r in refs.items()}
    if rank == 0:
        out = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.mode], "data": "synthetic",
            "config": {"workload": workload_name(args.workload), "mode": args.mode,
                       "groups": head["groups"], "cells_per_step": head["cells_per_step"],
                       "gamma": GAMMA, "cfl": CFL, "seed": SEED,
                       "l2": "inputs larger than L2 (level %.0f MB read, %.0f MB written per "
                             "step)" % (head["groups"] * 20480 * esz / 1e6,
                                        head["groups"] * 28160 * esz / 1e6),
                       "parallelism": f"{world} independent levels (weak scaling)"},
            "roofline": rl.get("alu"), "roofline_hbm": rl["hbm"], "cpu_baseline": cpu,
            "e2e": e2e, "clocks": clk,
            "gpu_launches": 4 * args.steps,
            "kernel_ms": {"hydro_step": head["kernel_ms"]},
            "tuned": head["tuned"], "status_or": head["status_or"],
            "conservation_rel": head["conservation_rel"],
            "per_config": per_config, "modes": modes,
            "bench_wall_s": time.perf_counter() - t_start,
        }
        print(json.dumps(out), flush=True)
    dist.finalize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
