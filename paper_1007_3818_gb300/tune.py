"""Autotuner for the launch shape of the hydro step and the host pipeline.

What is chosen per GPU, precision mode and batch size:

  * threads per group: 160 (a thread owns two interior columns, or one and a
    face-slab cell; 320 predictions and 800 Riemann solves per plane divide
    evenly) or 320 (variant 3: one column or slab cell per thread; FP32
    storage: 96 registers, 2 CTAs = 20 warps per SM; FP64: one CTA per SM,
    10 warps instead of 5);
  * the register / shared-memory split of the 160-thread build: sized for 2
    CTAs per SM (no register spills, three input planes in flight) or for 3
    (more warps per SM, two planes in flight);
  * on the tile path also the Riemann solver out of line (variant 1) and the
    two-problems-per-thread pair kernel (variant 2);
  * for the streamed host pipeline, the batch size in groups.

Each candidate is timed with CUDA events on a batch of the caller's shape and
the fastest is applied through ``gamer_set_hydro_ctas_per_sm``.  Results are
cached per (GPU name, mode, N bucket) in memory and, if a path is given, in a
JSON file.
"""
from __future__ import annotations

import json
import os
import statistics

from . import native

_cache = {}


def _bucket(n):
    b = 1
    while b < n:
        b *= 2
    return b


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def tune_hydro(mode, inp, out, face_flux, dt, dh, status, partials, params, reps=5,
               cache_path=None):
    """Time every launch shape of gamer_hydro_advance_<mode> on the given
    device tensors, apply the fastest and return {"ctas_per_sm", "ms", "all"}."""
    import torch
    key = (torch.cuda.get_device_name(), int(mode), _bucket(int(inp.shape[0])))
    if key in _cache:
        native.gamer_set_hydro_ctas_per_sm(mode, _cache[key]["ctas_per_sm"])
        native.gamer_set_hydro_variant(_cache[key]["variant"])
        return _cache[key]
    # (CTAs per SM, code variant): the FP32 3-CTA build also comes with the
    # Riemann solver out of line (smaller code for the instruction cache);
    # every mode has the pair kernel, the FP32-storage modes the 320-thread
    # build
    if mode == native.GAMER_MODE_F64:
        candidates = [(1, 0), (0, 2), (0, 3)]
    elif mode == native.GAMER_MODE_F32:
        candidates = [(2, 0), (3, 0), (3, 1), (0, 2), (0, 3)]
    else:
        candidates = [(2, 0), (3, 0), (0, 2), (0, 3)]
    results = {}
    for c, v in candidates:
        native.gamer_set_hydro_ctas_per_sm(mode, c)
        native.gamer_set_hydro_variant(v)
        results[(c, v)] = _time(lambda: native.hydro_advance(mode, inp, out, face_flux, dt, dh,
                                                             status, partials, params), reps)
    best = min(results, key=results.get)
    native.gamer_set_hydro_ctas_per_sm(mode, best[0])
    native.gamer_set_hydro_variant(best[1])
    res = {"ctas_per_sm": best[0], "variant": best[1],
           "threads_per_group": 320 if best[1] == 3 else 160, "ms": results[best],
           "all": {f"{c}x{v}": t for (c, v), t in results.items()}}
    _cache[key] = res
    if cache_path:
        _save(cache_path, key, res)
    return res


def tune_pipeline(mode, h_in, h_out, h_ff, h_dt, h_dh, h_st, h_part, params,
                  batches=(256, 512, 1024), reps=3):
    """Pick the pipeline batch size (groups) for host buffers of this shape."""
    import time
    results = {}
    for b in batches:
        pl = native.Pipeline(mode, b, with_flux=h_ff is not None)
        pl.advance_host(h_in, h_out, h_ff, h_dt, h_dh, h_st, h_part, params)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            pl.advance_host(h_in, h_out, h_ff, h_dt, h_dh, h_st, h_part, params)
            ts.append(time.perf_counter() - t0)
        pl.close()
        results[b] = statistics.median(ts) * 1e3
    best = min(results, key=results.get)
    return {"batch": best, "ms": results[best], "all": results}


def _save(path, key, res):
    data = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                data = json.load(f)
        except (OSError, ValueError):
            data = {}
    data["|".join(map(str, key))] = res
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, default=str)
    os.replace(tmp, path)


def tune_hydro_level(mode, level, out, face_flux, gx, gy, gz, bc, dt, dh, status, partials,
                     params, reps=5):
    """As tune_hydro for gamer_hydro_advance_level_<mode> (fused ghost gather);
    the level kernel comes in the one-problem-at-a-time shape only."""
    import torch
    key = ("level", torch.cuda.get_device_name(), int(mode), _bucket(gx * gy * gz))
    if key in _cache:
        native.gamer_set_hydro_ctas_per_sm(mode, _cache[key]["ctas_per_sm"])
        native.gamer_set_hydro_variant(_cache[key]["variant"])
        return _cache[key]
    # (CTAs per SM, variant): the 160-thread builds for 2 and 3 CTAs per SM
    # (one in FP64) and the 320-thread build
    candidates = ([(1, 0), (0, 3)] if mode == native.GAMER_MODE_F64
                  else [(2, 0), (3, 0), (0, 3)])
    results = {}
    for c, v in candidates:
        native.gamer_set_hydro_ctas_per_sm(mode, c)
        native.gamer_set_hydro_variant(v)
        results[(c, v)] = _time(lambda: native.hydro_advance_level(
            mode, level, out, face_flux, gx, gy, gz, bc, dt, dh, status, partials, params), reps)
    best = min(results, key=results.get)
    native.gamer_set_hydro_ctas_per_sm(mode, best[0])
    native.gamer_set_hydro_variant(best[1])
    res = {"ctas_per_sm": best[0], "variant": best[1],
           "threads_per_group": 320 if best[1] == 3 else 160, "ms": results[best],
           "all": {f"{c}x{v}": t for (c, v), t in results.items()}}
    _cache[key] = res
    return res
