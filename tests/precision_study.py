"""Precision study (config 3): all-FP32, FP32 with FP64 pressure recovery and
FP64, each against the FP64 oracle after a number of steps on a Sedov-Taylor
blast and a Kelvin-Helmholtz shear layer (periodic boxes, gamma 5/3, CFL 0.5,
the oracle's dt sequence for every mode).  Reported numbers, not a pass/fail
test.  Run on a GPU machine:

    python tests/precision_study.py [--n 256] [--steps 100] [--problems sedov kh]
                                    [--rho-floor R] [--p-floor P] [--cfl C]

With floors, the oracle and every GPU mode apply the same floors.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from gpu_util import rel_l1_fields  # noqa: E402
from paper_1007_3818_gb300 import workloads as wl  # noqa: E402


def run(problem, n, steps, cores, rho_floor=0.0, p_floor=0.0, cfl=0.5):
    import torch
    from paper_1007_3818_gb300 import native
    g = 5.0 / 3.0
    dh = 1.0 / n
    gx = n // 16
    U = wl.sedov_level(n, gamma=g) if problem == "sedov" else wl.kh_level(n, gamma=g)
    G = wl.level_to_groups(U)
    t0 = time.perf_counter()
    ref = G.copy()
    dts = []
    ref_status = 0
    tiles = oracle.fill_ghosts_uniform(ref, gx, gx, gx, 0)
    fl = {"rho_floor": rho_floor, "p_floor": p_floor}
    _, _, _, part = oracle.advance_groups(tiles, 0.0, dh, gamma=g, nthreads=cores,
                                          want_flux=False, **fl)
    for _ in range(steps):
        dt = oracle.hydro_dt(part, [dh], cfl)[0][0]   # CFL from the state at the step start
        ref, _, st_ref, part = oracle.advance_groups(tiles, dt, dh, gamma=g, nthreads=cores,
                                                     want_flux=False, **fl)
        tiles = oracle.fill_ghosts_uniform(ref, gx, gx, gx, 0)
        ref_status |= int(np.bitwise_or.reduce(st_ref))
        dts.append(dt)
    t_oracle = time.perf_counter() - t0
    out = {"problem": problem, "n": n, "steps": steps, "t_end": float(sum(dts)),
           "oracle_s": t_oracle, "floors": fl, "cfl": cfl, "oracle_status_or": ref_status}
    for mode, name in ((0, "f32"), (1, "mixed"), (3, "ff"), (2, "f64")):
        T = torch.float64 if mode == 2 else torch.float32
        cur = torch.from_numpy(G).to("cuda", T)
        nxt = torch.empty_like(cur)
        dh_t = torch.full((gx ** 3,), dh, device="cuda", dtype=torch.float64)
        st = torch.zeros(gx ** 3, device="cuda", dtype=torch.int32)
        params = native.make_params(g, **fl)
        status = 0
        for dt in dts:
            dt_t = torch.full((gx ** 3,), dt, device="cuda", dtype=torch.float64)
            native.hydro_advance_level(mode, cur, nxt, None, gx, gx, gx, 0, dt_t, dh_t, st, None,
                                       params)
            status |= int(np.bitwise_or.reduce(st.cpu().numpy()))
            cur, nxt = nxt, cur
        torch.cuda.synchronize()
        got = cur.double().cpu().numpy()
        out[name] = {"rel_l1": rel_l1_fields(got, ref),
                     "finite": bool(np.isfinite(got).all()), "status_or": status}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--problems", nargs="+", choices=["sedov", "kh"], default=["sedov", "kh"])
    ap.add_argument("--rho-floor", type=float, default=0.0)
    ap.add_argument("--p-floor", type=float, default=0.0)
    ap.add_argument("--cfl", type=float, default=0.5)
    args = ap.parse_args()
    cores = os.cpu_count() or 1
    for problem in args.problems:
        print(json.dumps(run(problem, args.n, args.steps, cores, args.rho_floor, args.p_floor,
                             args.cfl)), flush=True)


if __name__ == "__main__":
    main()
