"""Fixed small cases of the hydro step for profilers: a few launches of the
step kernel on one synthetic uniform level, and nothing else on the device
beyond the level's buffers (a 16x16x16-group FP32 level holds under 1 GB).

    python -m paper_1007_3818_gb300.profile_case --path both --groups 16 16 16

--path tiles: ghost fill into 20^3 tiles, then gamer_hydro_advance_<mode>;
--path level: gamer_hydro_advance_level_<mode> (gather fused in);
--path both:  per round, the tiles launch, then the level launch.
Each round is repeated --rounds times; with ncu, skip the first round's
launches (-s) to capture warm launches.  The level's groups are windows of
a smooth lognormal state (density, pressure and velocity fields).
"""
from __future__ import annotations

import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--path", choices=["tiles", "level", "both"], default="level")
    ap.add_argument("--mode", choices=["f32", "mixed", "f64", "ff"], default="f32")
    ap.add_argument("--groups", type=int, nargs=3, default=[16, 16, 8], metavar=("GX", "GY", "GZ"))
    ap.add_argument("--ctas", type=int, default=0, help="CTAs per SM (0: the library default)")
    ap.add_argument("--variant", type=int, default=0)
    ap.add_argument("--rounds", type=int, default=2)
    a = ap.parse_args(argv)

    import numpy as np
    import torch
    from . import native, workloads as wl

    mode = {"f32": native.GAMER_MODE_F32, "mixed": native.GAMER_MODE_MIXED,
            "f64": native.GAMER_MODE_F64, "ff": native.GAMER_MODE_FF}[a.mode]
    T = torch.float64 if mode == native.GAMER_MODE_F64 else torch.float32
    gx, gy, gz = a.groups
    G = gx * gy * gz
    base = wl.random_smooth_groups(64, seed=1, gamma=5 / 3)[:, :, 2:18, 2:18, 2:18]
    lv = np.ascontiguousarray(np.concatenate([base] * (G // 64 + 1))[:G])
    d_lv = torch.from_numpy(lv).to("cuda", T)
    out = torch.empty_like(d_lv)
    ff = torch.empty((G, 6, 5, 16, 16), device="cuda", dtype=T)
    dt = torch.full((G,), 1e-4, device="cuda", dtype=torch.float64)
    dh = torch.full((G,), 1 / 256, device="cuda", dtype=torch.float64)
    st = torch.zeros(G, device="cuda", dtype=torch.int32)
    part = torch.empty((G, 6), device="cuda", dtype=torch.float64)
    p = native.make_params(5 / 3)
    native.gamer_set_hydro_ctas_per_sm(mode, a.ctas)
    native.gamer_set_hydro_variant(a.variant)
    tiles = None
    if a.path in ("tiles", "both"):
        tiles = torch.empty((G, 5, 20, 20, 20), device="cuda", dtype=T)
        fill = (native.gamer_fill_ghosts_uniform_f64 if mode == native.GAMER_MODE_F64
                else native.gamer_fill_ghosts_uniform_f32)
        fill(d_lv, tiles, gx, gy, gz, 0)
    for _ in range(a.rounds):
        if tiles is not None:
            native.hydro_advance(mode, tiles, out, ff, dt, dh, st, part, p)
        if a.path in ("level", "both"):
            native.hydro_advance_level(mode, d_lv, out, ff, gx, gy, gz, 0, dt, dh, st, part, p)
    torch.cuda.synchronize()
    print("ok", G, "groups, status or", int(np.bitwise_or.reduce(st.cpu().numpy())))
    return 0


if __name__ == "__main__":
    sys.exit(main())
