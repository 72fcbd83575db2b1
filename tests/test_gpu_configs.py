"""Full-size workloads on the GPU against the oracle.

* uniform periodic 256^3 level (4096 groups): one step through the CUDA-graph
  launch that the benchmark times (ghost fill -> hydro step -> dt reduction),
  every group compared with the oracle, plus the next dt and the totals;
* Sedov blast and Kelvin-Helmholtz 256^3 boxes, every group, one step;
* the AMR-shaped batch of 54,000 independent tiles on 3 levels, per-level dt
  from the device reduction, sampled groups compared.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from gpu_util import (TOL_F32_1, TOL_F64, assert_elementwise, elementwise_excess, rel_l1_fields,
                      rel_l1_per_field)
from paper_1007_3818_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

F32, MIXED, F64 = 0, 1, 2
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def _device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def fourier_level():
    return wl.level_to_groups(wl.fourier_level(n=256, seed=1007, gamma=5 / 3))


def _graph_step(level_groups, mode, gamma, dt, dh, gx=16):
    """One device-resident level step through gamer_level_graph (bench path)."""
    import torch
    from paper_1007_3818_gb300 import native
    T = torch.float64 if mode == F64 else torch.float32
    G = gx ** 3
    a = torch.from_numpy(level_groups).to("cuda", T)
    b = torch.empty_like(a)
    tiles = torch.empty((G, 5, 20, 20, 20), device="cuda", dtype=T)
    ff = torch.empty((G, 6, 5, 16, 16), device="cuda", dtype=T)
    dt_g = torch.full((G,), dt, device="cuda", dtype=torch.float64)
    dh_g = torch.full((G,), dh, device="cuda", dtype=torch.float64)
    st = torch.zeros(G, device="cuda", dtype=torch.int32)
    part = torch.zeros((G, 6), device="cuda", dtype=torch.float64)
    dh_level = torch.tensor([dh], device="cuda", dtype=torch.float64)
    dt_level = torch.zeros(1, device="cuda", dtype=torch.float64)
    tot = torch.zeros(5, device="cuda", dtype=torch.float64)
    ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(G, 1), device="cuda", dtype=torch.uint8)
    params = native.make_params(gamma, cfl=0.5)
    g = native.LevelGraph(mode, a, b, tiles, ff, dt_g, dh_g, st, part, gx, gx, gx, 0, params,
                          dh_level, dt_level, tot, ws)
    g.launch()
    torch.cuda.synchronize()
    g.close()
    return (b.double().cpu().numpy(), ff.double().cpu().numpy(), st.cpu().numpy(),
            part.cpu().numpy(), float(dt_level.item()), tot.cpu().numpy(), dt_g.cpu().numpy())


@pytest.mark.parametrize("mode,tol", [(F32, TOL_F32_1), (MIXED, TOL_F32_1), (F64, TOL_F64)],
                         ids=["f32", "mixed", "f64"])
def test_uniform_level_full_size_graph_step(fourier_level, mode, tol):
    g, dh = 5 / 3, 1 / 256
    lv = fourier_level if mode == F64 else fourier_level.astype(np.float32).astype(np.float64)
    tiles = oracle.fill_ghosts_uniform(lv, 16, 16, 16, 0)
    _, _, _, p0 = oracle.advance_groups(tiles, 0.0, dh, gamma=g, nthreads=CORES, want_flux=False)
    dt = oracle.hydro_dt(p0, [dh], 0.5)[0][0]
    r_out, r_ff, r_st, r_part = oracle.advance_groups(tiles, dt, dh, gamma=g, nthreads=CORES)
    out, ff, st, part, dt_next, tot, dt_g = _graph_step(lv, mode, g, dt, dh)
    assert rel_l1_fields(out, r_out) <= tol
    assert max(rel_l1_per_field(out, r_out)) <= tol
    assert rel_l1_fields(ff.reshape(-1, 5, 256), r_ff.reshape(-1, 5, 256)) <= 10 * tol
    assert_elementwise(out, r_out, mode, "state")
    assert_elementwise(ff, r_ff, mode, "face flux", state=False)
    assert np.array_equal(st.astype(np.uint32), r_st)
    r_dt, r_tot = oracle.hydro_dt(r_part, [dh], 0.5)
    ptol = 1e-12 if mode == F64 else 10 * tol
    assert abs(dt_next - r_dt[0]) <= ptol * r_dt[0]
    assert np.all(np.abs(tot - r_tot) <= ptol * np.abs(r_out).reshape(-1, 5, 4096).sum(axis=(0, 2)))
    assert (dt_g == dt_next).all()


def _box_tiles(U):
    return oracle.fill_ghosts_uniform(wl.level_to_groups(U), U.shape[3] // 16, U.shape[2] // 16,
                                      U.shape[1] // 16, 0)


@pytest.mark.parametrize("problem", ["sedov", "kh"])
@pytest.mark.parametrize("mode", [F32, MIXED, F64], ids=["f32", "mixed", "f64"])
def test_sedov_and_kh_full_size_one_step(problem, mode):
    """Config 3 boxes (256^3 each), every group, one CFL-0.5 step.  FP64 holds
    1e-12; the FP32 modes are bounded by 1e-5 on KH (smooth away from the
    layers) and report the Sedov error, where the FP32 storage of E alone
    carries the cancellation (rho v^2 / 2 >> p)."""
    from gpu_util import gpu_advance, host_input
    g, dh = 5 / 3, 1 / 256
    U = wl.sedov_level(256, gamma=g) if problem == "sedov" else wl.kh_level(256, gamma=g)
    tiles = host_input(_box_tiles(U), mode)
    _, _, _, p0 = oracle.advance_groups(tiles, 0.0, dh, gamma=g, nthreads=CORES, want_flux=False)
    dt = oracle.hydro_dt(p0, [dh], 0.5)[0][0]
    r_out, _, r_st, _ = oracle.advance_groups(tiles, dt, dh, gamma=g, nthreads=CORES,
                                              want_flux=False)
    out, _, st, _ = gpu_advance(tiles, dt, dh, g, mode, with_flux=False)
    err = rel_l1_fields(out, r_out)
    per_field = rel_l1_per_field(out, r_out)
    excess = elementwise_excess(out, r_out, mode)[0]
    # per field, the KH layer's rho*vz (seeded noise only in vy) is tiny
    # after one step and carries a large plain relative error of its own; the
    # magnitude-normalised figure (max over fields) is the one bounded here
    print(f"{problem} mode {mode}: rel-L1 {err:.3e} (per field "
          f"{', '.join('%.2e' % x for x in per_field)}), element-wise excess {excess:.3g}")
    if mode == F64:
        assert err <= TOL_F64
        assert np.array_equal(st, r_st)
        assert excess <= 1.0
    elif problem == "kh":
        assert err <= TOL_F32_1
    else:
        assert err <= 1e-4


@pytest.mark.parametrize("mode,tol", [(F32, TOL_F32_1), (F64, TOL_F64)], ids=["f32", "f64"])
def test_amr_batch_full_size_sampled(mode, tol):
    """Config 4: 2,000 / 12,000 / 40,000 tiles at dh 1/256, 1/512, 1/1024,
    shuffled; dt per level from the device FP64 reduction of a zero-length
    step; one step of all 54,000 tiles in one launch, 48 sampled tiles checked."""
    import torch
    from paper_1007_3818_gb300 import native
    g = 5 / 3
    base, origins, level, dh_level = wl.amr_batch_parts()
    N = len(level)
    T = torch.float64 if mode == F64 else torch.float32
    tiles = wl.window_tiles_torch(base, origins, "cuda").to(T)
    d_level = torch.as_tensor(level, device="cuda")
    d_dhl = torch.as_tensor(dh_level, device="cuda")
    d_dh = d_dhl[d_level.long()].contiguous()
    d_dt = torch.zeros(N, device="cuda", dtype=torch.float64)
    out = torch.empty((N, 5, 16, 16, 16), device="cuda", dtype=T)
    part = torch.empty((N, 6), device="cuda", dtype=torch.float64)
    st = torch.zeros(N, device="cuda", dtype=torch.int32)
    params = native.make_params(g)
    native.hydro_advance(mode, tiles, out, None, d_dt, d_dh, None, part, params)
    dt_level = torch.zeros(3, device="cuda", dtype=torch.float64)
    ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(N, 3), device="cuda", dtype=torch.uint8)
    native.gamer_hydro_dt(part, d_level, d_dhl, 0.5, dt_level, None, d_dt, ws)
    native.hydro_advance(mode, tiles, out, None, d_dt, d_dh, st, part, params)
    torch.cuda.synchronize()
    sample = np.unique(np.r_[0, N - 1, np.random.default_rng(5).integers(0, N, 46)])
    host = wl.window_tiles(base, origins[sample])
    if mode != F64:
        host = host.astype(np.float32).astype(np.float64)
    dts = d_dt.cpu().numpy()[sample]
    r_out, _, r_st, r_part = oracle.advance_groups(host, dts, dh_level[level[sample]], gamma=g,
                                                   nthreads=CORES, want_flux=False)
    got = out.double().cpu().numpy()[sample]
    assert rel_l1_fields(got, r_out) <= tol
    assert max(rel_l1_per_field(got, r_out)) <= tol
    assert_elementwise(got, r_out, mode, "state")
    assert np.array_equal(st.cpu().numpy()[sample].astype(np.uint32), r_st)
    # the per-level dt are CFL-limited by each level's own groups
    assert (dt_level.cpu().numpy() > 0).all()


@pytest.mark.parametrize("level_mode", [1, 2], ids=["device-copy", "slab-windows"])
@pytest.mark.parametrize("mode,tol", [(F32, TOL_F32_1), (F64, TOL_F64)], ids=["f32", "f64"])
def test_pipeline_level_step_small(mode, tol, level_mode):
    """Host-resident level through the streamed pipeline (z-slabs with halo
    layers, ghost zones gathered on the device, H2D / step / D2H overlap)."""
    import torch
    from paper_1007_3818_gb300 import native
    g, dh, dt = 5 / 3, 1 / 64, 1.5e-3
    lv = wl.level_to_groups(wl.fourier_level(n=64, seed=3, gamma=g))
    T = torch.float64 if mode == F64 else torch.float32
    if mode != F64:
        lv = lv.astype(np.float32).astype(np.float64)
    h_in = torch.from_numpy(lv).to(T).pin_memory()
    h_out = torch.full_like(h_in, float("nan")).pin_memory()
    part = torch.zeros((64, 6), dtype=torch.float64).pin_memory()
    st = torch.zeros(64, dtype=torch.int32).pin_memory()
    pl = native.Pipeline(mode, 24, with_flux=False)
    pl.set_level_mode(level_mode)
    pl.level_step_host(h_in, h_out, 4, 4, 4, 0, dt, dh, st, part, native.make_params(g))
    h2d, d2h = pl.last_bytes()
    pl.close()
    esz = 8 if mode == F64 else 4
    if level_mode == 2:
        # slabs of one layer (16 groups <= 24): each sends its layer and both neighbours
        assert h2d == 4 * (3 * 16 * 20480 * esz + 16 * 16)
    else:
        # every layer once (the periodic wrap layer goes first, not again at
        # the end), and dt, dh of all groups
        assert h2d == 4 * 16 * 20480 * esz + 16 * 64
    assert d2h == 64 * (20480 * esz + 4 + 48)
    tiles = oracle.fill_ghosts_uniform(lv, 4, 4, 4, 0)
    r_out, _, r_st, r_part = oracle.advance_groups(tiles, dt, dh, gamma=g, want_flux=False)
    assert rel_l1_fields(h_out.double().numpy(), r_out) <= tol
    assert np.array_equal(st.numpy().astype(np.uint32), r_st)


def test_streamed_level_full_size_sampled():
    """Config 5: a 1024^3 level (64^3 = 262,144 groups, 21 GB of FP32
    interiors) held in pinned host memory, one streamed step (z-slabs with halo
    layers, ghost gather on the device, H2D / step / D2H overlapped on 3
    streams); 24 sampled groups checked.
    The level tiles a periodic 256^3 lognormal field of density contrast 1e4,
    so each group's ghost-padded input is that of a group of the 256^3 field."""
    import torch
    from paper_1007_3818_gb300 import native
    g = 5 / 3
    base = wl.level_to_groups(wl.lognormal_base(256, 1007 + 2, gamma=g, sigma_ln=np.log(1e4) / 8,
                                                clip=4.0, vel_rms=1.0)).astype(np.float32)
    gx = 64
    G = gx ** 3
    gid = np.arange(G)
    bx, by, bz = gid % gx, (gid // gx) % gx, gid // (gx * gx)
    src = ((bz % 16) * 16 + (by % 16)) * 16 + (bx % 16)
    h_in = torch.empty((G, 5, 16, 16, 16), dtype=torch.float32, pin_memory=True)
    torch.index_select(torch.from_numpy(base), 0, torch.from_numpy(src), out=h_in)
    h_out = torch.empty_like(h_in, pin_memory=True)
    part = torch.zeros((G, 6), dtype=torch.float64, pin_memory=True)
    st = torch.zeros(G, dtype=torch.int32, pin_memory=True)
    base64 = base.astype(np.float64)
    tiles = oracle.fill_ghosts_uniform(base64, 16, 16, 16, 0)
    dh = 1.0 / 1024
    _, _, _, p0 = oracle.advance_groups(tiles, 0.0, dh, gamma=g, nthreads=CORES, want_flux=False)
    dt = oracle.hydro_dt(p0, [dh], 0.5)[0][0]
    pl = native.Pipeline(F32, 4096, with_flux=False)
    pl.level_step_host(h_in, h_out, gx, gx, gx, 0, dt, dh, st, part, native.make_params(g))
    pl.close()
    sample = np.unique(np.r_[0, G - 1, np.random.default_rng(9).integers(0, G, 22)])
    r_out, _, r_st, _ = oracle.advance_groups(tiles[src[sample]], dt, dh, gamma=g,
                                              nthreads=CORES, want_flux=False)
    got = h_out[torch.from_numpy(sample)].double().numpy()
    assert rel_l1_fields(got, r_out) <= TOL_F32_1
    assert_elementwise(got, r_out, F32, "state")
    assert np.array_equal(st.numpy()[sample].astype(np.uint32), r_st)


@pytest.mark.parametrize("batch", [16, 32, 64], ids=["1-layer", "2-layer", "one-slab"])
@pytest.mark.parametrize("bc", [0, 1], ids=["periodic", "zero-gradient"])
@pytest.mark.parametrize("mode", [F32, F64], ids=["f32", "f64"])
def test_pipeline_level_run_equals_single_steps(mode, bc, batch):
    """Multi-step run of a host-resident level (slab order rotated every step,
    the next step's copies in overlapping this step's copies out, dt reduced
    on the device) against the same steps one call at a time with the dt
    worked out on the host from the returned partials: the same states, dt
    sequence, status and partials bit for bit, and the exact byte counts."""
    import torch
    from paper_1007_3818_gb300 import native
    g, dh, cfl, nsteps = 5 / 3, 1 / 64, 0.5, 5
    lv = wl.level_to_groups(wl.fourier_level(n=64, seed=5, gamma=g))
    T = torch.float64 if mode == F64 else torch.float32
    G = 64
    params = native.make_params(g)
    # reference: one call per step, dt from the previous step's partials
    ref = native.Pipeline(mode, batch, with_flux=False)
    ref.set_level_mode(1)
    a = torch.from_numpy(lv).to(T).pin_memory()
    b = torch.empty_like(a).pin_memory()
    st = torch.zeros(G, dtype=torch.int32).pin_memory()
    part = torch.zeros((G, 6), dtype=torch.float64).pin_memory()
    ref.level_step_host(a, b, 4, 4, 4, bc, 0.0, dh, st, part, params)   # partials of U^0
    dt0 = cfl * dh / float(part[:, 0].max())
    dts, st_or, dt = [], np.zeros(G, dtype=np.uint32), dt0
    cur, nxt = a.clone().pin_memory(), b
    for _ in range(nsteps):
        ref.level_step_host(cur, nxt, 4, 4, 4, bc, dt, dh, st, part, params)
        dts.append(dt)
        st_or |= st.numpy().astype(np.uint32)
        cur, nxt = nxt, cur
        dt = cfl * dh / float(part[:, 0].max())
    ref.close()
    want, want_part = cur.clone(), part.clone()
    # the run
    pl = native.Pipeline(mode, batch, with_flux=False)
    l0 = torch.from_numpy(lv).to(T).pin_memory()
    l1 = torch.full_like(l0, float("nan")).pin_memory()
    r_dt = torch.zeros(nsteps, dtype=torch.float64)
    r_st = torch.zeros(G, dtype=torch.int32)
    r_part = torch.zeros((G, 6), dtype=torch.float64)
    pl.level_run_host(l0, l1, 4, 4, 4, bc, nsteps, dt0, dh, cfl, params, r_dt, r_st, r_part)
    h2d, d2h = pl.last_bytes()
    pl.close()
    final = (l0, l1)[nsteps % 2]
    assert torch.equal(final, want)
    assert np.array_equal(r_dt.numpy(), np.array(dts))
    assert np.array_equal(r_st.numpy().astype(np.uint32), st_or)
    assert torch.equal(r_part, want_part)
    level_bytes = G * 20480 * (8 if mode == F64 else 4)
    assert h2d == 16 * G + 16 + nsteps * level_bytes
    assert d2h == nsteps * level_bytes + 8 * nsteps + 4 * G + 48 * G


@pytest.mark.parametrize("mode", [F32, F64], ids=["f32", "f64"])
def test_pipeline_level_run_edge_cases(mode):
    """nsteps 0 touches nothing; dt0 = 0 leaves the state bitwise unchanged;
    one step equals one level_step_host call bit for bit."""
    import torch
    from paper_1007_3818_gb300 import native
    g, dh, cfl = 1.4, 1 / 64, 0.4
    lv = wl.level_to_groups(wl.fourier_level(n=64, seed=6, gamma=g))
    T = torch.float64 if mode == F64 else torch.float32
    G, params = 64, native.make_params(g)
    pl = native.Pipeline(mode, 32, with_flux=False)
    l0 = torch.from_numpy(lv).to(T).pin_memory()
    l1 = torch.full_like(l0, float("nan")).pin_memory()
    pl.level_run_host(l0, l1, 4, 4, 4, 1, 0, 1e-3, dh, cfl, params)
    assert pl.last_bytes() == (0, 0) and torch.isnan(l1).all()
    r_dt = torch.full((1,), -1.0, dtype=torch.float64)
    r_st = torch.full((G,), -1, dtype=torch.int32)
    r_part = torch.zeros((G, 6), dtype=torch.float64)
    pl.level_run_host(l0, l1, 4, 4, 4, 1, 1, 0.0, dh, cfl, params, r_dt, r_st, r_part)
    assert torch.equal(l1, l0) and float(r_dt[0]) == 0.0 and (r_st == 0).all()
    dt = cfl * dh / float(r_part[:, 0].max())
    pl.level_run_host(l0, l1, 4, 4, 4, 1, 1, dt, dh, cfl, params, r_dt, r_st, r_part)
    pl.close()
    ref = native.Pipeline(mode, 32, with_flux=False)
    out = torch.empty_like(l0).pin_memory()
    st = torch.zeros(G, dtype=torch.int32).pin_memory()
    part = torch.zeros((G, 6), dtype=torch.float64).pin_memory()
    ref.level_step_host(l0, out, 4, 4, 4, 1, dt, dh, st, part, params)
    ref.close()
    assert torch.equal(l1, out) and torch.equal(r_part, part) and torch.equal(r_st, st)
    assert float(r_dt[0]) == dt


@pytest.mark.parametrize("mode", [F32, F64], ids=["f32", "f64"])
def test_amr_batch_graph_replays_equal_direct_calls(mode):
    """Config 4 (54,000 tiles on three levels, shuffled): three replays of the
    captured batch step (dt per level from the previous partials, scatter,
    persistent step of all groups) equal three rounds of the same calls made
    directly, bit for bit -- states, face fluxes, status, partials, dt per
    level and per group."""
    import torch
    from paper_1007_3818_gb300 import native
    g = 5 / 3
    base, origins, level, dh_level = wl.amr_batch_parts()
    N = len(level)
    T = torch.float64 if mode == F64 else torch.float32
    tiles = wl.window_tiles_torch(base, origins, "cuda").to(T)
    d_level = torch.as_tensor(level, device="cuda")
    d_dhl = torch.as_tensor(dh_level, device="cuda")
    d_dh = d_dhl[d_level.long()].contiguous()
    params = native.make_params(g, cfl=0.5)
    ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(N, 3), device="cuda", dtype=torch.uint8)

    def fresh():
        bufs = {"out": torch.empty((N, 5, 16, 16, 16), device="cuda", dtype=T),
                "ff": torch.empty((N, 6, 5, 16, 16), device="cuda", dtype=T),
                "dt": torch.zeros(N, device="cuda", dtype=torch.float64),
                "st": torch.zeros(N, device="cuda", dtype=torch.int32),
                "part": torch.empty((N, 6), device="cuda", dtype=torch.float64),
                "dtl": torch.zeros(3, device="cuda", dtype=torch.float64),
                "tot": torch.zeros(5, device="cuda", dtype=torch.float64)}
        # partials of the initial state (a zero-dt step)
        native.hydro_advance(mode, tiles, bufs["out"], None, bufs["dt"], d_dh, None, bufs["part"],
                             params)
        return bufs

    a, b = fresh(), fresh()
    graph = native.BatchGraph(mode, tiles, a["out"], a["ff"], a["dt"], d_dh, d_level, 3, a["st"],
                              a["part"], params, d_dhl, a["dtl"], a["tot"], ws)
    ws_b = torch.empty_like(ws)
    snaps = []
    for _ in range(3):
        graph.launch()
        native.gamer_hydro_dt(b["part"], d_level, d_dhl, 0.5, b["dtl"], b["tot"], b["dt"], ws_b)
        native.hydro_advance(mode, tiles, b["out"], b["ff"], b["dt"], d_dh, b["st"], b["part"],
                             params)
        torch.cuda.synchronize()
        snaps.append(float(a["dtl"][0]))
        for k in a:
            assert torch.equal(a[k], b[k]), k
    graph.close()
    assert (a["dtl"] > 0).all() and snaps[0] > 0


def test_host_alloc_levels_stream_like_pinned_ones():
    """Levels in gamer_host_alloc memory (huge-page backed, page-locked) go
    through the multi-step pipeline exactly as torch-pinned levels do."""
    import torch
    from paper_1007_3818_gb300 import native
    g, dh, cfl = 5 / 3, 1 / 64, 0.5
    lv = wl.level_to_groups(wl.fourier_level(n=64, seed=12, gamma=g)).astype(np.float32)
    shape = lv.shape
    bufs = [native.HostBuffer(shape, torch.float32) for _ in range(2)]
    assert not bufs[0].tensor.any()                # zero-filled
    bufs[0].tensor.copy_(torch.from_numpy(lv))
    pinned = [torch.from_numpy(lv).pin_memory(), torch.empty(shape).pin_memory()]
    res = []
    for pair in ([b.tensor for b in bufs], pinned):
        pl = native.Pipeline(F32, 32, with_flux=False)
        part = torch.zeros((64, 6), dtype=torch.float64)
        pl.level_run_host(pair[0], pair[1], 4, 4, 4, 0, 3, 1e-3, dh, cfl, native.make_params(g),
                          None, None, part)
        pl.close()
        res.append((pair[1].clone(), part))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    for b in bufs:
        b.close()
