"""Failure detection, made to happen without a GPU fault or hang.

* On-chip: a debug knob withholds one input-plane copy of one group, so that
  CTA's bounded mbarrier wait runs out after a short poll limit.  The CTA
  stops; the group and every later group it owned must carry
  GAMER_ST_INTERNAL_TIMEOUT and NaN partials, every other group must be
  untouched (bit for bit a normal run), and gamer_hydro_dt must turn the NaN
  partials into a NaN time step for the level -- so the failure shows even to
  a caller that passes no status array.
* Host side: the streamed pipeline's deadline.  A host callback that sleeps
  holds the pipeline's streams; with a 50 ms timeout the call returns
  GAMER_E_TIMEOUT, the next call (still held) returns it again without
  enqueuing anything, and once the hold is over a call succeeds and the first
  call's queued work has completed with the right results.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_1007_3818_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

F32, F64 = 0, 2
TIMEOUT_BIT = 0x10


@pytest.fixture(scope="module")
def native():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1007_3818_gb300 import native as n
    assert n.gamer_device_check() == 0
    return n


@pytest.fixture
def knobs(native):
    yield native
    native.gamer_set_debug_drop_plane(-1, 0)
    native.gamer_set_hydro_ctas_per_sm(F32, 0)
    native.gamer_set_hydro_ctas_per_sm(F64, 0)


def _run_tiles(native, tiles, mode):
    import torch
    T = torch.float64 if mode == F64 else torch.float32
    N = tiles.shape[0]
    d_in = torch.from_numpy(tiles).to("cuda", T)
    out = torch.zeros((N, 5, 16, 16, 16), device="cuda", dtype=T)
    st = torch.zeros(N, device="cuda", dtype=torch.int32)
    part = torch.zeros((N, 6), device="cuda", dtype=torch.float64)
    dt = torch.full((N,), 2e-3, device="cuda", dtype=torch.float64)
    dh = torch.full((N,), 1 / 256, device="cuda", dtype=torch.float64)
    native.hydro_advance(mode, d_in, out, None, dt, dh, st, part, native.make_params(5 / 3))
    torch.cuda.synchronize()
    return out.cpu().numpy(), st.cpu().numpy(), part.cpu().numpy()


@pytest.mark.parametrize("mode", [F32, F64], ids=["f32", "f64"])
def test_on_chip_wait_gives_up_and_flags_every_group_of_the_cta(knobs, mode):
    import torch
    native = knobs
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    # one CTA per SM in FP64; the FP32 2-CTA build with 2 per SM: grid known
    per_sm = 1 if mode == F64 else 2
    native.gamer_set_hydro_ctas_per_sm(mode, per_sm)
    grid = per_sm * sm
    N = 2 * grid + 7
    base = wl.random_smooth_groups(3, seed=31, gamma=5 / 3)
    tiles = base[np.arange(N) % 3]
    ref_out, ref_st, ref_part = _run_tiles(native, tiles, mode)
    drop = 5
    native.gamer_set_debug_drop_plane(drop, 2000)
    out, st, part = _run_tiles(native, tiles, mode)
    native.gamer_set_debug_drop_plane(-1, 0)
    abandoned = np.arange(drop, N, grid)
    assert len(abandoned) == 3
    keep = np.setdiff1d(np.arange(N), abandoned)
    assert (st[abandoned] == TIMEOUT_BIT).all()
    assert np.isnan(part[abandoned]).all()
    assert np.array_equal(st[keep], ref_st[keep])
    assert np.array_equal(part[keep], ref_part[keep])
    assert np.array_equal(out[keep], ref_out[keep])
    # the NaN partials make the level's time step NaN
    d_part = torch.as_tensor(part, device="cuda")
    dt_level = torch.zeros(1, device="cuda", dtype=torch.float64)
    ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(N, 1), device="cuda",
                     dtype=torch.uint8)
    native.gamer_hydro_dt(d_part, None, torch.tensor([1 / 256], device="cuda",
                                                     dtype=torch.float64),
                          0.5, dt_level, None, None, ws)
    assert np.isnan(dt_level.item())
    # and the library works normally afterwards
    again = _run_tiles(native, tiles, mode)
    assert np.array_equal(again[0], ref_out) and np.array_equal(again[1], ref_st)


def test_on_chip_give_up_in_the_fused_level_kernel(knobs):
    import torch
    native = knobs
    gx, gy, gz = 3, 2, 2
    G = gx * gy * gz
    lv = np.concatenate([wl.level_to_groups(wl.fourier_level(n=16, seed=300 + i, gamma=5 / 3))
                         for i in range(G)])
    d_lv = torch.from_numpy(lv).to("cuda", torch.float32)
    dt = torch.full((G,), 2e-3, device="cuda", dtype=torch.float64)
    dh = torch.full((G,), 1 / 64, device="cuda", dtype=torch.float64)
    p = native.make_params(5 / 3)

    def run():
        out = torch.zeros_like(d_lv)
        st = torch.zeros(G, device="cuda", dtype=torch.int32)
        part = torch.zeros((G, 6), device="cuda", dtype=torch.float64)
        native.hydro_advance_level(F32, d_lv, out, None, gx, gy, gz, 0, dt, dh, st, part, p)
        torch.cuda.synchronize()
        return out.cpu().numpy(), st.cpu().numpy(), part.cpu().numpy()

    ref = run()
    native.gamer_set_debug_drop_plane(7, 2000)
    got = run()
    native.gamer_set_debug_drop_plane(-1, 0)
    keep = np.arange(G) != 7
    assert got[1][7] == TIMEOUT_BIT and np.isnan(got[2][7]).all()
    for a, b in zip(got, ref):
        assert np.array_equal(a[keep], b[keep])


def test_dt_reduction_propagates_nan_partials(native):
    import torch
    rng = np.random.default_rng(8)
    N = 3000
    part = np.column_stack([rng.uniform(0.1, 3.0, N), rng.standard_normal((N, 5))])
    level = (np.arange(N) % 3).astype(np.int32)
    part[1234 - 1234 % 3 + 1, 0] = np.nan          # one group of level 1
    d = lambda a, t=torch.float64: torch.as_tensor(a, device="cuda", dtype=t)  # noqa: E731
    dt_out = torch.zeros(3, device="cuda", dtype=torch.float64)
    ws = torch.empty(native.gamer_hydro_dt_workspace_bytes(N, 3), device="cuda", dtype=torch.uint8)
    native.gamer_hydro_dt(d(part), d(level, torch.int32), d([1 / 256, 1 / 512, 1 / 1024]), 0.5,
                          dt_out, None, None, ws)
    torch.cuda.synchronize()
    got = dt_out.cpu().numpy()
    assert np.isnan(got[1]) and np.isfinite(got[[0, 2]]).all()
    for l, dh in ((0, 1 / 256), (2, 1 / 1024)):
        assert got[l] == 0.5 * dh / part[level == l, 0].max()


def test_pipeline_deadline_and_recovery(native):
    import torch
    g, dh, dt = 5 / 3, 1 / 64, 1.5e-3
    lv = wl.level_to_groups(wl.fourier_level(n=64, seed=3, gamma=g)).astype(np.float32)
    h_in = torch.from_numpy(lv).pin_memory()
    outs = [torch.full_like(h_in, float("nan")).pin_memory() for _ in range(3)]
    st = torch.zeros(64, dtype=torch.int32).pin_memory()
    part = torch.zeros((64, 6), dtype=torch.float64).pin_memory()
    params = native.make_params(g)
    pl = native.Pipeline(F32, 16, with_flux=False)
    pl.set_level_mode(1)
    ref = torch.empty_like(h_in).pin_memory()
    pl.level_step_host(h_in, ref, 4, 4, 4, 0, dt, dh, st, part, params)    # allocations
    pl.set_timeout(0.05)
    pl.debug_hold(0.8)
    t0 = time.perf_counter()
    with pytest.raises(native.GamerError) as e1:
        pl.level_step_host(h_in, outs[0], 4, 4, 4, 0, dt, dh, st, part, params)
    assert e1.value.code == -8
    with pytest.raises(native.GamerError) as e2:   # still held: nothing enqueued
        pl.level_step_host(h_in, outs[1], 4, 4, 4, 0, dt, dh, st, part, params)
    assert e2.value.code == -8
    assert time.perf_counter() - t0 < 0.7
    time.sleep(1.0)
    pl.level_step_host(h_in, outs[2], 4, 4, 4, 0, dt, dh, st, part, params)
    pl.close()
    assert torch.equal(outs[0], ref)               # the timed-out call's work completed
    assert torch.isnan(outs[1]).all()              # the refused call enqueued nothing
    assert torch.equal(outs[2], ref)
