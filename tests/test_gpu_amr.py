"""GPU parity of the coarse-fine coupling and of the nine-plane face-flux
layout, against the oracle.  The fix-up and restriction kernels compute in
FP64 in the oracle's order, so FP64 results are compared bit for bit, and so
is FP32 restriction; the FP32 fix-up rounds after each class, so a coarse cell
beside fine regions on several sides may differ by an ulp."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_util import TOL_F32_1, TOL_F64, assert_elementwise, host_input, rel_l1_fields
from paper_1007_3818_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

F32, F64 = 0, 2
G = 5.0 / 3.0
CG = (2, 2, 2)
REFINED = [(1, 1, 1), (2, 1, 1), (0, 3, 2), (3, 0, 3)]   # includes periodic-boundary patches


@pytest.fixture(scope="module", autouse=True)
def _device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _setup(seed=11):
    """Oracle two-level pieces: coarse state after its step, its nine-plane
    fluxes, the fine sub-steps' face fluxes and states, dt, dh."""
    children, faces = wl.cf_records(CG, REFINED)
    rng = np.random.default_rng(seed)
    C = wl.level_to_groups(wl.fourier_level(n=32, seed=seed, gamma=G))
    F = wl.composite_fine_level(C, CG, np.zeros((0, 5, 16, 16, 16)), [])
    fine = np.stack([F[:, 16 * p[2]:16 * p[2] + 16, 16 * p[1]:16 * p[1] + 16,
                       16 * p[0]:16 * p[0] + 16] for p in REFINED]).copy()
    fine[:, 0] *= 1.0 + 0.05 * rng.standard_normal(fine[:, 0].shape)
    dh = 1.0 / 32
    dt = 0.3 * dh / 2.0
    C1, cflux, _, _ = oracle.advance_groups(oracle.fill_ghosts_uniform(C, 2, 2, 2, 0), dt, dh,
                                            gamma=G, flux_layout=1)
    f1, ff1, _, _ = oracle.advance_groups(wl.fine_tiles(C, CG, fine, REFINED), dt / 2, dh / 2,
                                          gamma=G)
    f2, ff2, _, _ = oracle.advance_groups(wl.fine_tiles(C, CG, f1, REFINED), dt / 2, dh / 2,
                                          gamma=G)
    return dict(C=C, fine=fine, C1=C1, cflux=cflux, ff=np.stack([ff1, ff2]), f2=f2, dt=dt, dh=dh,
                children=children, faces=faces)


def _rounded(a, mode):
    return a if mode == F64 else a.astype(np.float32).astype(np.float64)


def _dev(a, mode):
    import torch
    T = torch.float64 if mode == F64 else torch.float32
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", T)


@pytest.mark.parametrize("mode", [F32, F64], ids=["f32", "f64"])
def test_flux_fixup_matches_oracle(mode):
    import torch
    from paper_1007_3818_gb300 import native
    s = _setup()
    C1, cflux, ff = (_rounded(s[k], mode) for k in ("C1", "cflux", "ff"))
    ref, bad_ref = oracle.flux_fixup(C1, cflux, ff, s["dt"], s["dh"], s["faces"])
    d_c = _dev(C1, mode)
    dt = torch.full((8,), s["dt"], device="cuda", dtype=torch.float64)
    dh = torch.full((8,), s["dh"], device="cuda", dtype=torch.float64)
    bad = torch.zeros(1, device="cuda", dtype=torch.int32)
    faces = native.records_to_device(s["faces"], native.CF_FACE_FIELDS, 32)
    native.flux_fixup(mode, d_c, _dev(cflux, mode), _dev(ff, mode), dt, dh, faces, bad)
    torch.cuda.synchronize()
    got = d_c.double().cpu().numpy()
    assert int(bad.item()) == 0 == bad_ref
    assert not np.array_equal(ref, C1)   # the fix-up did change cells
    if mode == F64:
        assert np.array_equal(got, ref)
    else:
        want = ref.astype(np.float32).astype(np.float64)
        assert np.all(np.abs(got - want) <= 2.0 * np.spacing(np.abs(want).astype(np.float32)))


@pytest.mark.parametrize("mode", [F32, F64], ids=["f32", "f64"])
def test_restrict_matches_oracle_bitwise(mode):
    import torch
    from paper_1007_3818_gb300 import native
    s = _setup()
    f2, C1 = _rounded(s["f2"], mode), _rounded(s["C1"], mode)
    ref, _ = oracle.restrict(f2, C1, s["children"])
    d_c = _dev(C1, mode)
    children = native.records_to_device(s["children"], native.CF_CHILD_FIELDS, 24)
    native.restrict(mode, _dev(f2, mode), d_c, children)
    torch.cuda.synchronize()
    got = d_c.double().cpu().numpy()
    want = ref if mode == F64 else ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(got, want)


def test_invalid_records_are_counted_and_skipped_on_gpu():
    import torch
    from paper_1007_3818_gb300 import native
    s = _setup()
    faces = np.concatenate([s["faces"], s["faces"][:2]])
    faces[-2]["quadrant"] = 4
    faces[-1]["coarse"] = 8
    ref, nbad = oracle.flux_fixup(s["C1"], s["cflux"], s["ff"], s["dt"], s["dh"], faces)
    d_c = _dev(s["C1"], F64)
    dt = torch.full((8,), s["dt"], device="cuda", dtype=torch.float64)
    dh = torch.full((8,), s["dh"], device="cuda", dtype=torch.float64)
    bad = torch.zeros(1, device="cuda", dtype=torch.int32)
    native.flux_fixup(F64, d_c, _dev(s["cflux"], F64), _dev(s["ff"], F64), dt, dh,
                      native.records_to_device(faces, native.CF_FACE_FIELDS, 32), bad)
    children = np.concatenate([s["children"], s["children"][:1]])
    children[-1]["fine"] = -1
    native.restrict(F64, _dev(s["f2"], F64), d_c,
                    native.records_to_device(children, native.CF_CHILD_FIELDS, 24), bad)
    torch.cuda.synchronize()
    assert nbad == 2 and int(bad.item()) == 3
    ref2, _ = oracle.restrict(s["f2"], ref, s["children"])
    assert np.array_equal(d_c.cpu().numpy(), ref2)


@pytest.mark.parametrize("mode,tol", [(F32, TOL_F32_1), (F64, TOL_F64)], ids=["f32", "f64"])
def test_nine_plane_flux_layout(mode, tol):
    """flux_layout 1: the outer planes equal the six-face layout bit for bit,
    and all nine planes match the oracle's."""
    import torch
    from paper_1007_3818_gb300 import native
    tiles = host_input(wl.random_smooth_groups(5, seed=31, gamma=G), mode)
    T = torch.float64 if mode == F64 else torch.float32
    d_in = torch.from_numpy(tiles).to("cuda", T)
    N = tiles.shape[0]
    dt = torch.full((N,), 2e-3, device="cuda", dtype=torch.float64)
    dh = torch.full((N,), 1 / 256, device="cuda", dtype=torch.float64)
    out6 = torch.empty((N, 5, 16, 16, 16), device="cuda", dtype=T)
    out9 = torch.empty_like(out6)
    ff6 = torch.full((N, 6, 5, 16, 16), float("nan"), device="cuda", dtype=T)
    ff9 = torch.full((N, 9, 5, 16, 16), float("nan"), device="cuda", dtype=T)
    native.hydro_advance(mode, d_in, out6, ff6, dt, dh, None, None, native.make_params(G))
    native.hydro_advance(mode, d_in, out9, ff9, dt, dh, None, None,
                         native.make_params(G, flux_layout=1))
    torch.cuda.synchronize()
    a6, a9 = ff6.double().cpu().numpy(), ff9.double().cpu().numpy()
    assert torch.equal(out6, out9)
    assert np.array_equal(a9[:, [0, 2, 3, 5, 6, 8]], a6)
    _, r9, _, _ = oracle.advance_groups(tiles, 2e-3, 1 / 256, gamma=G, flux_layout=1)
    assert np.isfinite(a9).all()
    assert rel_l1_fields(a9.reshape(N * 9, 5, -1), r9.reshape(N * 9, 5, -1)) <= 10 * tol
    # value by value too, the interior planes (x8, y8, z8) included
    assert_elementwise(a9, r9, mode, "nine-plane face flux", state=False)


@pytest.mark.parametrize("mode,tol", [(F32, 2e-6), (F64, 1e-13)], ids=["f32", "f64"])
def test_two_level_step_on_gpu_is_conservative(mode, tol):
    """Coarse step (nine-plane fluxes), two fine sub-steps, fix-up and
    restriction, every kernel on the GPU: the composite totals are conserved
    (FP64 to round-off; FP32 to its storage precision)."""
    import torch
    from paper_1007_3818_gb300 import native
    s = _setup()
    T = torch.float64 if mode == F64 else torch.float32
    C, fine = _rounded(s["C"], mode), _rounded(s["fine"], mode)
    Nc, Nf = 8, len(REFINED)
    dt, dh = s["dt"], s["dh"]

    def vec(v, n):
        return torch.full((n,), v, device="cuda", dtype=torch.float64)

    d_C = _dev(C, mode)
    tiles = torch.empty((Nc, 5, 20, 20, 20), device="cuda", dtype=T)
    (native.gamer_fill_ghosts_uniform_f64 if mode == F64
     else native.gamer_fill_ghosts_uniform_f32)(d_C, tiles, 2, 2, 2, 0)
    C1 = torch.empty_like(d_C)
    cflux = torch.empty((Nc, 9, 5, 16, 16), device="cuda", dtype=T)
    native.hydro_advance(mode, tiles, C1, cflux, vec(dt, Nc), vec(dh, Nc), None, None,
                         native.make_params(G, flux_layout=1))
    ff = torch.empty((2, Nf, 6, 5, 16, 16), device="cuda", dtype=T)
    cur = fine
    for sub in range(2):
        ft = _dev(wl.fine_tiles(C, CG, cur, REFINED), mode)
        nxt = torch.empty((Nf, 5, 16, 16, 16), device="cuda", dtype=T)
        native.hydro_advance(mode, ft, nxt, ff[sub], vec(dt / 2, Nf), vec(dh / 2, Nf), None,
                             None, native.make_params(G))
        torch.cuda.synchronize()
        cur = nxt.double().cpu().numpy()
    d_f2 = _dev(cur, mode)
    bad = torch.zeros(1, device="cuda", dtype=torch.int32)
    native.flux_fixup(mode, C1, cflux, ff, vec(dt, Nc), vec(dh, Nc),
                      native.records_to_device(s["faces"], native.CF_FACE_FIELDS, 32), bad)
    native.restrict(mode, d_f2, C1,
                    native.records_to_device(s["children"], native.CF_CHILD_FIELDS, 24), bad)
    torch.cuda.synchronize()
    C2 = C1.double().cpu().numpy()
    assert int(bad.item()) == 0
    cov = np.zeros((Nc, 16, 16, 16), dtype=bool)
    for c in s["children"]:
        o = int(c["octant"])
        x, y, z = 8 * (o & 1), 8 * ((o >> 1) & 1), 8 * ((o >> 2) & 1)
        cov[c["coarse"], z:z + 8, y:y + 8, x:x + 8] = True
    before = np.array([C[:, q][~cov].sum() * 8.0 + fine[:, q].sum() for q in range(5)])
    after = np.array([C2[:, q].sum() * 8.0 for q in range(5)])
    scale = np.abs(before).max()
    assert np.all(np.abs(after - before) <= tol * scale), (after - before) / scale
