"""Pins of the oracle's coarse-fine coupling (flux fix-up and restriction),
against properties the mathematics fixes: conservation of the composite
two-level state (the purpose of refluxing, Berger & Colella 1989), identity
on states where coarse and fine fluxes agree, and exact averages.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1007_3818_gb300 import workloads as wl

G = 5.0 / 3.0


def _covered(children, Nc):
    cov = np.zeros((Nc, 16, 16, 16), dtype=bool)
    for c in children:
        o = int(c["octant"])
        x, y, z = 8 * (o & 1), 8 * ((o >> 1) & 1), 8 * ((o >> 2) & 1)
        cov[c["coarse"], z:z + 8, y:y + 8, x:x + 8] = True
    return cov


def _composite_totals(coarse, fine, cov):
    """Totals of the composite state in fine-cell volumes: uncovered coarse
    cells count 8 times, fine cells once."""
    return np.array([coarse[:, q][~cov].sum() * 8.0 + fine[:, q].sum() for q in range(5)])


def _two_level_step(cg, refined, seed, with_fixup=True):
    """One coarse step, two fine sub-steps, fix-up and restriction, all through
    the oracle.  Returns (totals before, totals after, coarse after, fine
    after, children, faces)."""
    children, faces = wl.cf_records(cg, refined)
    cgx, cgy, cgz = cg
    Nc = cgx * cgy * cgz
    rng = np.random.default_rng(seed)
    assert cgx == cgy == cgz, "a cubic coarse level"
    C = wl.level_to_groups(wl.fourier_level(n=16 * cgx, seed=seed, gamma=G))
    F = wl.composite_fine_level(C, cg, np.zeros((0, 5, 16, 16, 16)), [])
    fine = np.stack([F[:, 16 * p[2]:16 * p[2] + 16, 16 * p[1]:16 * p[1] + 16,
                       16 * p[0]:16 * p[0] + 16] for p in refined]).copy()
    fine[:, 0] *= 1.0 + 0.05 * rng.standard_normal(fine[:, 0].shape)   # fine structure
    cov = _covered(children, Nc)
    before = _composite_totals(C, fine, cov)
    dh = 1.0 / (16 * cgx)
    dt = 0.3 * dh / 2.0
    C1, cflux, _, _ = oracle.advance_groups(oracle.fill_ghosts_uniform(C, cgx, cgy, cgz, 0), dt,
                                            dh, gamma=G, flux_layout=1)
    f1, ff1, _, _ = oracle.advance_groups(wl.fine_tiles(C, cg, fine, refined), dt / 2, dh / 2,
                                          gamma=G)
    f2, ff2, _, _ = oracle.advance_groups(wl.fine_tiles(C, cg, f1, refined), dt / 2, dh / 2,
                                          gamma=G)
    if with_fixup:
        C1, bad = oracle.flux_fixup(C1, cflux, np.stack([ff1, ff2]), dt, dh, faces)
        assert bad == 0
    C2, bad = oracle.restrict(f2, C1, children)
    assert bad == 0
    return before, _composite_totals(C2, f2, cov), C2, f2, children, faces


@pytest.mark.parametrize("refined", [
    [(1, 1, 1)],                          # one patch, inner corner of group 0
    [(1, 1, 1), (2, 1, 1)],               # two adjacent patches in two groups
    [(0, 3, 2), (3, 3, 2), (0, 0, 1)],    # patches on the periodic boundary
])
def test_fixup_makes_the_two_level_step_conservative(refined):
    before, after, C2, f2, children, faces = _two_level_step((2, 2, 2), refined, seed=11)
    scale = np.abs(before).max()
    assert np.all(np.abs(after - before) <= 1e-14 * scale), (after - before) / scale
    # restriction: the coarse level alone then carries the same totals
    coarse_tot = np.array([C2[:, q].sum() * 8.0 for q in range(5)])
    assert np.all(np.abs(coarse_tot - after) <= 1e-14 * scale)
    # without the fix-up the composite state is not conserved
    b0, a0, *_ = _two_level_step((2, 2, 2), refined, seed=11, with_fixup=False)
    assert np.abs(a0 - b0).max() > 1e-9 * scale


def test_records_cover_every_coarse_fine_interface():
    refined = [(1, 1, 1), (2, 1, 1), (2, 2, 1)]
    children, faces = wl.cf_records((2, 2, 2), refined)
    # 6 faces per fine group minus 2 per adjacent fine pair: (1,1,1)-(2,1,1), (2,1,1)-(2,2,1)
    assert len(faces) == 6 * 3 - 2 * 2
    assert children["octant"].tolist() == [7, 6, 4]
    # every record names a valid coarse layer next to a fine patch
    for f in faces:
        assert (f["side"] == 1 and f["plane"] >= 1) or (f["side"] == 0 and f["plane"] <= 1)


def test_fixup_is_identity_when_fine_and_coarse_fluxes_agree():
    """A uniform state: every face flux is F(U), the fine mean equals it
    exactly, so the correction is exactly zero."""
    cg, refined = (2, 2, 2), [(1, 1, 1), (3, 0, 2)]
    children, faces = wl.cf_records(cg, refined)
    U = oracle.cons(np.array([1.3, 0.4, -0.2, 0.7, 2.0]), G)
    C = np.broadcast_to(U[None, :, None, None, None], (8, 5, 16, 16, 16)).copy()
    fine = np.broadcast_to(U[None, :, None, None, None], (2, 5, 16, 16, 16)).copy()
    C1, cflux, _, _ = oracle.advance_groups(oracle.fill_ghosts_uniform(C, 2, 2, 2, 0), 1e-3,
                                            1 / 32, gamma=G, flux_layout=1)
    f1, ff1, _, _ = oracle.advance_groups(wl.fine_tiles(C, cg, fine, refined), 5e-4, 1 / 64,
                                          gamma=G)
    out, bad = oracle.flux_fixup(C1, cflux, np.stack([ff1, ff1]), 1e-3, 1 / 32, faces)
    assert bad == 0 and np.array_equal(out, C1) and np.array_equal(C1, C)


def test_restriction_is_the_exact_mean():
    rng = np.random.default_rng(3)
    cg, refined = (1, 1, 2), [(0, 1, 3), (1, 0, 0)]
    children, _ = wl.cf_records(cg, refined)
    # FP32-representable values: the 8-term sums are exact in FP64
    coarse = rng.standard_normal((2, 5, 16, 16, 16)).astype(np.float32).astype(np.float64)
    # injected fine groups (each coarse value repeated 2x2x2) restrict to the coarse values
    inj = wl.composite_fine_level(coarse, cg, np.zeros((0, 5, 16, 16, 16)), [])
    fine = np.stack([inj[:, 16 * p[2]:16 * p[2] + 16, 16 * p[1]:16 * p[1] + 16,
                         16 * p[0]:16 * p[0] + 16] for p in refined])
    out, bad = oracle.restrict(fine, np.zeros_like(coarse), children)
    cov = _covered(children, 2)
    assert bad == 0 and np.array_equal(out[:, :][np.broadcast_to(cov[:, None], out.shape)],
                                       coarse[np.broadcast_to(cov[:, None], out.shape)])
    assert not out[np.broadcast_to(~cov[:, None], out.shape)].any()   # untouched
    # a linear field in every direction restricts to its value at the coarse centre
    z, y, x = np.meshgrid(*(np.arange(16.0),) * 3, indexing="ij")
    lin = np.broadcast_to((1.0 + 0.5 * x - 0.25 * y + 0.125 * z)[None, None], (2, 5, 16, 16, 16))
    out, _ = oracle.restrict(lin, np.zeros_like(coarse), children)
    zc, yc, xc = np.meshgrid(*(np.arange(8.0),) * 3, indexing="ij")
    want = 1.0 + 0.5 * (2 * xc + 0.5) - 0.25 * (2 * yc + 0.5) + 0.125 * (2 * zc + 0.5)
    o = int(children[0]["octant"])
    x0, y0, z0 = 8 * (o & 1), 8 * ((o >> 1) & 1), 8 * ((o >> 2) & 1)
    assert np.array_equal(out[children[0]["coarse"], 2, z0:z0 + 8, y0:y0 + 8, x0:x0 + 8], want)


def test_invalid_records_are_counted_and_skipped():
    cg, refined = (2, 2, 2), [(1, 1, 1)]
    children, faces = wl.cf_records(cg, refined)
    rng = np.random.default_rng(5)
    C = rng.standard_normal((8, 5, 16, 16, 16))
    cflux = rng.standard_normal((8, 9, 5, 16, 16))
    ff = rng.standard_normal((2, 1, 6, 5, 16, 16))
    good, bad = oracle.flux_fixup(C, cflux, ff, 1e-3, 1 / 32, faces)
    broken = np.concatenate([faces, faces[:3]])
    broken[-3]["dir"] = 3
    broken[-2]["fine"] = 1           # only one fine group
    broken[-1]["plane"] = 0          # side 1 needs plane >= 1
    broken[-1]["side"] = 1
    out, nbad = oracle.flux_fixup(C, cflux, ff, 1e-3, 1 / 32, broken)
    assert bad == 0 and nbad == 3 and np.array_equal(out, good)
    ch = np.concatenate([children, children])
    ch[1]["octant"] = 8
    r, nb = oracle.restrict(rng.standard_normal((1, 5, 16, 16, 16)), C, ch)
    assert nb == 1


@pytest.mark.parametrize("patch", [(1, 2, 1), (0, 3, 2)])
def test_fixup_lands_on_the_coarse_cell_beside_each_fine_face(patch):
    """A unit flux on one fine face (coarse fluxes zero): exactly one coarse
    cell changes, by -s * lam / (4 n_sub), and it is the coarse cell adjacent
    to that fine face in global coordinates (periodic wrap)."""
    cg = (2, 2, 2)
    children, faces = wl.cf_records(cg, [patch])
    assert len(faces) == 6
    rng = np.random.default_rng(17)
    n = 32                                   # coarse level edge in cells
    lam = 1e-3 / (1 / 32)
    for face in range(6):
        d, hi = face // 2, face % 2          # the fine group's face: direction, + side?
        A, B = (int(v) for v in rng.integers(0, 16, size=2))
        ff = np.zeros((2, 1, 6, 5, 16, 16))
        ff[1, 0, face, 3, A, B] = 1.0
        C0 = np.zeros((8, 5, 16, 16, 16))
        out, bad = oracle.flux_fixup(C0, np.zeros((8, 9, 5, 16, 16)), ff, 1e-3, 1 / 32, faces)
        lvl = wl.groups_to_level(out, *cg)[3]
        changed = np.argwhere(lvl != 0.0)
        # geometry: fine face plane and in-plane fine cell -> coarse neighbour
        fine0 = [16 * patch[0], 16 * patch[1], 16 * patch[2]]   # fine-cell origin (x, y, z)
        tz, ty = {0: (2, 1), 1: (2, 0), 2: (1, 0)}[d]             # [A][B] axes
        pos = [None, None, None]
        pos[tz], pos[ty] = (fine0[tz] + A) // 2, (fine0[ty] + B) // 2
        pos[d] = (fine0[d] // 2 - 1) if hi == 0 else (fine0[d] // 2 + 8)
        pos = [p % n for p in pos]
        s = 1.0 if hi == 0 else -1.0          # fine region on the + side of the cell for a - face
        assert bad == 0 and changed.tolist() == [[pos[2], pos[1], pos[0]]], (face, changed, pos)
        assert lvl[pos[2], pos[1], pos[0]] == -s * lam * (1.0 / 8.0)
