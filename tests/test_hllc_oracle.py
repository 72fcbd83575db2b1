"""Pins of the oracle's HLLC scheme variant (Toro 2009, Sec. 10.4): the
properties that define it -- consistency, exact resolution of isolated contact
and shear waves, upwinding, mirror symmetry -- and the whole scheme with HLLC
converging to the exact Riemann solution of the Sod and Lax tubes.  CPU only."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle_helpers import exact_cell_average_1d, l1, run_box
from paper_1007_3818_gb300 import workloads as wl


def _U(r, u, v, w, p, g):
    return np.array([r, r * u, r * v, r * w, p / (g - 1) + 0.5 * r * (u * u + v * v + w * w)])


def _F(d, r, vel, p, g):
    """Closed-form Euler flux in direction d."""
    un = vel[d]
    E = p / (g - 1) + 0.5 * r * sum(x * x for x in vel)
    F = np.array([r * un, r * un * vel[0], r * un * vel[1], r * un * vel[2], un * (E + p)])
    F[1 + d] += p
    return F


def _vel(d, n, t1, t2):
    """Velocity vector with normal component n and tangential t1, t2 (cyclic)."""
    v = [0.0, 0.0, 0.0]
    v[d], v[(d + 1) % 3], v[(d + 2) % 3] = n, t1, t2
    return v


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_consistency(d):
    g = 5.0 / 3.0
    vel = (0.3, -0.7, 1.1)
    U = _U(1.3, *vel, 0.8, g)
    assert np.allclose(oracle.hllc_flux(d, U, U, g), _F(d, 1.3, vel, 0.8, g), rtol=1e-14,
                       atol=1e-15)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_resolves_stationary_contact_and_shear_exactly(d):
    """u = 0, equal pressures, different densities and tangential velocities:
    the exact flux is (0, p along d, 0, 0, 0).  HLLC returns it; HLLE smears
    (non-zero mass and tangential-momentum flux), which shows the test bites."""
    g = 1.4
    vl, vr = _vel(d, 0.0, 1.0, -0.5), _vel(d, 0.0, -1.0, 0.25)
    UL, UR = _U(1.0, *vl, 1.0, g), _U(0.2, *vr, 1.0, g)
    F = oracle.hllc_flux(d, UL, UR, g)
    want = np.zeros(5)
    want[1 + d] = 1.0
    assert np.abs(F - want).max() <= 1e-14
    H = oracle.hlle_flux(d, UL, UR, g)
    assert abs(H[0]) > 1e-3 and abs(H[1 + (d + 1) % 3]) > 1e-3


@pytest.mark.parametrize("un", [0.5, -0.5])
def test_hllc_moving_contact_is_upwinded(un):
    g = 1.4
    d = 1
    vl, vr = _vel(d, un, 0.3, 0.0), _vel(d, un, -0.2, 0.1)
    UL, UR = _U(1.0, *vl, 0.7, g), _U(0.3, *vr, 0.7, g)
    F = oracle.hllc_flux(d, UL, UR, g)
    up = _F(d, 1.0, vl, 0.7, g) if un > 0 else _F(d, 0.3, vr, 0.7, g)
    assert np.abs(F - up).max() <= 1e-13 * np.abs(up).max()


def test_hllc_supersonic_is_pure_upwind():
    g = 1.4
    vl, vr = (4.0, 0.2, 0.0), (3.5, -0.1, 0.3)
    UL, UR = _U(1.0, *vl, 1.0, g), _U(0.5, *vr, 0.4, g)
    assert np.array_equal(oracle.hllc_flux(0, UL, UR, g), oracle.hllc_flux(0, UL, UL, g))
    UL2, UR2 = _U(1.0, -4.0, 0.2, 0.0, 1.0, g), _U(0.5, -3.5, -0.1, 0.3, 0.4, g)
    assert np.array_equal(oracle.hllc_flux(0, UL2, UR2, g), oracle.hllc_flux(0, UR2, UR2, g))


@pytest.mark.parametrize("d", [0, 1, 2])
def test_hllc_mirror_symmetry(d):
    """Mirroring across the face swaps the states and flips the normal
    velocity: mass, tangential-momentum and energy fluxes change sign, the
    normal-momentum flux does not."""
    g = 5.0 / 3.0
    rng = np.random.default_rng(d + 3)
    for _ in range(20):
        WL = (rng.uniform(0.2, 2), *rng.uniform(-2, 2, 3), rng.uniform(0.1, 3))
        WR = (rng.uniform(0.2, 2), *rng.uniform(-2, 2, 3), rng.uniform(0.1, 3))
        UL, UR = _U(*WL, g), _U(*WR, g)
        F = oracle.hllc_flux(d, UL, UR, g)

        def mirror(U):
            M = U.copy()
            M[1 + d] = -M[1 + d]
            return M
        Fm = oracle.hllc_flux(d, mirror(UR), mirror(UL), g)
        want = -F
        want[1 + d] = F[1 + d]
        assert np.allclose(Fm, want, rtol=1e-12, atol=1e-13 * np.abs(F).max())


@pytest.mark.parametrize("tube,bounds", [(wl.SOD, (3e-2, 3e-3)), (wl.LAX, (8e-2, 1.2e-2))],
                         ids=["sod", "lax"])
def test_hllc_scheme_converges_on_shock_tubes(tube, bounds):
    g = 1.4
    t_end = 0.2 if tube is wl.SOD else 0.13
    errs = []
    ns = (16, 32, 64, 128)
    for n in ns:
        U, st = run_box(wl.shock_tube_level(n, *tube, g), t_end, 1.0 / n, g, riemann=1)
        errs.append(l1(U[0, 0, 0], exact_cell_average_1d(tube[0], tube[1], g, n, t_end)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert min(orders) >= 0.6, (errs, orders)
    assert errs[0] <= bounds[0], errs


def test_hllc_scheme_preserves_uniform_state_and_differs_from_roe():
    g = 5.0 / 3.0
    U = _U(1.2, 0.3, -0.4, 0.2, 0.9, g)
    tile = np.broadcast_to(U[:, None, None, None], (5, 20, 20, 20)).copy()
    out, _, st, _ = oracle.advance_groups(tile[None], 1e-2, 1 / 64, gamma=g, riemann=1)
    assert np.array_equal(out[0], tile[:, 2:18, 2:18, 2:18]) and st[0] == 0
    # on a smooth state the two solvers differ by far less than the step itself
    t = wl.random_smooth_groups(1, seed=5, gamma=g)
    a = oracle.advance_groups(t, 2e-3, 1 / 256, gamma=g)[0]
    b = oracle.advance_groups(t, 2e-3, 1 / 256, gamma=g, riemann=1)[0]
    step = np.abs(a - t[:, :, 2:18, 2:18, 2:18]).sum()
    assert not np.array_equal(a, b) and np.abs(a - b).sum() <= 1e-2 * step
