"""Pins of the oracle's operation counter (the numerator of the ALU roofline)
against hand counts.

Each scheme piece is tallied on the counting scalar and compared with a count
made by hand from the formulas of the scheme's readings (Sec. 2 of the paper
names the four stages; the readings R1-R8 fix their formulas).  Then one whole
16^3 group on a uniform state -- where every branch is known: slopes are zero,
no fallback fires, the entropy fix's smoothing does not apply -- must tally
exactly the sum of the pieces times the number of times the step runs each
(8,000 conversions, 5,632 predictions, 13,056 Riemann solves, 4,096 updates).
Dropping an operation kind from the tally, or a stage from the step, fails
here; the earlier order-of-magnitude bound could not tell."""
from __future__ import annotations

import numpy as np
import pytest

import oracle

G = 5.0 / 3.0


def _c(add=0, mul=0, div=0, sqrt=0):
    return {"add": add, "mul": mul, "div": div, "sqrt": sqrt}


def _sum(*terms):
    out = _c()
    for k, t in terms:
        for key in out:
            out[key] += k * t[key]
    return out


def _flops(d):
    return {k: d[k] for k in ("add", "mul", "div", "sqrt")}


# --- hand counts, formula by formula ----------------------------------------
# prim: v_d = m_d / rho (3 div); ke = 0.5 (mx^2 + my^2 + mz^2) / rho (4 mul,
# 2 add, 1 div); p = (gamma - 1)(E - ke) (1 mul, 1 add)
PRIM = _c(add=3, mul=5, div=4)
# cons: m_d = rho v_d (3 mul); E = p / (gamma - 1) + (0.5 rho)(vx^2 + vy^2 +
# vz^2) (1 div, 5 mul, 3 add)
CONS = _c(add=3, mul=8, div=1)
# Euler flux along d: m = rho u_n (1 mul); m v (3 mul); + p on the normal
# component (1 add); (E + p) u_n (1 add, 1 mul)
FLUX = _c(add=2, mul=5)
# van Leer: a b (1 mul, tested); when a b > 0: (2 a) b / (a + b) (2 mul, 1 add,
# 1 div)
VL_ACTIVE = _c(add=1, mul=3, div=1)
VL_ZERO = _c(mul=1)
# admissibility rho > 0 and p > 0, p as in prim without the velocities
POSITIVE = _c(add=3, mul=5, div=1)
# Harten's smoothing of one acoustic eigenvalue where it applies:
# (l^2 + d^2) / (2 d) (3 mul, 1 add, 1 div)
FIX_BRANCH = _c(add=1, mul=3, div=1)
# One Roe flux with the entropy fix, no fallback, no smoothing applied:
ROE = _sum(
    (2, PRIM), (2, FLUX),                      # W_L, W_R and F_L, F_R
    (1, _c(mul=2, div=2, sqrt=2)),             # c_L, c_R = sqrt(gamma p / rho)
    (1, _c(add=2, div=2)),                     # H_L, H_R = (E + p) / rho
    (1, _c(div=1, sqrt=1)),                    # R = sqrt(rho_R / rho_L)
    (4, _c(add=2, mul=1, div=1)),              # u~, v~, w~, H~ = (a + R b) / (1 + R)
    (1, _c(add=2, mul=3)),                     # q2 = |v~|^2
    (1, _c(add=1, mul=2)),                     # c~^2 = (gamma - 1)(H~ - 0.5 q2)
    (1, _c(sqrt=1)),                           # c~
    (1, _c(mul=1)),                            # rho~ = R rho_L
    (1, _c(add=5)),                            # jumps of rho, u, v, w, p
    (2, _c(add=1, mul=3, div=1)),              # alpha_1, alpha_5
    (1, _c(add=1, div=1)),                     # alpha_2 = drho - dp / c~^2
    (2, _c(mul=1)),                            # alpha_3, alpha_4
    (2, _c(add=2, mul=1)),                     # K1, K5 (u~ -/+ c~, H~ -/+ u~ c~)
    (10, _c(add=1, mul=1)),                    # U*_L = U_L + a1 K1, U*_R = U_R - a5 K5
    (2, POSITIVE),                             # fallback test of both
    (1, _c(add=2)),                            # lambda_1, lambda_5
    (2, PRIM),                                 # the intermediate states' primitives
    (2, _c(add=1, mul=1, div=1, sqrt=1)),      # their lambda_1, lambda_5
    (2, _c(add=3)),                            # Harten-Hyman widths d1, d5
    (1, _c(mul=5)),                            # s_k = |lambda_k| alpha_k
    (1, _c(add=2)),                            # D0
    (1, _c(add=2, mul=3)),                     # D1
    (2, _c(add=3, mul=3)),                     # D2, D3
    (1, _c(add=4, mul=6)),                     # D4 (with 0.5 q2)
    (5, _c(add=2, mul=2)),                     # F = 0.5 (F_L + F_R) - 0.5 D
)
# One Hancock prediction of a cell on a uniform state (all slopes zero):
PRED_UNIFORM = _sum(
    (15, _c(add=2)), (15, VL_ZERO),            # 3 x 5 limited slopes of two differences
    (30, _c(add=1, mul=1)),                    # face values W -/+ 0.5 slope
    (6, CONS), (6, FLUX),                      # six face states and their fluxes
    (15, _c(add=2)),                           # acc += F(W-) - F(W+), 3 directions x 5
    (30, _c(add=1, mul=1)),                    # six evolved states U + (lambda/2) acc
    (6, POSITIVE),                             # their admissibility
)
# Update of one cell and its epilogue: acc = sum of three flux differences
# (5 x 5 add); U - lambda acc (5 mul, 5 add); prim of the result; c^2 =
# gamma p / rho (1 mul, 1 div), c (1 sqrt), max |v_d| + c (1 add); the five
# conserved sums (5 add)
UPDATE = _sum((1, _c(add=30, mul=5)), (1, PRIM), (1, _c(add=6, mul=1, div=1, sqrt=1)))
# lambda = dt / dh and lambda / 2 once per group
GROUP_ONCE = _c(mul=1, div=1)


def test_piece_counts_match_hand_counts():
    W = np.array([1.7, 0.4, -1.3, 0.25, 0.6])
    U = oracle.cons(W, G)
    assert _flops(oracle.count_ops_piece("prim", U)) == PRIM
    assert _flops(oracle.count_ops_piece("cons", W)) == CONS
    for d in range(3):
        assert _flops(oracle.count_ops_piece("flux", W, [U[4]], d=d)) == FLUX
    assert _flops(oracle.count_ops_piece("limiter", [0.3], [0.7])) == VL_ACTIVE
    assert _flops(oracle.count_ops_piece("limiter", [0.3], [-0.7])) == VL_ZERO
    assert _flops(oracle.count_ops_piece("positive", U)) == POSITIVE
    # a smooth face: no fallback, no smoothing (|lambda| well above the widths)
    UL = oracle.cons(np.array([1.0, 0.3, 0.1, -0.2, 1.0]), G)
    UR = oracle.cons(np.array([1.1, 0.25, 0.12, -0.18, 1.05]), G)
    for d in range(3):
        F, used = oracle.roe_flux(d, UL, UR, G)
        assert not used
        assert _flops(oracle.count_ops_piece("roe", UL, UR, d=d)) == ROE


def test_roe_count_adds_the_smoothing_where_it_applies():
    # a transonic expansion: the right state lies on the 1-rarefaction curve
    # through the left one and u - c changes sign across it, so the smoothing
    # applies to lambda_1 (and not to lambda_5, far from sonic)
    g = 1.4
    rL, uL, pL, pR = 1.0, 0.8, 1.0, 0.3
    cL = np.sqrt(g * pL / rL)
    rR = rL * (pR / pL) ** (1 / g)
    cR = np.sqrt(g * pR / rR)
    uR = uL + 2 / (g - 1) * (cL - cR)
    assert uL - cL < 0 < uR - cR
    UL = oracle.cons(np.array([rL, uL, 0.0, 0.0, pL]), g)
    UR = oracle.cons(np.array([rR, uR, 0.0, 0.0, pR]), g)
    F, used = oracle.roe_flux(0, UL, UR, g)
    assert not used
    got = _flops(oracle.count_ops_piece("roe", UL, UR, gamma=g))
    extra = {k: got[k] - ROE[k] for k in ROE}
    assert extra == FIX_BRANCH, extra
    # the same expansion moved far from the sonic point: the plain count
    UL2 = oracle.cons(np.array([rL, uL + 5, 0.0, 0.0, pL]), g)
    UR2 = oracle.cons(np.array([rR, uR + 5, 0.0, 0.0, pR]), g)
    assert _flops(oracle.count_ops_piece("roe", UL2, UR2, gamma=g)) == ROE


def test_whole_group_tally_is_the_sum_of_its_pieces():
    W = np.array([1.7, 0.4, -1.3, 0.25, 0.6])
    U = oracle.cons(W, G)
    tile = np.broadcast_to(U[:, None, None, None], (5, 20, 20, 20)).copy()
    counts = oracle.count_ops_group(tile, 1e-3, 1 / 64, gamma=G)
    want = _sum((1, GROUP_ONCE), (8000, PRIM), (5632, PRED_UNIFORM), (13056, ROE),
                (4096, UPDATE))
    assert _flops(counts) == want, (_flops(counts), want)
    assert counts["cells"] == 4096


def test_counting_scalar_on_a_smooth_group_is_within_the_uniform_bounds():
    """On a smooth, non-uniform group the slopes are active (each limited
    slope adds VL_ACTIVE - VL_ZERO) and a few faces may apply the smoothing;
    the tally lies between the uniform-state count and that count plus every
    slope active and every face smoothed twice."""
    from paper_1007_3818_gb300 import workloads as wl
    tile = wl.random_smooth_groups(1, seed=9, gamma=G)[0]
    got = _flops(oracle.count_ops_group(tile, 2e-3, 1 / 256, gamma=G))
    lo = _sum((1, GROUP_ONCE), (8000, PRIM), (5632, PRED_UNIFORM), (13056, ROE), (4096, UPDATE))
    slope_extra = {k: VL_ACTIVE[k] - VL_ZERO[k] for k in lo}
    hi = _sum((1, lo), (5632 * 15, slope_extra), (2 * 13056, FIX_BRANCH))
    for k in lo:
        assert lo[k] <= got[k] <= hi[k], (k, lo[k], got[k], hi[k])
    # most slopes of a smooth field are active
    assert got["div"] - lo["div"] > 0.5 * 5632 * 15
