"""FP64 CPU oracle of the MUSCL-Hancock + Roe hydro step -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The CUDA product path never does: it shares no code with
the oracle and fails loudly when its own extension is missing.

The arithmetic lives in ``gamer_oracle.cpp`` (plain C++, FP64, compiled with
``-O2 -ffp-contract=off`` so each operation is rounded as written).  This
module only builds that file and marshals numpy arrays through ctypes.

Method (paper Sec. 2): MUSCL-Hancock (Toro 2009) with Roe's Riemann solver
(Roe 1981); unsplit; four stages (reconstruction, half-step prediction, Riemann
solver, full-step update); five-point stencil per direction.  The readings
taken where the paper is silent are listed at the top of ``gamer_oracle.cpp``.

Pins (tests/test_oracle_pins.py, test_hllc_oracle.py, test_char_oracle.py,
test_amr_oracle.py, test_host_fill_cpu.py): exact Riemann star values for Sod
(textbook), Rankine-Hugoniot and Riemann-invariant residuals, Roe's exactness
on isolated shocks and stationary contacts, HLLE limits, limiter closed forms,
exact preservation of uniform states, conservation on periodic boxes,
permutation and mirror symmetry, L1 convergence on Sod / Lax, second-order
convergence on a linear sound wave, ghost-independence of unread corner cells;
the floors' closed forms; HLLC's exactness on isolated contact and shear
waves, upwinding and consistency; characteristic limiting reducing to the
primitive scheme on an entropy wave and limiting single waves along their
eigenvectors; composite conservation, locality and exact means of the
coarse-fine fix-up and restriction; the ghost fill against index arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gamer_oracle.cpp")
_HDR = os.path.join(_HERE, "gamer_oracle.h")
_SO = os.path.join(_HERE, "libgamer_oracle.so")
_lock = threading.Lock()
_lib = None

ST_PREDICTOR_FALLBACK = 1
ST_HLLE_FALLBACK = 2
ST_NONPOSITIVE_OUT = 4
ST_BAD_INPUT = 8
ST_FLOOR = 32


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, no GPU needed)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("limiter", ctypes.c_int32),
                ("predictor_fallback", ctypes.c_int32), ("rho_floor", ctypes.c_double),
                ("p_floor", ctypes.c_double), ("flux_layout", ctypes.c_int32),
                ("riemann", ctypes.c_int32), ("reconstruction", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        pd, pu32, pi32 = P(d), P(ctypes.c_uint32), P(i32)
        lib.oracle_advance_box.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int, pd, pd, d,
                                           d, P(_Params), pu32, pd]
        lib.oracle_advance_groups.argtypes = [pd, pd, pd, pd, pd, i64, P(_Params), pu32, pd,
                                              ctypes.c_int]
        lib.oracle_fill_ghosts_uniform.argtypes = [pd, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, pd]
        lib.oracle_hydro_dt.argtypes = [pd, i64, pi32, i32, pd, d, pd, pd]
        lib.oracle_prim_from_cons.argtypes = [pd, d, pd]
        lib.oracle_cons_from_prim.argtypes = [pd, d, pd]
        lib.oracle_euler_flux.argtypes = [ctypes.c_int, pd, d, pd]
        lib.oracle_limiter.argtypes = [ctypes.c_int, d, d]
        lib.oracle_limiter.restype = d
        lib.oracle_roe_flux.argtypes = [ctypes.c_int, pd, pd, d, ctypes.c_int, pd]
        lib.oracle_hlle_flux.argtypes = [ctypes.c_int, pd, pd, d, pd]
        lib.oracle_hllc_flux.argtypes = [ctypes.c_int, pd, pd, d, pd]
        lib.oracle_char_slopes.argtypes = [ctypes.c_int, pd, pd, pd, d, ctypes.c_int, pd]
        lib.oracle_exact_riemann_star.argtypes = [d, d, d, d, d, d, d, pd]
        lib.oracle_exact_riemann_sample.argtypes = [d, d, d, d, d, d, d, d, pd]
        lib.oracle_count_ops_group.argtypes = [pd, d, d, P(_Params), pd]
        lib.oracle_count_ops_piece.argtypes = [ctypes.c_int, ctypes.c_int, pd, pd, d, pd]
        vp = ctypes.c_void_p
        lib.oracle_flux_fixup.argtypes = [pd, pd, pd, ctypes.c_int, pd, pd, i64, i64, vp, i64]
        lib.oracle_flux_fixup.restype = i64
        lib.oracle_restrict.argtypes = [pd, pd, i64, i64, vp, i64]
        lib.oracle_restrict.restype = i64
        for name in ("oracle_advance_box", "oracle_advance_groups", "oracle_fill_ghosts_uniform",
                     "oracle_hydro_dt", "oracle_roe_flux", "oracle_exact_riemann_star",
                     "oracle_count_ops_group", "oracle_count_ops_piece"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _params(gamma, limiter, predictor_fallback, rho_floor=0.0, p_floor=0.0, flux_layout=0,
            riemann=0, reconstruction=0):
    return _Params(float(gamma), int(limiter), int(predictor_fallback), float(rho_floor),
                   float(p_floor), int(flux_layout), int(riemann), int(reconstruction))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def advance_box(U_in, dt, dh, gamma=1.4, limiter=0, predictor_fallback=0, rho_floor=0.0,
                p_floor=0.0, flux_layout=0, riemann=0, reconstruction=0):
    """One step on a ghost-padded box U_in[5][nz+4][ny+4][nx+4].

    Returns (out[5][nz][ny][nx], face_flux (list of 6 arrays: -x, +x, -y, +y,
    -z, +z; or of 9 with flux_layout=1: x at 0, nx/2, nx, then y, then z),
    status, partials[6])."""
    U_in = _f64(U_in)
    _, pz, py, px = U_in.shape
    nx, ny, nz = px - 4, py - 4, pz - 4
    out = np.empty((5, nz, ny, nx))
    per = 3 if flux_layout == 1 else 2
    ff = np.empty(per * 5 * (nz * ny + nz * nx + ny * nx))
    st = np.zeros(1, dtype=np.uint32)
    part = np.empty(6)
    p = _params(gamma, limiter, predictor_fallback, rho_floor, p_floor, flux_layout, riemann,
                reconstruction)
    rc = _load().oracle_advance_box(_ptr(U_in), nx, ny, nz, _ptr(out), _ptr(ff), float(dt),
                                    float(dh), ctypes.byref(p), _ptr(st, ctypes.c_uint32),
                                    _ptr(part))
    if rc != 0:
        raise ValueError(f"oracle_advance_box rejected its arguments (rc={rc})")
    faces, o = [], 0
    for shape in ((5, nz, ny),) * per + ((5, nz, nx),) * per + ((5, ny, nx),) * per:
        n = int(np.prod(shape))
        faces.append(ff[o:o + n].reshape(shape))
        o += n
    return out, faces, int(st[0]), part


def advance_groups(U_in, dt, dh, gamma=1.4, limiter=0, predictor_fallback=0, nthreads=1,
                   want_flux=True, rho_floor=0.0, p_floor=0.0, flux_layout=0, riemann=0,
                   reconstruction=0):
    """N independent patch groups U_in[N][5][20][20][20] (dt, dh scalars or [N]).

    Returns (out[N][5][16][16][16], face_flux[N][6 or 9][5][16][16] or None,
    status[N] uint32, partials[N][6])."""
    U_in = _f64(U_in)
    N = U_in.shape[0]
    assert U_in.shape[1:] == (5, 20, 20, 20), U_in.shape
    dt = _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (N,)))
    dh = _f64(np.broadcast_to(np.asarray(dh, dtype=np.float64), (N,)))
    out = np.empty((N, 5, 16, 16, 16))
    ff = np.empty((N, 9 if flux_layout == 1 else 6, 5, 16, 16)) if want_flux else None
    st = np.zeros(N, dtype=np.uint32)
    part = np.empty((N, 6))
    p = _params(gamma, limiter, predictor_fallback, rho_floor, p_floor, flux_layout, riemann,
                reconstruction)
    rc = _load().oracle_advance_groups(_ptr(U_in), _ptr(out), _ptr(ff), _ptr(dt), _ptr(dh), N,
                                       ctypes.byref(p), _ptr(st, ctypes.c_uint32), _ptr(part),
                                       int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_advance_groups rejected its arguments (rc={rc})")
    return out, ff, st, part


def _records(a, names, itemsize):
    a = np.ascontiguousarray(a)
    assert a.dtype.names == names and a.dtype.itemsize == itemsize, a.dtype
    return a


def flux_fixup(coarse, coarse_flux, fine_flux, dt, dh, faces):
    """Coarse-fine flux fix-up on a copy of coarse[Nc][5][16][16][16].

    coarse_flux[Nc][9][5][16][16] (nine-plane layout), fine_flux
    [n_sub][Nf][6][5][16][16] (the fine groups' sub-steps), dt, dh [Nc] (or
    scalars), faces: records (coarse, fine, dir, plane, side, quadrant).
    Returns (corrected coarse, number of invalid records)."""
    out = _f64(coarse).copy()
    Nc = out.shape[0]
    cf = _f64(coarse_flux)
    ff = _f64(fine_flux)
    n_sub, Nf = ff.shape[0], ff.shape[1]
    assert cf.shape == (Nc, 9, 5, 16, 16) and ff.shape[2:] == (6, 5, 16, 16)
    dt = _f64(np.broadcast_to(np.asarray(dt, dtype=np.float64), (Nc,)))
    dh = _f64(np.broadcast_to(np.asarray(dh, dtype=np.float64), (Nc,)))
    faces = _records(faces, ("coarse", "fine", "dir", "plane", "side", "quadrant"), 32)
    bad = _load().oracle_flux_fixup(_ptr(out), _ptr(cf), _ptr(ff), int(n_sub), _ptr(dt),
                                    _ptr(dh), Nc, Nf, faces.ctypes.data_as(ctypes.c_void_p),
                                    len(faces))
    if bad < 0:
        raise ValueError("oracle_flux_fixup rejected its arguments")
    return out, int(bad)


def restrict(fine, coarse, children):
    """Restriction of fine[Nf][5][16]^3 into a copy of coarse[Nc][5][16]^3 by
    the child records (coarse, fine, octant, reserved).  Returns (coarse, bad)."""
    out = _f64(coarse).copy()
    fine = _f64(fine)
    children = _records(children, ("coarse", "fine", "octant", "reserved"), 24)
    bad = _load().oracle_restrict(_ptr(fine), _ptr(out), out.shape[0], fine.shape[0],
                                  children.ctypes.data_as(ctypes.c_void_p), len(children))
    if bad < 0:
        raise ValueError("oracle_restrict rejected its arguments")
    return out, int(bad)


def fill_ghosts_uniform(level, gx, gy, gz, bc):
    """level[G][5][16][16][16] (group id (z*gy+y)*gx+x) -> in[G][5][20][20][20]."""
    level = _f64(level)
    G = gx * gy * gz
    assert level.shape == (G, 5, 16, 16, 16), level.shape
    out = np.empty((G, 5, 20, 20, 20))
    rc = _load().oracle_fill_ghosts_uniform(_ptr(level), gx, gy, gz, int(bc), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_fill_ghosts_uniform rejected its arguments")
    return out


def hydro_dt(partials, dh_level, cfl, level=None):
    partials = _f64(partials)
    N = partials.shape[0]
    dh_level = _f64(np.atleast_1d(dh_level))
    L = dh_level.shape[0]
    lev = None if level is None else np.ascontiguousarray(level, dtype=np.int32)
    dt = np.empty(L)
    tot = np.empty(5)
    rc = _load().oracle_hydro_dt(_ptr(partials), N, _ptr(lev, ctypes.c_int32), L, _ptr(dh_level),
                                 float(cfl), _ptr(dt), _ptr(tot))
    if rc != 0:
        raise ValueError("oracle_hydro_dt rejected its arguments")
    return dt, tot


def prim(U, gamma):
    U = _f64(U)
    W = np.empty(5)
    _load().oracle_prim_from_cons(_ptr(U), float(gamma), _ptr(W))
    return W


def cons(W, gamma):
    W = _f64(W)
    U = np.empty(5)
    _load().oracle_cons_from_prim(_ptr(W), float(gamma), _ptr(U))
    return U


def euler_flux(d, W, E):
    W = _f64(W)
    F = np.empty(5)
    _load().oracle_euler_flux(int(d), _ptr(W), float(E), _ptr(F))
    return F


def limiter(idx, a, b):
    return _load().oracle_limiter(int(idx), float(a), float(b))


def roe_flux(d, UL, UR, gamma, entropy_fix=True):
    """Returns (F[5], hlle_used)."""
    UL, UR = _f64(UL), _f64(UR)
    F = np.empty(5)
    used = _load().oracle_roe_flux(int(d), _ptr(UL), _ptr(UR), float(gamma), int(entropy_fix),
                                   _ptr(F))
    return F, bool(used)


def hlle_flux(d, UL, UR, gamma):
    UL, UR = _f64(UL), _f64(UR)
    F = np.empty(5)
    _load().oracle_hlle_flux(int(d), _ptr(UL), _ptr(UR), float(gamma), _ptr(F))
    return F


def char_slopes(d, Wl, Wc, Wr, gamma, limiter=0):
    """Characteristic-limited slope (primitive variables) of Wc along d."""
    Wl, Wc, Wr = _f64(Wl), _f64(Wc), _f64(Wr)
    s = np.empty(5)
    _load().oracle_char_slopes(int(d), _ptr(Wl), _ptr(Wc), _ptr(Wr), float(gamma), int(limiter),
                               _ptr(s))
    return s


def hllc_flux(d, UL, UR, gamma):
    UL, UR = _f64(UL), _f64(UR)
    F = np.empty(5)
    _load().oracle_hllc_flux(int(d), _ptr(UL), _ptr(UR), float(gamma), _ptr(F))
    return F


def exact_star(rl, ul, pl, rr, ur, pr, gamma):
    """(p*, u*, rho*_L, rho*_R) of the exact Riemann problem."""
    s = np.empty(4)
    it = _load().oracle_exact_riemann_star(rl, ul, pl, rr, ur, pr, gamma, _ptr(s))
    if it < 0:
        raise ValueError("vacuum is generated")
    return tuple(float(x) for x in s)


def exact_sample(rl, ul, pl, rr, ur, pr, gamma, xi):
    """(rho, u, p) of the exact Riemann solution at x/t = xi."""
    W = np.empty(3)
    _load().oracle_exact_riemann_sample(rl, ul, pl, rr, ur, pr, gamma, float(xi), _ptr(W))
    return tuple(float(x) for x in W)


def count_ops_group(U_in_group, dt, dh, gamma=5.0 / 3.0, limiter=0, predictor_fallback=0):
    """Operation tally of one 16^3-group step: dict of add, mul, div, sqrt, cmp, cells."""
    U = _f64(U_in_group)
    assert U.shape == (5, 20, 20, 20)
    c = np.empty(6)
    p = _params(gamma, limiter, predictor_fallback)
    rc = _load().oracle_count_ops_group(_ptr(U), float(dt), float(dh), ctypes.byref(p), _ptr(c))
    if rc != 0:
        raise ValueError("oracle_count_ops_group rejected its arguments")
    return dict(zip(("add", "mul", "div", "sqrt", "cmp", "cells"), c.tolist()))


PIECES = {"prim": 0, "cons": 1, "flux": 2, "limiter": 3, "roe": 4, "positive": 5}


def count_ops_piece(piece, a, b=None, gamma=5.0 / 3.0, d=0):
    """Operation tally of one scheme piece (see PIECES) on the counting scalar:
    dict of add, mul, div, sqrt, cmp.  a, b: length-5 arrays (the limiter and
    the flux read a[0], b[0] / a, b[0])."""
    A = _f64(np.resize(np.asarray(a, dtype=np.float64), 5))
    B = None if b is None else _f64(np.resize(np.asarray(b, dtype=np.float64), 5))
    c = np.empty(5)
    rc = _load().oracle_count_ops_piece(PIECES[piece], int(d), _ptr(A), _ptr(B), float(gamma),
                                        _ptr(c))
    if rc != 0:
        raise ValueError("oracle_count_ops_piece rejected its arguments")
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), c.tolist()))
