"""CPU-only checks of the C-ABI library: it builds, loads, exports every symbol
the public header declares, and rejects bad arguments on the host before any
device work (these calls never reach a launch, so they run without a GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_1007_3818_gb300 import build as cuda_build
from paper_1007_3818_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gamer_gb300.h")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return native.lib()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gamer_\w+)\s*\(", text)))


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for required in ("gamer_hydro_advance_f32", "gamer_hydro_advance_mixed",
                     "gamer_hydro_advance_f64", "gamer_fill_ghosts_uniform_f32",
                     "gamer_fill_ghosts_uniform_f64", "gamer_hydro_dt",
                     "gamer_hydro_dt_workspace_bytes", "gamer_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_covers_codes(lib):
    for code in range(0, -9, -1):
        assert native.strerror(code) != "unknown error code"
    assert native.strerror(-99) == "unknown error code"


def test_version_string(lib):
    assert "sm_103a" in native.gamer_version()


P = ctypes.c_void_p
FAKE = 0x7F0000000000  # never dereferenced: every call below fails validation first


def _adv(lib, name, in_=FAKE, out=FAKE + (1 << 30), ff=None, dt=FAKE + (2 << 30),
         dh=FAKE + (3 << 30), st=None, part=None, N=4, params=None):
    if params is None:
        params = native.make_params(1.4)
    f = getattr(lib, name)
    return f(P(in_) if in_ else None, P(out) if out else None, P(ff) if ff else None,
             P(dt) if dt else None, P(dh) if dh else None, P(st) if st else None,
             P(part) if part else None, N, ctypes.byref(params), None)


@pytest.mark.parametrize("name", ["gamer_hydro_advance_f32", "gamer_hydro_advance_mixed",
                                  "gamer_hydro_advance_f64", "gamer_hydro_advance_ff"])
def test_advance_rejects_bad_arguments(lib, name):
    assert _adv(lib, name, N=-1) == -2
    assert _adv(lib, name, N=0) == 0  # no-op, returns before touching the device
    assert _adv(lib, name, in_=None) == -1
    assert _adv(lib, name, dt=None) == -1
    assert _adv(lib, name, params=native.make_params(1.0)) == -2
    assert _adv(lib, name, params=native.make_params(float("nan"))) == -2
    assert _adv(lib, name, params=native.make_params(1.4, limiter=3)) == -2
    assert _adv(lib, name, params=native.make_params(1.4, predictor_fallback=2)) == -2
    assert _adv(lib, name, params=native.make_params(1.4, riemann=2)) == -2
    assert _adv(lib, name, params=native.make_params(1.4, reconstruction=2)) == -2
    bad = native.make_params(1.4)
    bad.reserved = 1
    assert _adv(lib, name, params=bad) == -2
    assert _adv(lib, name, params=native.make_params(1.4, flux_layout=2)) == -2
    assert _adv(lib, name, params=native.make_params(1.4, rho_floor=-1e-3)) == -2
    assert _adv(lib, name, params=native.make_params(1.4, p_floor=float("nan"))) == -2
    assert _adv(lib, name, params=native.make_params(1.4, p_floor=float("inf"))) == -2
    assert _adv(lib, name, in_=FAKE + 8) == -3           # TMA source needs 16 B alignment
    assert _adv(lib, name, dt=FAKE + (2 << 30) + 4) == -3
    assert _adv(lib, name, out=FAKE + 64) == -6          # out inside in
    assert _adv(lib, name, ff=FAKE + (1 << 30) + 128) == -6  # face flux inside out
    f = getattr(lib, name)
    assert f(P(FAKE), P(FAKE + (1 << 30)), None, P(FAKE + (2 << 30)), P(FAKE + (3 << 30)),
             None, None, 4, None, None) == -1            # params NULL


@pytest.mark.parametrize("name", ["gamer_hydro_advance_level_f32",
                                  "gamer_hydro_advance_level_mixed",
                                  "gamer_hydro_advance_level_f64",
                                  "gamer_hydro_advance_level_ff"])
def test_advance_level_rejects_bad_arguments(lib, name):
    f = getattr(lib, name)
    prm = native.make_params(1.4)

    def call(level=FAKE, out=FAKE + (1 << 32), gx=2, gy=2, gz=2, bc=0, dt=FAKE + (2 << 32)):
        return f(P(level) if level else None, P(out), None, gx, gy, gz, bc, P(dt),
                 P(FAKE + (3 << 32)), None, None, ctypes.byref(prm), None)

    assert call(bc=2) == -2
    assert call(gx=-1) == -2
    assert call(gz=1 << 27) == -2                     # extent above 2^26 groups
    assert call(gx=1300, gy=1300, gz=1) == -2         # z-layer beyond the gather's offsets
    assert call(gx=0) == 0                            # empty level
    assert call(level=None) == -1
    assert call(level=FAKE + 8) == -3                 # level needs 16 B alignment
    assert call(out=FAKE + 4096) == -6                # out inside the level


@pytest.mark.parametrize("name", ["gamer_hydro_advance_level_window_f32",
                                  "gamer_hydro_advance_level_window_f64"])
def test_level_window_rejects_missing_layers(lib, name):
    f = getattr(lib, name)
    prm = native.make_params(1.4)
    GB = 1 << 32

    def call(gz=8, bc=0, zb=0, zn=8, z0=0, nz=8):
        return f(P(FAKE), P(FAKE + GB), None, 2, 2, gz, bc, zb, zn, z0, nz, P(FAKE + 2 * GB),
                 P(FAKE + 3 * GB), None, None, ctypes.byref(prm), None)

    # only calls that fail validation (never reach the device with these fake pointers)
    assert call(nz=0) == 0                           # nothing to do
    assert call(z0=6, nz=3) == -2                    # beyond the level
    assert call(zb=8) == -2 and call(zn=9) == -2
    assert call(zb=3, zn=3, z0=3, nz=2) == -2        # needs 2..5: layer 2 below is missing
    assert call(zb=2, zn=3, z0=3, nz=2) == -2        # needs 2..5: layer 5 above is missing
    assert call(zb=0, zn=2, z0=0, nz=1, bc=0) == -2  # periodic: layer 7 below is missing


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_flux_fixup_and_restrict_reject_bad_arguments(lib, prec):
    fix = getattr(lib, f"gamer_flux_fixup_{prec}")
    res = getattr(lib, f"gamer_restrict_{prec}")
    GB = 1 << 32

    def call_fix(coarse=FAKE, cflux=FAKE + GB, fflux=FAKE + 2 * GB, n_sub=2, dt=FAKE + 3 * GB,
                 faces=FAKE + 4 * GB, n=5, bad=None):
        return fix(P(coarse) if coarse else None, P(cflux), P(fflux), n_sub, P(dt),
                   P(FAKE + 5 * GB), 8, 4, P(faces) if faces else None, n,
                   P(bad) if bad else None, None)

    assert call_fix(n=0) == 0                       # no records: no-op
    assert call_fix(n_sub=0) == -2
    assert call_fix(n=-1) == -2
    assert call_fix(coarse=None) == -1
    assert call_fix(faces=None) == -1
    assert call_fix(faces=FAKE + 4 * GB + 4) == -3   # records need 8-byte alignment
    assert call_fix(bad=FAKE + 6 * GB + 2) == -3
    assert call_fix(cflux=FAKE + 64) == -6           # coarse state overlaps its fluxes
    assert res(P(FAKE), P(FAKE + GB), 8, 4, P(FAKE + 2 * GB), 0, None, None) == 0
    assert res(P(FAKE), P(FAKE + GB), -1, 4, P(FAKE + 2 * GB), 3, None, None) == -2
    assert res(None, P(FAKE + GB), 8, 4, P(FAKE + 2 * GB), 3, None, None) == -1
    assert res(P(FAKE), P(FAKE + 128), 8, 4, P(FAKE + 2 * GB), 3, None, None) == -6


def test_fill_ghosts_rejects_bad_arguments(lib):
    f = lib.gamer_fill_ghosts_uniform_f32
    assert f(P(FAKE), P(FAKE + (1 << 30)), 2, 2, 2, 2, None) == -2     # bc
    assert f(P(FAKE), P(FAKE + (1 << 30)), -1, 2, 2, 0, None) == -2
    assert f(P(FAKE), P(FAKE + (1 << 30)), 0, 2, 2, 0, None) == 0      # empty level
    assert f(None, P(FAKE + (1 << 30)), 2, 2, 2, 0, None) == -1
    assert f(P(FAKE), P(FAKE + (1 << 30) + 4), 2, 2, 2, 0, None) == -3  # in not 16 B aligned
    assert f(P(FAKE), P(FAKE + 1024), 2, 2, 2, 0, None) == -6


def test_hydro_dt_rejects_bad_arguments(lib):
    ws = native.gamer_hydro_dt_workspace_bytes(1000, 3)
    assert ws >= 8 * (3 + 5)
    assert native.gamer_hydro_dt_workspace_bytes(10, 0) == 0
    assert native.gamer_hydro_dt_workspace_bytes(10, 65) == 0
    f = lib.gamer_hydro_dt
    a = [P(FAKE), 1000, None, 3, P(FAKE + (1 << 20)), 0.5, P(FAKE + (2 << 20)), None, None,
         P(FAKE + (3 << 20)), ws, None]
    b = list(a); b[3] = 0
    assert f(*b) == -2
    b = list(a); b[5] = -0.5
    assert f(*b) == -2
    b = list(a); b[10] = ws - 8
    assert f(*b) == -7
    b = list(a); b[9] = None
    assert f(*b) == -7
    b = list(a); b[0] = None
    assert f(*b) == -1
    b = list(a); b[0] = P(FAKE + 4)
    assert f(*b) == -3


def test_level_run_rejects_a_missing_pipeline(lib):
    f = lib.gamer_pipeline_level_run_host
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int32] * 5 + [ctypes.c_double] * 3 + \
        [ctypes.c_void_p] * 4
    assert f(None, None, None, 1, 1, 1, 0, 1, 1e-3, 1.0, 0.5, None, None, None, None) == -1


def test_set_launch_shape_validation(lib):
    assert lib.gamer_set_hydro_ctas_per_sm(4, 1) == -2
    assert lib.gamer_set_hydro_ctas_per_sm(0, -1) == -2
    assert lib.gamer_set_hydro_ctas_per_sm(0, 0) == 0
    assert lib.gamer_set_hydro_ctas_per_sm(3, 0) == 0                # the float-float mode


def test_binding_fails_loudly_without_library(monkeypatch):
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB_PATH", "/nonexistent/libgamer_gb300.so")
    with pytest.raises(native.GamerError):
        native.lib()


def test_level_run_binding_checks_tensors_before_the_call(lib):
    """The binding rejects a non-contiguous host level before any C call, and
    a pipeline without a handle (NULL) gets GAMER_E_NULL from the library --
    no device is touched on either path."""
    torch = pytest.importorskip("torch")
    pl = native.Pipeline.__new__(native.Pipeline)
    pl.handle = None
    pl.mode = native.GAMER_MODE_F32
    good = torch.zeros((1, 5, 16, 16, 16), dtype=torch.float32)
    strided = torch.zeros((1, 5, 16, 16, 32), dtype=torch.float32)[..., ::2]
    params = native.make_params(1.4)
    with pytest.raises(native.GamerError) as e:
        pl.level_run_host(strided, good, 1, 1, 1, 0, 1, 1e-3, 1.0, 0.5, params)
    assert e.value.code == -2
    with pytest.raises(native.GamerError) as e:
        pl.level_run_host(good, good.clone(), 1, 1, 1, 0, 1, 1e-3, 1.0, 0.5, params,
                          dt_out=torch.zeros(4, dtype=torch.float64)[::2])
    assert e.value.code == -2
    with pytest.raises(native.GamerError) as e:
        pl.level_run_host(good, good.clone(), 1, 1, 1, 0, 1, 1e-3, 1.0, 0.5, params)
    assert e.value.code == -1


def test_debug_knobs_and_hold_validate_on_the_host(lib):
    """The failure-detection test facilities check their arguments before any
    device work: a drop group below -1 or a negative poll limit is
    GAMER_E_PARAM, a NULL pipeline is GAMER_E_NULL, a hold outside 0..60 s is
    GAMER_E_PARAM (checked before the pipeline is touched)."""
    assert lib.gamer_set_debug_drop_plane(-2, 0) == -2
    assert lib.gamer_set_debug_drop_plane(0, -1) == -2
    assert lib.gamer_set_debug_drop_plane(-1, 0) == 0          # normal operation
    assert lib.gamer_pipeline_debug_hold(None, 0.1) == -1


def test_host_alloc_validates_on_the_host(lib):
    """gamer_host_alloc / gamer_host_free reject bad arguments before mapping
    anything; a pointer the allocator did not return is refused."""
    p = ctypes.c_void_p()
    assert lib.gamer_host_alloc(0, 1, ctypes.byref(p)) == -2
    assert lib.gamer_host_alloc(1 << 47, 1, ctypes.byref(p)) == -2
    assert lib.gamer_host_alloc(4096, 1, None) == -1
    assert lib.gamer_host_free(None) == -1
    buf = ctypes.create_string_buffer(64)
    assert lib.gamer_host_free(ctypes.cast(buf, ctypes.c_void_p)) == -2
