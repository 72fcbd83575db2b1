"""Thin ctypes binding of ``libgamer_gb300.so`` (C ABI in ``include/gamer_gb300.h``).

Argument marshalling only: every step of the hydro path runs in the library's
CUDA kernels.  Functions keep the C names and take torch tensors (device
memory) plus an optional CUDA stream (default: torch's current stream).  The
library is loaded on first use; if it has not been built the call raises
``GamerError`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgamer_gb300.so")

GAMER_MODE_F32, GAMER_MODE_MIXED, GAMER_MODE_F64, GAMER_MODE_FF = 0, 1, 2, 3
ST_PREDICTOR_FALLBACK, ST_HLLE_FALLBACK, ST_NONPOSITIVE_OUT = 0x1, 0x2, 0x4
ST_BAD_INPUT, ST_INTERNAL_TIMEOUT, ST_FLOOR = 0x8, 0x10, 0x20

_lock = threading.Lock()
_lib = None


class GamerError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = strerror(code) if _lib is not None else f"error {code}"
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")


class gh_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("cfl", ctypes.c_double),
                ("limiter", ctypes.c_int32), ("predictor_fallback", ctypes.c_int32),
                ("flux_layout", ctypes.c_int32), ("riemann", ctypes.c_int32),
                ("rho_floor", ctypes.c_double), ("p_floor", ctypes.c_double),
                ("reconstruction", ctypes.c_int32), ("reserved", ctypes.c_int32)]


FLUX_PLANES = {0: 6, 1: 9}  # face-flux planes per group by gh_params.flux_layout


def make_params(gamma, cfl=0.5, limiter=0, predictor_fallback=0, rho_floor=0.0, p_floor=0.0,
                flux_layout=0, riemann=0, reconstruction=0):
    return gh_params(float(gamma), float(cfl), int(limiter), int(predictor_fallback),
                     int(flux_layout), int(riemann), float(rho_floor), float(p_floor),
                     int(reconstruction), 0)


def lib():
    """Load the CUDA library (raises GamerError if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise GamerError(-4, f"{LIB_PATH} is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        for name in ("gamer_hydro_advance_f32", "gamer_hydro_advance_mixed",
                     "gamer_hydro_advance_f64", "gamer_hydro_advance_ff"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, vp, vp, vp, vp, vp, i64, P(gh_params), vp]
            f.restype = ctypes.c_int
        for name in ("gamer_hydro_advance_level_f32", "gamer_hydro_advance_level_mixed",
                     "gamer_hydro_advance_level_f64", "gamer_hydro_advance_level_ff"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp, vp, vp, vp, P(gh_params), vp]
            f.restype = ctypes.c_int
        for name in ("gamer_hydro_advance_level_window_f32", "gamer_hydro_advance_level_window_mixed",
                     "gamer_hydro_advance_level_window_f64", "gamer_hydro_advance_level_window_ff"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, vp, vp, vp,
                          P(gh_params), vp]
            f.restype = ctypes.c_int
        for name in ("gamer_fill_ghosts_uniform_f32", "gamer_fill_ghosts_uniform_f64"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, i32, i32, i32, i32, vp]
            f.restype = ctypes.c_int
        for name in ("gamer_flux_fixup_f32", "gamer_flux_fixup_f64"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, vp, i32, vp, vp, i64, i64, vp, i64, vp, vp]
            f.restype = ctypes.c_int
        for name in ("gamer_restrict_f32", "gamer_restrict_f64"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, i64, i64, vp, i64, vp, vp]
            f.restype = ctypes.c_int
        L.gamer_hydro_dt_workspace_bytes.argtypes = [i64, i32]
        L.gamer_hydro_dt_workspace_bytes.restype = ctypes.c_size_t
        L.gamer_hydro_dt.argtypes = [vp, i64, vp, i32, vp, d, vp, vp, vp, vp, ctypes.c_size_t,
                                     vp]
        L.gamer_hydro_dt.restype = ctypes.c_int
        L.gamer_hydro_dt_noalloc.argtypes = [vp, i64, vp, i32, vp, d, vp, vp, vp, vp]
        L.gamer_hydro_dt_noalloc.restype = ctypes.c_int
        L.gamer_strerror.argtypes = [ctypes.c_int]
        L.gamer_strerror.restype = ctypes.c_char_p
        L.gamer_device_check.argtypes = []
        L.gamer_device_check.restype = ctypes.c_int
        L.gamer_version.argtypes = []
        L.gamer_version.restype = ctypes.c_char_p
        L.gamer_set_hydro_variant.argtypes = [i32]
        L.gamer_set_hydro_variant.restype = ctypes.c_int
        L.gamer_set_debug_poison.argtypes = [i32]
        L.gamer_set_debug_poison.restype = ctypes.c_int
        L.gamer_set_debug_drop_plane.argtypes = [i64, i32]
        L.gamer_set_debug_drop_plane.restype = ctypes.c_int
        L.gamer_set_hydro_ctas_per_sm.argtypes = [i32, i32]
        L.gamer_set_hydro_ctas_per_sm.restype = ctypes.c_int
        L.gamer_microbench.argtypes = [i32, i64, vp, i64, P(d), vp]
        L.gamer_microbench.restype = ctypes.c_int
        L.gamer_level_graph_create.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32,
                                               i32, P(gh_params), vp, vp, vp, vp,
                                               ctypes.c_size_t, P(vp)]
        L.gamer_level_graph_create.restype = ctypes.c_int
        L.gamer_batch_graph_create.argtypes = [i32, vp, vp, vp, vp, vp, vp, i32, vp, vp, i64,
                                               P(gh_params), vp, vp, vp, vp, ctypes.c_size_t,
                                               P(vp)]
        L.gamer_batch_graph_create.restype = ctypes.c_int
        L.gamer_level_graph_launch.argtypes = [vp, vp]
        L.gamer_level_graph_launch.restype = ctypes.c_int
        L.gamer_level_graph_destroy.argtypes = [vp]
        L.gamer_level_graph_destroy.restype = ctypes.c_int
        L.gamer_pipeline_create.argtypes = [i32, i64, i32, P(vp)]
        L.gamer_pipeline_create.restype = ctypes.c_int
        L.gamer_pipeline_advance_host.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i64,
                                                  P(gh_params)]
        L.gamer_pipeline_advance_host.restype = ctypes.c_int
        L.gamer_pipeline_set_timeout.argtypes = [vp, d]
        L.gamer_pipeline_set_timeout.restype = ctypes.c_int
        L.gamer_pipeline_debug_hold.argtypes = [vp, d]
        L.gamer_pipeline_debug_hold.restype = ctypes.c_int
        L.gamer_pipeline_level_step_host.argtypes = [vp, vp, vp, i32, i32, i32, i32, d, d, vp, vp,
                                                     P(gh_params), i32]
        L.gamer_pipeline_level_step_host.restype = ctypes.c_int
        L.gamer_pipeline_level_run_host.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, d, d,
                                                    d, vp, vp, vp, P(gh_params)]
        L.gamer_pipeline_level_run_host.restype = ctypes.c_int
        L.gamer_pipeline_last_bytes.argtypes = [vp, P(i64), P(i64)]
        L.gamer_pipeline_last_bytes.restype = ctypes.c_int
        L.gamer_pipeline_set_level_mode.argtypes = [vp, i32]
        L.gamer_pipeline_set_level_mode.restype = ctypes.c_int
        for name in ("gamer_fill_ghosts_uniform_host_f32", "gamer_fill_ghosts_uniform_host_f64"):
            f = getattr(L, name)
            f.argtypes = [vp, vp, i32, i32, i32, i32, i32]
            f.restype = ctypes.c_int
        L.gamer_host_alloc.argtypes = [ctypes.c_size_t, i32, P(vp)]
        L.gamer_host_alloc.restype = ctypes.c_int
        L.gamer_host_free.argtypes = [vp]
        L.gamer_host_free.restype = ctypes.c_int
        L.gamer_pipeline_destroy.argtypes = [vp]
        L.gamer_pipeline_destroy.restype = ctypes.c_int
        _lib = L
        return L


def strerror(code):
    return lib().gamer_strerror(int(code)).decode()


def _check(rc, what):
    if rc != 0:
        raise GamerError(rc, what)


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t, dtype=None, shape_tail=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise GamerError(-1, f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise GamerError(-2, f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise GamerError(-2, f"{name} must be {dtype}, got {t.dtype}")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise GamerError(-2, f"{name} has shape {tuple(t.shape)}, expected (N, {shape_tail})")
    return ctypes.c_void_p(t.data_ptr())


_ADV = {GAMER_MODE_F32: "gamer_hydro_advance_f32", GAMER_MODE_MIXED: "gamer_hydro_advance_mixed",
        GAMER_MODE_F64: "gamer_hydro_advance_f64", GAMER_MODE_FF: "gamer_hydro_advance_ff"}


def _advance(mode, inp, out, face_flux, dt, dh, status, partials, params, stream):
    import torch
    T = torch.float64 if mode == GAMER_MODE_F64 else torch.float32
    N = int(inp.shape[0])
    args = [_ptr(inp, T, (5, 20, 20, 20), "in"), _ptr(out, T, (5, 16, 16, 16), "out"),
            _ptr(face_flux, T, (FLUX_PLANES[params.flux_layout], 5, 16, 16), "face_flux"),
            _ptr(dt, torch.float64, (), "dt"),
            _ptr(dh, torch.float64, (), "dh"), _ptr(status, torch.int32, (), "status"),
            _ptr(partials, torch.float64, (6,), "partials")]
    for t, nm in ((out, "out"), (face_flux, "face_flux"), (dt, "dt"), (dh, "dh"),
                  (status, "status"), (partials, "partials")):
        if t is not None and int(t.shape[0]) != N:
            raise GamerError(-2, f"{nm} has {int(t.shape[0])} groups, in has {N}")
    rc = getattr(lib(), _ADV[mode])(*args, N, ctypes.byref(params), _stream(stream))
    _check(rc, _ADV[mode])


def gamer_hydro_advance_f32(inp, out, face_flux, dt, dh, status, partials, params, stream=None):
    """One step of N groups, FP32.  Tensors: in[N,5,20,20,20] f32, out[N,5,16,16,16]
    f32, face_flux[N,6,5,16,16] f32 or None, dt/dh[N] f64, status[N] int32 or
    None, partials[N,6] f64 or None; params from make_params()."""
    _advance(GAMER_MODE_F32, inp, out, face_flux, dt, dh, status, partials, params, stream)


def gamer_hydro_advance_mixed(inp, out, face_flux, dt, dh, status, partials, params, stream=None):
    """As gamer_hydro_advance_f32 with FP64 pressure recovery."""
    _advance(GAMER_MODE_MIXED, inp, out, face_flux, dt, dh, status, partials, params, stream)


def gamer_hydro_advance_f64(inp, out, face_flux, dt, dh, status, partials, params, stream=None):
    """As gamer_hydro_advance_f32 with float64 arrays and arithmetic."""
    _advance(GAMER_MODE_F64, inp, out, face_flux, dt, dh, status, partials, params, stream)


def hydro_advance(mode, inp, out, face_flux, dt, dh, status, partials, params, stream=None):
    _advance(mode, inp, out, face_flux, dt, dh, status, partials, params, stream)


_ADV_LEVEL = {GAMER_MODE_F32: "gamer_hydro_advance_level_f32",
              GAMER_MODE_MIXED: "gamer_hydro_advance_level_mixed",
              GAMER_MODE_FF: "gamer_hydro_advance_level_ff",
              GAMER_MODE_F64: "gamer_hydro_advance_level_f64"}


def hydro_advance_level(mode, level, out, face_flux, gx, gy, gz, bc, dt, dh, status, partials,
                        params, stream=None):
    """One step of every group of a uniform level with the ghost gather fused
    into the kernel: level/out [G,5,16,16,16] (G = gx*gy*gz), face_flux
    [G,6,5,16,16] or None, dt/dh [G] f64, status [G] int32 or None, partials
    [G,6] f64 or None."""
    import torch
    T = torch.float64 if mode == GAMER_MODE_F64 else torch.float32
    G = gx * gy * gz
    for t, nm in ((level, "level"), (out, "out"), (face_flux, "face_flux"), (dt, "dt"),
                  (dh, "dh"), (status, "status"), (partials, "partials")):
        if t is not None and int(t.shape[0]) != G:
            raise GamerError(-2, f"{nm} must hold gx*gy*gz = {G} groups")
    args = [_ptr(level, T, (5, 16, 16, 16), "level"), _ptr(out, T, (5, 16, 16, 16), "out"),
            _ptr(face_flux, T, (FLUX_PLANES[params.flux_layout], 5, 16, 16), "face_flux"),
            int(gx), int(gy), int(gz), int(bc),
            _ptr(dt, torch.float64, (), "dt"), _ptr(dh, torch.float64, (), "dh"),
            _ptr(status, torch.int32, (), "status"), _ptr(partials, torch.float64, (6,), "partials")]
    rc = getattr(lib(), _ADV_LEVEL[mode])(*args, ctypes.byref(params), _stream(stream))
    _check(rc, _ADV_LEVEL[mode])


def hydro_advance_level_window(mode, window, out, face_flux, gx, gy, gz, bc, zb, z0, nz, dt, dh,
                               status, partials, params, stream=None):
    """Layers z0 .. z0+nz-1 of a gx*gy*gz level from a device window
    [zn*gx*gy, 5, 16, 16, 16] holding level layers zb, zb+1, ... (mod gz)."""
    import torch
    T = torch.float64 if mode == GAMER_MODE_F64 else torch.float32
    layer = gx * gy
    if layer == 0 or int(window.shape[0]) % layer:
        raise GamerError(-2, "window must hold whole layers of gx*gy groups")
    zn = int(window.shape[0]) // layer
    N = layer * nz
    for t, nm in ((out, "out"), (face_flux, "face_flux"), (dt, "dt"), (dh, "dh"),
                  (status, "status"), (partials, "partials")):
        if t is not None and int(t.shape[0]) != N:
            raise GamerError(-2, f"{nm} must hold gx*gy*nz = {N} groups")
    name = {GAMER_MODE_F32: "gamer_hydro_advance_level_window_f32",
            GAMER_MODE_MIXED: "gamer_hydro_advance_level_window_mixed",
            GAMER_MODE_FF: "gamer_hydro_advance_level_window_ff",
            GAMER_MODE_F64: "gamer_hydro_advance_level_window_f64"}[mode]
    rc = getattr(lib(), name)(
        _ptr(window, T, (5, 16, 16, 16), "window"), _ptr(out, T, (5, 16, 16, 16), "out"),
        _ptr(face_flux, T, (FLUX_PLANES[params.flux_layout], 5, 16, 16), "face_flux"),
        int(gx), int(gy), int(gz), int(bc), int(zb), zn, int(z0), int(nz),
        _ptr(dt, torch.float64, (), "dt"), _ptr(dh, torch.float64, (), "dh"),
        _ptr(status, torch.int32, (), "status"), _ptr(partials, torch.float64, (6,), "partials"),
        ctypes.byref(params), _stream(stream))
    _check(rc, name)


def gamer_hydro_advance_level_f32(level, out, face_flux, gx, gy, gz, bc, dt, dh, status,
                                  partials, params, stream=None):
    hydro_advance_level(GAMER_MODE_F32, level, out, face_flux, gx, gy, gz, bc, dt, dh, status,
                        partials, params, stream)


def gamer_hydro_advance_level_mixed(level, out, face_flux, gx, gy, gz, bc, dt, dh, status,
                                    partials, params, stream=None):
    hydro_advance_level(GAMER_MODE_MIXED, level, out, face_flux, gx, gy, gz, bc, dt, dh, status,
                        partials, params, stream)


def gamer_hydro_advance_level_f64(level, out, face_flux, gx, gy, gz, bc, dt, dh, status,
                                  partials, params, stream=None):
    hydro_advance_level(GAMER_MODE_F64, level, out, face_flux, gx, gy, gz, bc, dt, dh, status,
                        partials, params, stream)


def _fill(name, T, level, inp, gx, gy, gz, bc, stream):
    G = gx * gy * gz
    if int(level.shape[0]) != G or int(inp.shape[0]) != G:
        raise GamerError(-2, f"{name}: level/in must hold gx*gy*gz = {G} groups")
    rc = getattr(lib(), name)(_ptr(level, T, (5, 16, 16, 16), "level"),
                              _ptr(inp, T, (5, 20, 20, 20), "in"), gx, gy, gz, bc, _stream(stream))
    _check(rc, name)


def gamer_fill_ghosts_uniform_f32(level, inp, gx, gy, gz, bc, stream=None):
    import torch
    _fill("gamer_fill_ghosts_uniform_f32", torch.float32, level, inp, gx, gy, gz, bc, stream)


def gamer_fill_ghosts_uniform_f64(level, inp, gx, gy, gz, bc, stream=None):
    import torch
    _fill("gamer_fill_ghosts_uniform_f64", torch.float64, level, inp, gx, gy, gz, bc, stream)


# Records of the coarse-fine coupling (layouts of gamer_cf_face and
# gamer_cf_child): numpy structured arrays, moved to the device as bytes.
CF_FACE_FIELDS = ("coarse", "fine", "dir", "plane", "side", "quadrant")
CF_CHILD_FIELDS = ("coarse", "fine", "octant", "reserved")


def records_to_device(records, fields, itemsize, device="cuda"):
    """Copy a numpy structured array of coarse-fine records to a device byte
    tensor (the C structs' layout: int64 indices, then int32 fields)."""
    import numpy as np
    import torch
    a = np.ascontiguousarray(records)
    if a.dtype.names != fields or a.dtype.itemsize != itemsize:
        raise GamerError(-2, f"records must have fields {fields} ({itemsize} bytes each)")
    raw = np.frombuffer(a.tobytes(), dtype=np.uint8).copy()
    return torch.from_numpy(raw).to(device)


def _bytes_ptr(t, name):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise GamerError(-1, f"{name} must be a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def flux_fixup(mode, coarse, coarse_flux, fine_flux, dt, dh, faces, bad=None, stream=None):
    """Coarse-fine flux fix-up in place on coarse [Nc,5,16,16,16]:
    coarse_flux [Nc,9,5,16,16] (nine-plane layout), fine_flux
    [n_sub,Nf,6,5,16,16], dt/dh [Nc] f64, faces: device bytes of gamer_cf_face
    records (records_to_device), bad: int32 [1] device counter or None."""
    import torch
    T = torch.float64 if mode == GAMER_MODE_F64 else torch.float32
    Nc = int(coarse.shape[0])
    if fine_flux.dim() != 6 or tuple(fine_flux.shape[2:]) != (6, 5, 16, 16):
        raise GamerError(-2, "fine_flux must be [n_sub, Nf, 6, 5, 16, 16]")
    n_sub, Nf = int(fine_flux.shape[0]), int(fine_flux.shape[1])
    if int(coarse_flux.shape[0]) != Nc or int(dt.shape[0]) != Nc or int(dh.shape[0]) != Nc:
        raise GamerError(-2, "coarse_flux, dt and dh must hold Nc groups")
    if faces.numel() % 32:
        raise GamerError(-2, "faces must hold whole 32-byte records")
    name = "gamer_flux_fixup_f64" if mode == GAMER_MODE_F64 else "gamer_flux_fixup_f32"
    rc = getattr(lib(), name)(
        _ptr(coarse, T, (5, 16, 16, 16), "coarse"), _ptr(coarse_flux, T, (9, 5, 16, 16),
                                                        "coarse_flux"),
        _ptr(fine_flux, T, None, "fine_flux"), n_sub, _ptr(dt, torch.float64, (), "dt"),
        _ptr(dh, torch.float64, (), "dh"), Nc, Nf, _bytes_ptr(faces, "faces"),
        faces.numel() // 32, _ptr(bad, torch.int32, (), "bad"), _stream(stream))
    _check(rc, name)


def restrict(mode, fine, coarse, children, bad=None, stream=None):
    """Restriction of fine [Nf,5,16,16,16] onto the covered octants of coarse
    [Nc,5,16,16,16]; children: device bytes of gamer_cf_child records."""
    import torch
    T = torch.float64 if mode == GAMER_MODE_F64 else torch.float32
    if children.numel() % 24:
        raise GamerError(-2, "children must hold whole 24-byte records")
    name = "gamer_restrict_f64" if mode == GAMER_MODE_F64 else "gamer_restrict_f32"
    rc = getattr(lib(), name)(
        _ptr(fine, T, (5, 16, 16, 16), "fine"), _ptr(coarse, T, (5, 16, 16, 16), "coarse"),
        int(coarse.shape[0]), int(fine.shape[0]), _bytes_ptr(children, "children"),
        children.numel() // 24, _ptr(bad, torch.int32, (), "bad"), _stream(stream))
    _check(rc, name)


def gamer_hydro_dt_workspace_bytes(N, n_levels):
    return int(lib().gamer_hydro_dt_workspace_bytes(int(N), int(n_levels)))


def gamer_hydro_dt(partials, level, dh_level, cfl, dt_out, totals, dt_group, workspace,
                   stream=None):
    """dt per level, conservation totals and per-group dt (FP64) on the device.
    workspace: a CUDA tensor of at least gamer_hydro_dt_workspace_bytes(N, L) bytes."""
    import torch
    N = int(partials.shape[0])
    L = int(dh_level.shape[0])
    ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    rc = lib().gamer_hydro_dt(_ptr(partials, torch.float64, (6,), "partials"), N,
                              _ptr(level, torch.int32, (), "level"), L,
                              _ptr(dh_level, torch.float64, (), "dh_level"), float(cfl),
                              _ptr(dt_out, torch.float64, (), "dt_out"),
                              _ptr(totals, torch.float64, (), "totals"),
                              _ptr(dt_group, torch.float64, (), "dt_group"),
                              _ptr(workspace, None, None, "workspace"), ws_bytes, _stream(stream))
    _check(rc, "gamer_hydro_dt")


def gamer_hydro_dt_noalloc(partials, level, dh_level, cfl, dt_out, totals, dt_group,
                           stream=None):
    """gamer_hydro_dt for callers that cannot allocate device memory: the
    library's fixed 64 KiB device scratch replaces the workspace."""
    import torch
    rc = lib().gamer_hydro_dt_noalloc(_ptr(partials, torch.float64, (6,), "partials"),
                                      int(partials.shape[0]),
                                      _ptr(level, torch.int32, (), "level"),
                                      int(dh_level.shape[0]),
                                      _ptr(dh_level, torch.float64, (), "dh_level"), float(cfl),
                                      _ptr(dt_out, torch.float64, (), "dt_out"),
                                      _ptr(totals, torch.float64, (), "totals"),
                                      _ptr(dt_group, torch.float64, (), "dt_group"),
                                      _stream(stream))
    _check(rc, "gamer_hydro_dt_noalloc")


def gamer_device_check():
    return int(lib().gamer_device_check())


def gamer_version():
    return lib().gamer_version().decode()


def gamer_set_hydro_ctas_per_sm(mode, ctas_per_sm):
    _check(lib().gamer_set_hydro_ctas_per_sm(int(mode), int(ctas_per_sm)),
           "gamer_set_hydro_ctas_per_sm")


def gamer_set_debug_poison(on):
    """Debug: NaN-fill the level kernels' input slots before each gather."""
    _check(lib().gamer_set_debug_poison(int(on)), "gamer_set_debug_poison")


def gamer_set_debug_drop_plane(group, wait_polls=0):
    """Failure-detection test facility: withhold one input-plane copy of
    `group` (-1: none) so its bounded on-chip wait runs out after
    `wait_polls` polls (0: the default bound)."""
    _check(lib().gamer_set_debug_drop_plane(int(group), int(wait_polls)),
           "gamer_set_debug_drop_plane")


def gamer_set_hydro_variant(variant):
    _check(lib().gamer_set_hydro_variant(int(variant)), "gamer_set_hydro_variant")


def gamer_microbench(kind, iters, buf, n=0, stream=None):
    """Launches one throughput probe; returns its operation / byte count."""
    work = ctypes.c_double(0.0)
    rc = lib().gamer_microbench(int(kind), int(iters), _ptr(buf, None, None, "buf"), int(n),
                                ctypes.byref(work), _stream(stream))
    _check(rc, "gamer_microbench")
    return work.value


class LevelGraph:
    """gamer_level_graph_*: one device-resident uniform-level step (level_a ->
    level_b) per launch.  Keeps references to the tensors it was captured with."""

    def __init__(self, mode, level_a, level_b, tiles, face_flux, dt_group, dh_group, status,
                 partials, gx, gy, gz, bc, params, dh_level, dt_level, totals, workspace):
        self._keep = (level_a, level_b, tiles, face_flux, dt_group, dh_group, status, partials,
                      dh_level, dt_level, totals, workspace, params)
        h = ctypes.c_void_p()
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        ws_bytes = workspace.numel() * workspace.element_size()
        rc = lib().gamer_level_graph_create(int(mode), p(level_a), p(level_b), p(tiles),
                                            p(face_flux), p(dt_group), p(dh_group), p(status),
                                            p(partials), gx, gy, gz, bc, ctypes.byref(params),
                                            p(dh_level), p(dt_level), p(totals), p(workspace),
                                            ws_bytes, ctypes.byref(h))
        _check(rc, "gamer_level_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib().gamer_level_graph_launch(self.handle, _stream(stream)),
               "gamer_level_graph_launch")

    def close(self):
        if self.handle:
            lib().gamer_level_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchGraph(LevelGraph):
    """gamer_batch_graph_create: one step of an uneven AMR batch (dt per level
    from the previous partials, then the persistent step of all groups) per
    launch.  Keeps references to the tensors it was captured with."""

    def __init__(self, mode, inp, out, face_flux, dt_group, dh_group, level, n_levels, status,
                 partials, params, dh_level, dt_level, totals, workspace):
        import torch
        T = torch.float64 if mode == GAMER_MODE_F64 else torch.float32
        N = int(inp.shape[0])
        args = [_ptr(inp, T, (5, 20, 20, 20), "in"), _ptr(out, T, (5, 16, 16, 16), "out"),
                _ptr(face_flux, T, (FLUX_PLANES[params.flux_layout], 5, 16, 16), "face_flux"),
                _ptr(dt_group, torch.float64, (), "dt_group"),
                _ptr(dh_group, torch.float64, (), "dh_group"),
                _ptr(level, torch.int32, (), "level")]
        for t, nm in ((out, "out"), (dt_group, "dt_group"), (dh_group, "dh_group"),
                      (level, "level"), (status, "status"), (partials, "partials")):
            if t is not None and int(t.shape[0]) != N:
                raise GamerError(-2, f"{nm} has {int(t.shape[0])} groups, in has {N}")
        self._keep = (inp, out, face_flux, dt_group, dh_group, level, status, partials, dh_level,
                      dt_level, totals, workspace, params)
        h = ctypes.c_void_p()
        ws_bytes = workspace.numel() * workspace.element_size()
        rc = lib().gamer_batch_graph_create(
            int(mode), *args, int(n_levels), _ptr(status, torch.int32, (), "status"),
            _ptr(partials, torch.float64, (6,), "partials"), N, ctypes.byref(params),
            _ptr(dh_level, torch.float64, (), "dh_level"),
            _ptr(dt_level, torch.float64, (), "dt_level"), _ptr(totals, torch.float64),
            _ptr(workspace), ws_bytes, ctypes.byref(h))
        _check(rc, "gamer_batch_graph_create")
        self.handle = h


class Pipeline:
    """gamer_pipeline_*: host-resident batches streamed through the GPU."""

    def __init__(self, mode, batch_groups, with_flux=True):
        h = ctypes.c_void_p()
        _check(lib().gamer_pipeline_create(int(mode), int(batch_groups), int(bool(with_flux)),
                                           ctypes.byref(h)), "gamer_pipeline_create")
        self.handle = h
        self.mode = mode

    def set_timeout(self, seconds):
        _check(lib().gamer_pipeline_set_timeout(self.handle, float(seconds)),
               "gamer_pipeline_set_timeout")

    def debug_hold(self, seconds):
        """Test facility: hold the pipeline's streams for `seconds` (host sleep)."""
        _check(lib().gamer_pipeline_debug_hold(self.handle, float(seconds)),
               "gamer_pipeline_debug_hold")

    def advance_host(self, inp, out, face_flux, dt, dh, status, partials, params):
        """Host (CPU, ideally pinned) tensors with the layouts of hydro_advance."""
        import torch
        T = torch.float64 if self.mode == GAMER_MODE_F64 else torch.float32
        for t, nm, dtype in ((inp, "in", T), (out, "out", T), (face_flux, "face_flux", T),
                             (dt, "dt", torch.float64), (dh, "dh", torch.float64),
                             (status, "status", torch.int32), (partials, "partials", torch.float64)):
            if t is None:
                continue
            if t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
                raise GamerError(-2, f"{nm} must be a contiguous host tensor of {dtype}")
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        rc = lib().gamer_pipeline_advance_host(self.handle, p(inp), p(out), p(face_flux), p(dt),
                                               p(dh), p(status), p(partials), int(inp.shape[0]),
                                               ctypes.byref(params))
        _check(rc, "gamer_pipeline_advance_host")

    def level_step_host(self, level_in, level_out, gx, gy, gz, bc, dt, dh, status, partials,
                        params, nthreads=0):
        """One step of a host-resident uniform level (host tensors [G,5,16,16,16])."""
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        for t, nm in ((level_in, "level_in"), (level_out, "level_out")):
            if t.is_cuda or not t.is_contiguous():
                raise GamerError(-2, f"{nm} must be a contiguous host tensor")
        rc = lib().gamer_pipeline_level_step_host(self.handle, p(level_in), p(level_out), gx, gy,
                                                  gz, bc, float(dt), float(dh), p(status),
                                                  p(partials), ctypes.byref(params),
                                                  int(nthreads))
        _check(rc, "gamer_pipeline_level_step_host")

    def level_run_host(self, level0, level1, gx, gy, gz, bc, nsteps, dt0, dh, cfl, params,
                       dt_out=None, status=None, partials=None):
        """nsteps steps between two host tensors [G,5,16,16,16]: step n reads
        level[n % 2] and writes level[(n + 1) % 2]; dt0 for step 0, then the
        CFL dt from the previous step's partials (on the device).  dt_out
        [nsteps] float64, status [G] int32 (OR over the steps), partials [G,6]
        float64 (last step): host tensors or None."""
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        for t, nm in ((level0, "level0"), (level1, "level1")):
            if t.is_cuda or not t.is_contiguous():
                raise GamerError(-2, f"{nm} must be a contiguous host tensor")
        for t, nm in ((dt_out, "dt_out"), (status, "status"), (partials, "partials")):
            if t is not None and (t.is_cuda or not t.is_contiguous()):
                raise GamerError(-2, f"{nm} must be a contiguous host tensor")
        rc = lib().gamer_pipeline_level_run_host(self.handle, p(level0), p(level1), gx, gy, gz, bc,
                                                 int(nsteps), float(dt0), float(dh), float(cfl),
                                                 p(dt_out), p(status), p(partials),
                                                 ctypes.byref(params))
        _check(rc, "gamer_pipeline_level_run_host")

    def set_level_mode(self, mode):
        """0 automatic, 1 device copy of the whole level, 2 slab windows."""
        _check(lib().gamer_pipeline_set_level_mode(self.handle, int(mode)),
               "gamer_pipeline_set_level_mode")

    def last_bytes(self):
        """(host->device, device->host) bytes copied by the last call."""
        h2d, d2h = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().gamer_pipeline_last_bytes(self.handle, ctypes.byref(h2d), ctypes.byref(d2h)),
               "gamer_pipeline_last_bytes")
        return int(h2d.value), int(d2h.value)

    def close(self):
        if self.handle:
            lib().gamer_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gamer_fill_ghosts_uniform_host(level, inp, gx, gy, gz, bc, nthreads=0):
    """Host-array ghost fill (CPU threads); level/inp contiguous CPU tensors or
    numpy arrays of float32 / float64."""
    import numpy as np
    lv = level.numpy() if hasattr(level, "numpy") else level
    out = inp.numpy() if hasattr(inp, "numpy") else inp
    if lv.dtype != out.dtype or lv.dtype not in (np.float32, np.float64):
        raise GamerError(-2, "level and in must share a float32 / float64 dtype")
    if not (lv.flags.c_contiguous and out.flags.c_contiguous):
        raise GamerError(-2, "level and in must be contiguous")
    name = ("gamer_fill_ghosts_uniform_host_f32" if lv.dtype == np.float32
            else "gamer_fill_ghosts_uniform_host_f64")
    rc = getattr(lib(), name)(ctypes.c_void_p(lv.ctypes.data), ctypes.c_void_p(out.ctypes.data),
                              gx, gy, gz, bc, int(nthreads))
    _check(rc, name)


class HostBuffer:
    """gamer_host_alloc: page-locked, huge-page-backed host memory for levels
    streamed through the device.  ``.tensor`` views it with the given shape and
    dtype (a CPU tensor); call close() (or drop the object) once no device work
    uses it any more."""

    def __init__(self, shape, dtype, nthreads=0):
        import math
        import torch
        self.nbytes = int(math.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        p = ctypes.c_void_p()
        _check(lib().gamer_host_alloc(self.nbytes, int(nthreads), ctypes.byref(p)),
               "gamer_host_alloc")
        self.ptr = p
        arr = (ctypes.c_uint8 * self.nbytes).from_address(p.value)
        self.tensor = torch.frombuffer(arr, dtype=dtype).view(*shape)

    def close(self):
        if getattr(self, "ptr", None):
            self.tensor = None
            lib().gamer_host_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
