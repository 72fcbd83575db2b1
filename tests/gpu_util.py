"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle on identical inputs."""
from __future__ import annotations

import numpy as np

TOL_F64 = 1e-12      # relative L1 per field, per step
TOL_F32_1 = 1e-5     # relative L1 after one step (smooth flows)
TOL_F32_10 = 1e-4    # relative L1 after ten steps (smooth flows)

# Element-wise bound, next to the summed norms: every value a of the GPU
# result (state and face flux) must satisfy |a - b| <= C * eps * (|b| + S)
# against the oracle's b, with S the scale of that field in that group (the
# largest |b| of the field in the group; for a momentum component of the
# state, the largest momentum magnitude |m|).  FP32-storage modes (f32,
# mixed, float-float): eps = 2^-23 and C = ELEM_C_F32; FP64: C * eps = 1e-12.
# One step of the scheme rounds each value a few dozen times: the
# reconstruction and the half-step (~10 roundings of values of size S), a Roe
# flux (~30), and the update of U by the six flux differences scaled by
# lambda = dt/dh (|lambda F| <= CFL |U|); with rcp/sqrt.approx at 1-2 ulp
# and errors that mostly do not add up coherently, a few eps * S is typical.
# Measured on a GB300 over every compared state and face-flux array of the
# GPU suite (all configs, FP32, mixed and float-float modes): at most
# 6.3 eps * (|b| + S).  ELEM_C_F32 = 32 = 2^5 leaves a factor 5 above that
# and fails any value off by 4e-6 of its field's scale, which a summed L1
# over a few groups lets pass (one value off by 10 % adds only ~5e-6 to the
# rel-L1 of seven groups).
EPS_F32 = 2.0 ** -23
ELEM_C_F32 = 32.0
ELEM_TOL_F64 = 1e-12


def torch_dtype(mode):
    import torch
    from paper_1007_3818_gb300 import native
    return torch.float64 if mode == native.GAMER_MODE_F64 else torch.float32


def host_input(tiles, mode):
    """The oracle sees exactly what the GPU sees: FP32 modes round the input."""
    from paper_1007_3818_gb300 import native
    if mode == native.GAMER_MODE_F64:
        return np.ascontiguousarray(tiles, dtype=np.float64)
    return np.ascontiguousarray(tiles, dtype=np.float32).astype(np.float64)


def gpu_advance(tiles, dt, dh, gamma, mode, limiter=0, predictor_fallback=0, with_flux=True,
                rho_floor=0.0, p_floor=0.0, riemann=0, reconstruction=0):
    """One step on the GPU; returns numpy (out, face_flux, status, partials)."""
    import torch
    from paper_1007_3818_gb300 import native
    T = torch_dtype(mode)
    N = tiles.shape[0]
    d_in = torch.from_numpy(np.ascontiguousarray(tiles)).to("cuda", T)
    d_out = torch.full((N, 5, 16, 16, 16), float("nan"), device="cuda", dtype=T)
    d_ff = torch.full((N, 6, 5, 16, 16), float("nan"), device="cuda", dtype=T) if with_flux else None
    d_dt = torch.as_tensor(np.broadcast_to(np.asarray(dt, np.float64), (N,)).copy(), device="cuda")
    d_dh = torch.as_tensor(np.broadcast_to(np.asarray(dh, np.float64), (N,)).copy(), device="cuda")
    d_st = torch.full((N,), -1, device="cuda", dtype=torch.int32)
    d_part = torch.full((N, 6), float("nan"), device="cuda", dtype=torch.float64)
    params = native.make_params(gamma, limiter=limiter, predictor_fallback=predictor_fallback,
                                rho_floor=rho_floor, p_floor=p_floor, riemann=riemann,
                                reconstruction=reconstruction)
    native.hydro_advance(mode, d_in, d_out, d_ff, d_dt, d_dh, d_st, d_part, params)
    torch.cuda.synchronize()
    ff = d_ff.double().cpu().numpy() if with_flux else None
    return (d_out.double().cpu().numpy(), ff, d_st.cpu().numpy().astype(np.uint32),
            d_part.cpu().numpy())


def rel_l1_fields(a, b):
    """Relative L1 error, max over the conserved fields (axis 1):
    density and energy sum|a-b| / sum|b|; each momentum component
    sum|a-b| / sum|m_b|, with |m_b| the momentum magnitude per cell (so the
    measure does not depend on the orientation of the flow and a component
    that happens to be tiny is not judged against itself).  A field that is
    identically zero in b must be exactly zero in a (else inf)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if not np.isfinite(a).all():
        return float("inf")
    worst = 0.0
    nf = a.shape[1]
    mag = None
    if nf == 5:
        mag = np.abs(np.sqrt(b[:, 1] ** 2 + b[:, 2] ** 2 + b[:, 3] ** 2)).sum()
    for v in range(nf):
        av, bv = a[:, v], b[:, v]
        num = np.abs(av - bv).sum()
        if not np.abs(bv).any():
            if num != 0.0:
                return float("inf")
            continue
        den = mag if (mag is not None and 1 <= v <= 3) else np.abs(bv).sum()
        worst = max(worst, num / den)
    return worst


def rel_l1_per_field(a, b):
    """Relative L1 error of each field v (axis 1): sum|a_v - b_v| / sum|b_v|,
    the plain per-field definition (no magnitude normalisation); 0 for a field
    that is identically zero in both, inf for one that is zero in b only."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = np.zeros(a.shape[1])
    for v in range(a.shape[1]):
        num = np.abs(a[:, v] - b[:, v]).sum()
        den = np.abs(b[:, v]).sum()
        out[v] = (0.0 if num == 0.0 else float("inf")) if den == 0.0 else num / den
    return out


def elementwise_excess(a, b, mode, state=True):
    """max over values of |a - b| / (C eps (|b| + S)) (<= 1 passes) and the
    index of the worst value; a, b with groups on axis 0 and fields on axis 1
    (state [N][5][...] or face flux [N][F][5][...], the latter reshaped)."""
    from paper_1007_3818_gb300 import native
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if not state:  # [N][F][5][a][b] -> [N][5][F*a*b]
        N, F = a.shape[:2]
        a = a.reshape(N, F, 5, -1).transpose(0, 2, 1, 3).reshape(N, 5, -1)
        b = b.reshape(N, F, 5, -1).transpose(0, 2, 1, 3).reshape(N, 5, -1)
    N, nf = a.shape[:2]
    flat_b = b.reshape(N, nf, -1)
    S = np.abs(flat_b).max(axis=2)                                   # [N][5]
    if state and nf == 5:
        S[:, 1:4] = np.sqrt((flat_b[:, 1:4] ** 2).sum(axis=1)).max(axis=1)[:, None]
    tol = ELEM_TOL_F64 if mode == native.GAMER_MODE_F64 else ELEM_C_F32 * EPS_F32
    bound = tol * (np.abs(b) + S.reshape((N, nf) + (1,) * (b.ndim - 2)))
    with np.errstate(invalid="ignore", divide="ignore"):
        ratio = np.abs(a - b) / bound
    ratio = np.where(np.isnan(ratio), np.inf, ratio)   # NaN on either side fails
    ratio = np.where((a == b), 0.0, ratio)             # exact zeros of zero fields
    idx = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    return float(ratio[idx]), idx, float(a[idx]), float(b[idx])


def assert_elementwise(a, b, mode, what, state=True):
    r, idx, av, bv = elementwise_excess(a, b, mode, state)
    print(f"element-wise excess mode {mode} {what}: {r:.3g}")
    assert r <= 1.0, (f"{what}: value {idx} (group, field, ...) is {av!r}, oracle {bv!r}: "
                      f"{r:.3g} x the element-wise bound")
    return r


def flux_rel_l1(a, b):
    N = a.shape[0]
    return rel_l1_fields(a.reshape(N * 6, 5, -1).transpose(0, 1, 2),
                         b.reshape(N * 6, 5, -1))


def compare_step(tiles, dt, dh, gamma, mode, tol, limiter=0, predictor_fallback=0,
                 check_status=True, riemann=0, reconstruction=0):
    """GPU vs oracle for one step of the given tiles; returns the error dict."""
    import oracle
    host = host_input(tiles, mode)
    out, ff, st, part = gpu_advance(host, dt, dh, gamma, mode, limiter, predictor_fallback,
                                    riemann=riemann, reconstruction=reconstruction)
    r_out, r_ff, r_st, r_part = oracle.advance_groups(host, dt, dh, gamma=gamma, limiter=limiter,
                                                      predictor_fallback=predictor_fallback,
                                                      riemann=riemann,
                                                      reconstruction=reconstruction)
    err = {
        "out": rel_l1_fields(out, r_out),
        "out_per_field": rel_l1_per_field(out, r_out).tolist(),
        "flux": flux_rel_l1(ff, r_ff),
        "maxspeed": float(np.max(np.abs(part[:, 0] - r_part[:, 0]) / np.abs(r_part[:, 0]))),
        "sums": float(np.max(np.abs(part[:, 1:] - r_part[:, 1:]) /
                             np.maximum(np.abs(r_out).reshape(len(out), 5, -1).sum(-1), 1e-300))),
    }
    assert err["out"] <= tol, err
    # the plain per-field rel-L1 too: these inputs move in every direction,
    # so no momentum component is small against the flow
    assert max(err["out_per_field"]) <= tol, err
    assert err["flux"] <= 10 * tol, err
    # and value by value (state and face fluxes)
    err["elem_out"] = assert_elementwise(out, r_out, mode, "state")
    err["elem_flux"] = assert_elementwise(ff, r_ff, mode, "face flux", state=False)
    print(f"mode {mode}: rel-L1 {err['out']:.2e}, element-wise excess state "
          f"{err['elem_out']:.3g} flux {err['elem_flux']:.3g}")
    # the per-group partials are FP64 reductions of the written state
    part_tol = 1e-12 if mode == 2 else 10 * tol
    assert err["maxspeed"] <= part_tol and err["sums"] <= part_tol, err
    if check_status:
        assert np.array_equal(st, r_st), (st, r_st)
    return err
