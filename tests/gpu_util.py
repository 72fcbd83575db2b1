"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the FP64 oracle on identical inputs."""
from __future__ import annotations

import numpy as np

TOL_F64 = 1e-12      # relative L1 per field, per step
TOL_F32_1 = 1e-5     # relative L1 after one step (smooth flows)
TOL_F32_10 = 1e-4    # relative L1 after ten steps (smooth flows)


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
        "flux": flux_rel_l1(ff, r_ff),
        "maxspeed": float(np.max(np.abs(part[:, 0] - r_part[:, 0]) / np.abs(r_part[:, 0]))),
        "sums": float(np.max(np.abs(part[:, 1:] - r_part[:, 1:]) /
                             np.maximum(np.abs(r_out).reshape(len(out), 5, -1).sum(-1), 1e-300))),
    }
    assert err["out"] <= tol, err
    assert err["flux"] <= 10 * tol, err
    # the per-group partials are FP64 reductions of the written state
    part_tol = 1e-12 if mode == 2 else 10 * tol
    assert err["maxspeed"] <= part_tol and err["sums"] <= part_tol, err
    if check_status:
        assert np.array_equal(st, r_st), (st, r_st)
    return err
