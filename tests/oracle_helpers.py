"""Small drivers around the oracle used by the CPU pin tests (no GPU)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1007_3818_gb300 import workloads as wl


def box_step(U, bc, dt, dh, gamma, **kw):
    """One oracle step of a whole box U[5][nz][ny][nx] with numpy ghost padding."""
    out, faces, st, part = oracle.advance_box(wl.pad_box(U, bc), dt, dh, gamma=gamma, **kw)
    return out, faces, st, part


def cfl_dt(U, dh, gamma, cfl, bc):
    """dt from the oracle's own max-signal-speed partial of the current state."""
    # a zero-length step returns the partials of the unchanged state
    _, _, _, part = box_step(U, bc, 0.0, dh, gamma)
    return cfl * dh / part[0]


def run_box(U, t_end, dh, gamma, cfl=0.5, bc=1, max_steps=100000, **kw):
    """Advance a box to t_end with CFL steps (last step shortened)."""
    t = 0.0
    status = 0
    for _ in range(max_steps):
        if t >= t_end * (1 - 1e-14):
            break
        dt = min(cfl_dt(U, dh, gamma, cfl, bc), t_end - t)
        U, _, st, _ = box_step(U, bc, dt, dh, gamma, **kw)
        status |= st
        t += dt
    return U, status


def exact_cell_average_1d(left, right, gamma, n, t, x0=0.5, sub=32):
    """Cell averages of the exact Riemann solution (rho, u, p) on n cells of [0,1]."""
    h = 1.0 / n
    rho = np.zeros(n)
    for i in range(n):
        xs = i * h + (np.arange(sub) + 0.5) * h / sub
        acc = 0.0
        for x in xs:
            acc += oracle.exact_sample(*left, *right, gamma, (x - x0) / t)[0]
        rho[i] = acc / sub
    return rho


def l1(a, b):
    return float(np.mean(np.abs(a - b)))
