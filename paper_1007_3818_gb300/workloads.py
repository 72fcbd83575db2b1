"""Seeded synthetic initial conditions for the patch-group hydro step.

This module only *defines states*: density, velocity and pressure fields and
their conserved form through the ideal-gas equation of state
E = p/(gamma-1) + rho|v|^2/2.  It holds none of the scheme's arithmetic, imports
neither the CUDA binding nor the oracle, and serves both of them, so that both
sides see bit-identical inputs.  numpy only; every generator takes a seed
(default 1007).

Layouts: a level is U[5][nz][ny][nx] (x fastest); a batch of patch groups is
U[N][5][16][16][16] (interior) or U[N][5][20][20][20] (with the 2-cell ghost
shell).  Group id on a uniform level of gx*gy*gz groups is (z*gy + y)*gx + x.

Workloads (each a stand-in for the paper's cosmology runs, whose data are not
available and not needed for the hydro step):
  * sod / lax shock tubes along x in one 16^3 group, zero-gradient ghosts;
  * a periodic uniform level with a smooth Fourier-mode density and a smooth
    Gaussian velocity field (sigma = 0.3 c_s), p = 1;
  * a Sedov-Taylor blast (E = 1 deposited in the central 2^3 cells) and a 3-D
    Kelvin-Helmholtz shear layer with 1 % seeded v_y noise;
  * lognormal, pressure ~ rho^gamma tiles for AMR-shaped batches and for the
    large streamed run.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1007


# ---------------------------------------------------------------------------
def to_conserved(rho, vx, vy, vz, p, gamma):
    """Stack (rho, rho vx, rho vy, rho vz, E) with the ideal-gas energy."""
    rho = np.asarray(rho, dtype=np.float64)
    E = p / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz)
    return np.stack([rho, rho * vx, rho * vy, rho * vz, E * np.ones_like(rho)])


def level_to_groups(U):
    """U[5][nz][ny][nx] -> groups[G][5][16][16][16] in (z*gy + y)*gx + x order."""
    _, nz, ny, nx = U.shape
    gz, gy, gx = nz // 16, ny // 16, nx // 16
    t = U.reshape(5, gz, 16, gy, 16, gx, 16)
    t = t.transpose(1, 3, 5, 0, 2, 4, 6)
    return np.ascontiguousarray(t.reshape(gz * gy * gx, 5, 16, 16, 16))


def groups_to_level(G, gx, gy, gz):
    """Inverse of level_to_groups."""
    t = np.asarray(G).reshape(gz, gy, gx, 5, 16, 16, 16)
    t = t.transpose(3, 0, 4, 1, 5, 2, 6)
    return np.ascontiguousarray(t.reshape(5, gz * 16, gy * 16, gx * 16))


def pad_box(U, bc):
    """Ghost shell of 2 cells around U[5][nz][ny][nx]: bc 0 periodic, 1 zero-gradient."""
    mode = "wrap" if bc == 0 else "edge"
    return np.pad(U, ((0, 0), (2, 2), (2, 2), (2, 2)), mode=mode)


# ---------------------------------------------------------------------------
def _centres(n):
    return (np.arange(n) + 0.5) / n


def fourier_mode_sum(n, modes):
    """sum_m a_m cos(2 pi k_m . x + phi_m) on the n^3 cell centres of the unit cube.

    modes: iterable of (kx, ky, kz, phi, a).  Evaluated separably through
    complex exponentials.  Returns [n][n][n] (z, y, x)."""
    x = _centres(n)
    out = np.zeros((n, n, n))
    for kx, ky, kz, phi, a in modes:
        ex = np.exp(2j * np.pi * kx * x + 1j * phi)
        ey = np.exp(2j * np.pi * ky * x)
        ez = np.exp(2j * np.pi * kz * x)
        out += a * (ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).real
    return out


def random_modes(rng, count, kmax):
    """count integer wave vectors with 1 <= |k| <= kmax and uniform phases."""
    modes = []
    while len(modes) < count:
        k = rng.integers(-kmax, kmax + 1, size=3)
        kk = float(np.sqrt((k * k).sum()))
        if kk < 1.0 or kk > kmax:
            continue
        modes.append((int(k[0]), int(k[1]), int(k[2]), float(rng.uniform(0, 2 * np.pi)), 1.0))
    return modes


def gaussian_field(n, rng, kmax=8.0, slope=-2.0):
    """Zero-mean, unit-rms periodic Gaussian random field on n^3 cells with
    power only at 1 <= |k| <= kmax (power ~ |k|^slope)."""
    kf = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(kf, kf, kr, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    mask = (kk >= 1.0) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[mask] = kk[mask] ** (slope / 2.0)
    spec = amp * (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape))
    f = np.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2))
    f -= f.mean()
    rms = np.sqrt((f * f).mean())
    return f / rms if rms > 0 else f


# ---------------------------------------------------------------------------
SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))


def shock_tube_level(n, left, right, gamma, x0=0.5, ny=1, nz=1):
    """1-D Riemann problem along x on an n x ny x nz box (cell centres vs x0)."""
    x = _centres(n)
    L = x < x0
    rho = np.where(L, left[0], right[0])
    u = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    shape = (nz, ny, n)
    b = lambda a: np.broadcast_to(a[None, None, :], shape)
    z = np.zeros(shape)
    return to_conserved(b(rho), b(u), z, z, b(p), gamma)


def sod_group(gamma=1.4):
    """Config 1: one 16^3 group, Sod along x (dh = 1/16); interior only."""
    return shock_tube_level(16, *SOD, gamma, ny=16, nz=16)


def lax_group(gamma=1.4):
    return shock_tube_level(16, *LAX, gamma, ny=16, nz=16)


def fourier_level(n=256, seed=DEFAULT_SEED, gamma=5.0 / 3.0, nmodes=8, kmax=8, amp=0.1,
                  vel_sigma_cs=0.3, p0=1.0):
    """Config 2: periodic level, rho = 1 + amp * sum of nmodes random-phase
    Fourier modes (|k| <= kmax), p = p0, each velocity component a smooth
    Gaussian field of rms vel_sigma_cs * c_s with c_s = sqrt(gamma p0 / 1)."""
    rng = np.random.default_rng(seed)
    modes = random_modes(rng, nmodes, kmax)
    rho = 1.0 + amp * fourier_mode_sum(n, modes)
    cs = np.sqrt(gamma * p0 / 1.0)
    v = [vel_sigma_cs * cs * gaussian_field(n, rng, kmax=kmax) for _ in range(3)]
    p = np.full((n, n, n), p0)
    return to_conserved(rho, v[0], v[1], v[2], p, gamma)


def sedov_level(n=256, gamma=5.0 / 3.0, E_blast=1.0, rho0=1.0, p0=1e-5):
    """Config 3a: uniform gas, E_blast deposited as thermal energy in the
    central 2^3 cells of a unit periodic box (dh = 1/n)."""
    rho = np.full((n, n, n), rho0)
    p = np.full((n, n, n), p0)
    z = np.zeros((n, n, n))
    U = to_conserved(rho, z, z, z, p, gamma)
    c = n // 2
    dV = (1.0 / n) ** 3
    U[4, c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] += E_blast / (8.0 * dV)
    return U


def kh_level(n=256, seed=DEFAULT_SEED, gamma=5.0 / 3.0, p0=2.5, noise=0.01):
    """Config 3b: rho = 2, v_x = +0.5 for |y - 1/2| < 1/4, else rho = 1,
    v_x = -0.5; p = p0; v_y = noise * U(-1, 1) per cell (seeded)."""
    rng = np.random.default_rng(seed)
    y = _centres(n)
    band = (np.abs(y - 0.5) < 0.25)[None, :, None]
    shape = (n, n, n)
    rho = np.broadcast_to(np.where(band, 2.0, 1.0), shape)
    vx = np.broadcast_to(np.where(band, 0.5, -0.5), shape)
    vy = noise * rng.uniform(-1.0, 1.0, size=shape)
    vz = np.zeros(shape)
    return to_conserved(rho, vx, vy, vz, np.full(shape, p0), gamma)


def lognormal_base(n, seed, gamma=5.0 / 3.0, sigma_ln=1.5, clip=None, vel_rms=1.0, kmax=8.0):
    """Periodic lognormal density, p = rho^gamma / gamma (so c_s(rho=1) = 1),
    velocity components smooth Gaussian fields of rms vel_rms."""
    rng = np.random.default_rng(seed)
    g = gaussian_field(n, rng, kmax=kmax)
    if clip is not None:
        g = np.clip(g, -clip, clip)
    rho = np.exp(sigma_ln * g)
    p = rho ** gamma / gamma
    v = [vel_rms * gaussian_field(n, rng, kmax=kmax) for _ in range(3)]
    return to_conserved(rho, v[0], v[1], v[2], p, gamma)


def window_tiles(base, origins):
    """20^3 periodic windows of base[5][n][n][n] at the given (x, y, z) origins
    -> tiles[N][5][20][20][20]."""
    n = base.shape[1]
    off = np.arange(20)
    origins = np.asarray(origins)
    out = np.empty((len(origins), 5, 20, 20, 20), dtype=base.dtype)
    for t, (ox, oy, oz) in enumerate(origins):
        ix = (ox + off) % n
        iy = (oy + off) % n
        iz = (oz + off) % n
        out[t] = base[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]
    return out


def amr_batch(counts=(2000, 12000, 40000), seed=DEFAULT_SEED, gamma=5.0 / 3.0, base_n=128,
              dh0=1.0 / 256.0, sigma_ln=1.5, subset=None):
    """Config 4: independent ghost-padded tiles from 3 AMR levels (dh halves per
    level), shuffled so every launch mixes levels.

    Returns (tiles[N][5][20][20][20] float64, level[N] int32, dh_level[L]).
    `subset` (array of indices) generates only those tiles of the full batch."""
    rng = np.random.default_rng(seed)
    base = lognormal_base(base_n, seed + 1, gamma=gamma, sigma_ln=sigma_ln, vel_rms=1.0)
    level = np.concatenate([np.full(c, l, dtype=np.int32) for l, c in enumerate(counts)])
    perm = rng.permutation(level.shape[0])
    level = level[perm]
    origins = rng.integers(0, base_n, size=(level.shape[0], 3))
    dh_level = np.array([dh0 / (2 ** l) for l in range(len(counts))])
    idx = np.arange(level.shape[0]) if subset is None else np.asarray(subset)
    return window_tiles(base, origins[idx]), level[idx], dh_level


def streamed_batch_tiles(N, seed=DEFAULT_SEED, gamma=5.0 / 3.0, base_n=128, subset=None,
                         contrast=1e4):
    """Config 5: lognormal tiles with density contrast `contrast` (ln rho =
    sigma * clip(g, -4, 4), sigma = ln(contrast)/8), v rms 1 c_s.
    Returns tiles for the indices in `subset` (default all N)."""
    rng = np.random.default_rng(seed)
    sigma = np.log(contrast) / 8.0
    base = lognormal_base(base_n, seed + 2, gamma=gamma, sigma_ln=sigma, clip=4.0, vel_rms=1.0)
    origins = rng.integers(0, base_n, size=(N, 3))
    idx = np.arange(N) if subset is None else np.asarray(subset)
    return window_tiles(base, origins[idx])


def random_smooth_groups(N, seed=DEFAULT_SEED, gamma=5.0 / 3.0, base_n=64, sigma_ln=0.5,
                         vel_rms=0.5):
    """Small generic batch for parity tests: windows of a smooth lognormal state."""
    rng = np.random.default_rng(seed)
    base = lognormal_base(base_n, seed + 3, gamma=gamma, sigma_ln=sigma_ln, vel_rms=vel_rms)
    origins = rng.integers(0, base_n, size=(N, 3))
    return window_tiles(base, origins)


def stress_groups(N, seed=DEFAULT_SEED, gamma=1.4):
    """White-noise stress tiles (not a physical workload): per-cell random
    log-density in [-4, 0], velocities in [-3, 3], log-pressure in [-7, -2],
    periodic ghosts of each tile.  Strong enough to fire both fallbacks."""
    rng = np.random.default_rng(seed)
    out = np.empty((N, 5, 20, 20, 20))
    idx = (np.arange(20) - 2) % 16
    for t in range(N):
        shape = (16, 16, 16)
        rho = np.exp(rng.uniform(-4.0, 0.0, shape))
        u, v, w = (rng.uniform(-3.0, 3.0, shape) for _ in range(3))
        p = np.exp(rng.uniform(-7.0, -2.0, shape))
        U = to_conserved(rho, u, v, w, p, gamma)
        out[t] = U[:, idx[:, None, None], idx[None, :, None], idx[None, None, :]]
    return out


def window_tiles_torch(base, origins, device):
    """window_tiles on a torch device: the same periodic 20^3 windows by pure
    indexing (bit-identical values).  base: numpy [5][n][n][n]; origins [N][3]
    (x, y, z).  Returns a float64 tensor [N][5][20][20][20] on `device`."""
    import torch
    n = base.shape[1]
    b = torch.as_tensor(np.ascontiguousarray(base), device=device)
    o = torch.as_tensor(np.asarray(origins), device=device, dtype=torch.int64)
    off = torch.arange(20, device=device)
    ix = (o[:, 0:1] + off) % n
    iy = (o[:, 1:2] + off) % n
    iz = (o[:, 2:3] + off) % n
    flat = b.reshape(5, -1)
    lin = (iz[:, :, None, None] * n + iy[:, None, :, None]) * n + ix[:, None, None, :]
    return flat[:, lin.reshape(-1)].reshape(5, len(o), 20, 20, 20).transpose(0, 1).contiguous()


def amr_batch_parts(counts=(2000, 12000, 40000), seed=DEFAULT_SEED, gamma=5.0 / 3.0, base_n=128,
                    dh0=1.0 / 256.0, sigma_ln=1.5):
    """The pieces amr_batch draws (base field, origins, level, dh per level),
    for generating the full batch on a device with window_tiles_torch."""
    rng = np.random.default_rng(seed)
    base = lognormal_base(base_n, seed + 1, gamma=gamma, sigma_ln=sigma_ln, vel_rms=1.0)
    level = np.concatenate([np.full(c, l, dtype=np.int32) for l, c in enumerate(counts)])
    perm = rng.permutation(level.shape[0])
    level = level[perm]
    origins = rng.integers(0, base_n, size=(level.shape[0], 3))
    dh_level = np.array([dh0 / (2 ** l) for l in range(len(counts))])
    return base, origins, level, dh_level


# --------------------------------------------------------------------------
# Two-level (refinement ratio 2) bookkeeping for the coarse-fine coupling:
# which fine patch group covers which coarse octant, and where the interfaces
# between refined and unrefined coarse patches lie.  Index arithmetic and
# copies only.

# one interface record: 8x8 coarse faces of one coarse group's flux plane
# covered by one face of one fine group (layout of gamer_cf_face)
CF_FACE_DTYPE = np.dtype([("coarse", "<i8"), ("fine", "<i8"), ("dir", "<i4"), ("plane", "<i4"),
                          ("side", "<i4"), ("quadrant", "<i4")])
# one child record: the fine group covering one octant of a coarse group
# (layout of gamer_cf_child)
CF_CHILD_DTYPE = np.dtype([("coarse", "<i8"), ("fine", "<i8"), ("octant", "<i4"),
                           ("reserved", "<i4")])


def cf_records(cg, refined):
    """Records of a periodic coarse level of cg = (cgx, cgy, cgz) groups whose
    coarse patches (8^3-cell octants, integer coords in [0, 2*cg)) listed in
    `refined` are each covered by one fine group (fine id = list position).

    Returns (children, faces): CF_CHILD_DTYPE and CF_FACE_DTYPE arrays.  A face
    record is made for every fine-group face whose neighbouring coarse patch is
    not refined; the corrected coarse cells are that patch's layer next to it."""
    cg = tuple(int(c) for c in cg)
    refined = [tuple(int(v) for v in p) for p in refined]
    index = {p: f for f, p in enumerate(refined)}
    children = np.zeros(len(refined), dtype=CF_CHILD_DTYPE)
    faces = []

    def group_of(p):
        g = [p[d] // 2 for d in range(3)]
        return (g[2] * cg[1] + g[1]) * cg[0] + g[0]

    for f, p in enumerate(refined):
        children[f] = (group_of(p), f, (p[0] & 1) | ((p[1] & 1) << 1) | ((p[2] & 1) << 2), 0)
        for d in range(3):
            for s in (-1, 1):
                q = list(p)
                q[d] = (q[d] + s) % (2 * cg[d])
                q = tuple(q)
                if q in index:
                    continue
                # the fine region lies on the + side of patch q when s = -1
                side = 1 if s == -1 else 0
                low = q[d] & 1          # position of patch q in its group along d
                plane = (low + 1) if side == 1 else low
                # in-plane octant bits of patch q: [a][b] = [k][j], [k][i], [j][i]
                ta, tb = {0: (2, 1), 1: (2, 0), 2: (1, 0)}[d]
                quadrant = (q[ta] & 1) | ((q[tb] & 1) << 1)
                faces.append((group_of(q), f, d, plane, side, quadrant))
    return children, np.array(faces, dtype=CF_FACE_DTYPE)


def composite_fine_level(coarse_groups, cg, fine_groups, refined):
    """Fine-resolution copy [5][2*16*cgz][2*16*cgy][2*16*cgx] of a two-level
    state: every coarse cell injected into its 2x2x2 fine cells, then the fine
    groups written over the patches they cover."""
    cgx, cgy, cgz = cg
    U = groups_to_level(coarse_groups, cgx, cgy, cgz)
    F = U.repeat(2, axis=1).repeat(2, axis=2).repeat(2, axis=3)
    for f, p in enumerate(refined):
        x0, y0, z0 = 16 * p[0], 16 * p[1], 16 * p[2]
        F[:, z0:z0 + 16, y0:y0 + 16, x0:x0 + 16] = fine_groups[f]
    return F


def fine_tiles(coarse_groups, cg, fine_groups, refined):
    """Ghost-padded 20^3 tiles of the fine groups, ghosts taken (periodically)
    from the composite fine-resolution state: neighbouring fine groups where
    refined, injected coarse cells elsewhere."""
    F = composite_fine_level(coarse_groups, cg, fine_groups, refined)
    nz, ny, nx = F.shape[1:]
    out = np.empty((len(refined), 5, 20, 20, 20), dtype=F.dtype)
    for f, p in enumerate(refined):
        zi = (16 * p[2] - 2 + np.arange(20)) % nz
        yi = (16 * p[1] - 2 + np.arange(20)) % ny
        xi = (16 * p[0] - 2 + np.arange(20)) % nx
        out[f] = F[:, zi][:, :, yi][:, :, :, xi]
    return out
