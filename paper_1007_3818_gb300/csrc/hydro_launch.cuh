// hydro_launch.cuh -- argument validation and launch of the hydro step kernel.
#pragma once

#include "abi_common.h"
#include "hydro_kernel.cuh"
#include "hydro_pair.cuh"

namespace gamer {

// Launch-shape override (0 = automatic: every SM filled to its occupancy).
int& hydro_ctas_per_sm_override(int mode);
// Code-shape variant of the FP32 kernel (0: inline Riemann solver, 1: one
// out-of-line copy); chosen by the autotuner.
int& hydro_variant();
int& hydro_debug_poison();
// debug: group whose plane-5 copy is withheld (-1: none) and the poll limit
// of the on-chip waits (0: default)
int64_t& hydro_debug_drop_group();
uint32_t& hydro_debug_wait_polls();

// Common launch path.  SRC 0: `in` = N tiles [N][5][20]^3; SRC 1: `in` = the
// level `geo` (N = gx*gy*gz), ghosts gathered in the kernel.
template <int MODE, int SRC>
int hydro_launch(const typename Prec<MODE>::T* in, typename Prec<MODE>::T* out,
                 typename Prec<MODE>::T* face_flux, const double* dt, const double* dh,
                 uint32_t* status, double* partials, int64_t N, const gh_params* p,
                 LevelGeom geo, void* stream, int64_t win_layers = 0) {
    using T = typename Prec<MODE>::T;
    using P = typename Prec<MODE>::P;
    if (N < 0) return GAMER_E_PARAM;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    if (N == 0) return GAMER_OK;
    if (!in || !out || !dt || !dh) return GAMER_E_NULL;
    if (!aligned(in, 16) || !aligned(out, sizeof(T)) || !aligned(face_flux, sizeof(T)) ||
        !aligned(dt, 8) || !aligned(dh, 8) || !aligned(status, 4) || !aligned(partials, 8))
        return GAMER_E_ALIGN;
    // input: N tiles, or the window of win_layers z-layers of the level
    const size_t nin = (SRC == 0 ? size_t(N) * 40000
                                 : size_t(win_layers) * size_t(geo.gx) * size_t(geo.gy) * 20480) *
                       sizeof(T);
    const size_t nout = size_t(N) * 20480 * sizeof(T);
    const size_t nff =
        face_flux ? size_t(N) * (p->flux_layout ? 9 : 6) * 1280 * sizeof(T) : 0;
    const size_t nst = status ? size_t(N) * 4 : 0, npa = partials ? size_t(N) * 48 : 0;
    const void* ins[3] = {in, dt, dh};
    const size_t insz[3] = {nin, size_t(N) * 8, size_t(N) * 8};
    const void* outs[4] = {out, face_flux, status, partials};
    const size_t outsz[4] = {nout, nff, nst, npa};
    for (int a = 0; a < 4; ++a) {
        for (int b = 0; b < 3; ++b)
            if (overlaps(outs[a], outsz[a], ins[b], insz[b])) return GAMER_E_OVERLAP;
        for (int b = a + 1; b < 4; ++b)
            if (overlaps(outs[a], outsz[a], outs[b], outsz[b])) return GAMER_E_OVERLAP;
    }
    DeviceInfo dev = current_device();
    if (dev.status != GAMER_OK) return dev.status;

    KConst<T, P> kc;
    kc.gamma = T(p->gamma);
    kc.gm1 = T(p->gamma - 1.0);
    kc.gm1_lo = T((p->gamma - 1.0) - double(kc.gm1));
    kc.gm1p = P(p->gamma - 1.0);
    kc.limiter = p->limiter;
    kc.pfb = p->predictor_fallback;
    kc.flux9 = p->flux_layout;
    kc.floors = (p->rho_floor > 0.0 ? 1 : 0) | (p->p_floor > 0.0 ? 2 : 0);
    kc.rho_floor = T(p->rho_floor);
    kc.p_floor = T(p->p_floor);
    kc.eth_floor = P(p->p_floor / (p->gamma - 1.0));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int want = hydro_ctas_per_sm_override(MODE);
    const int var = hydro_variant();

    // variants: 0 -- one problem at a time, FP32 modes built for 3 (default)
    // or 2 CTAs/SM, FP64 for 1; 1 (FP32 tiles only) -- the same with the
    // Riemann solver out of line; 2 (tiles only) -- two interleaved problems
    // per thread (pair kernel, 2 CTAs/SM in FP32, 1 in FP64), van Leer limiter
    // compiled in plus a runtime-limiter build for the others.  The HLLC
    // solver (p->riemann = 1) and characteristic limiting (p->reconstruction
    // = 1) come in the default shape only (3 CTAs/SM in FP32 modes, 1 in
    // FP64) and override the variant and CTA settings.
    const bool hllc = p->riemann == 1;
    const bool chr = p->reconstruction == 1;
    const bool special = hllc || chr;  // builds in the default shape only
    if constexpr (SRC == 0) {
      if (var == 2 && !special) {
        constexpr int MB = (MODE == GAMER_MODE_F64) ? 1 : 2;
        auto kern = (p->limiter == 0) ? hydro_pair_kernel<MODE, MB, 0>
                                      : hydro_pair_kernel<MODE, MB, -1>;
        const int smem = int(sizeof(SmemPair<T>));
        int per_sm = 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) !=
                cudaSuccess ||
            per_sm < 1)
            return GAMER_E_CUDA;
        if (want > 0 && want < per_sm) per_sm = want;
        const int64_t grid = std::min<int64_t>(N, int64_t(per_sm) * dev.sm_count);
        kern<<<dim3(unsigned(grid)), dim3(kThreads), smem, s>>>(in, out, face_flux, dt, dh,
                                                                status, partials, N, kc);
        return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
      }
    }
    // builds with room to spare in shared memory (2 CTAs/SM in FP32, FP64)
    // keep three input planes in flight instead of two
    void (*kern)(const T*, T*, T*, const double*, const double*, uint32_t*, double*, int64_t,
                 KConst<T, P>, LevelGeom);
    // (the fused gather adds its per-thread plans after the Smem block)
    constexpr int extra = int(PlaneLoader<SRC, 2, T>::kExtraSmem);
    int smem = int(sizeof(Smem<T, 2>)) + extra;
    int threads = kThreads;
    // the default limiter (van Leer) is compiled into the default builds;
    // the others are read per slope from kc.limiter
    const bool vl = p->limiter == 0;
    if constexpr (MODE == GAMER_MODE_F64) {
        kern = vl ? hydro_step_kernel<MODE, 1, 8, SRC, 3> : hydro_step_kernel<MODE, 1, 0, SRC, 3>;
        smem = int(sizeof(Smem<T, 3>)) + extra;
        // variant 3: 320 threads per group, still one CTA per SM (shared
        // memory), twice the warps
        if (var == 3) {
            kern = vl ? hydro_step_kernel<MODE, 1, 8, SRC, 3, 320>
                      : hydro_step_kernel<MODE, 1, 0, SRC, 3, 320>;
            smem = int(sizeof(Smem<T, 3>)) + int(PlaneLoader<SRC, 3, T, 320>::kExtraSmem);
            threads = 320;
        }
    } else {
        if (want == 2) {
            kern = vl ? hydro_step_kernel<MODE, 2, 8, SRC, 3>
                      : hydro_step_kernel<MODE, 2, 0, SRC, 3>;
            smem = int(sizeof(Smem<T, 3>)) + extra;
        } else {
            kern = vl ? hydro_step_kernel<MODE, 3, 8, SRC, 2>
                      : hydro_step_kernel<MODE, 3, 0, SRC, 2>;
        }
        if constexpr (MODE == GAMER_MODE_F32 && SRC == 0) {
            if (var == 1 && want != 2) kern = hydro_step_kernel<MODE, 3, 1, SRC, 2>;
        }
        // variant 3: 320 threads per group (one column per thread), 2 CTAs
        // per SM, three input planes in flight
        if (var == 3) {
            kern = vl ? hydro_step_kernel<MODE, 2, 8, SRC, 3, 320>
                      : hydro_step_kernel<MODE, 2, 0, SRC, 3, 320>;
            smem = int(sizeof(Smem<T, 3>)) + int(PlaneLoader<SRC, 3, T, 320>::kExtraSmem);
            threads = 320;
        }
    }
    if (special) {
        // Riemann solver in bits 0-1, characteristic limiting in bit 2; HLLC
        // with the van Leer limiter also has it compiled in (bit 3)
        const int rsv = (hllc ? 2 : 0) | (chr ? 4 : 0) | ((hllc && !chr && vl) ? 8 : 0);
        if constexpr (MODE == GAMER_MODE_F64) {
            kern = rsv == 10  ? hydro_step_kernel<MODE, 1, 10, SRC, 3>
                   : rsv == 2 ? hydro_step_kernel<MODE, 1, 2, SRC, 3>
                   : rsv == 4 ? hydro_step_kernel<MODE, 1, 4, SRC, 3>
                              : hydro_step_kernel<MODE, 1, 6, SRC, 3>;
        } else {
            kern = rsv == 10  ? hydro_step_kernel<MODE, 3, 10, SRC, 2>
                   : rsv == 2 ? hydro_step_kernel<MODE, 3, 2, SRC, 2>
                   : rsv == 4 ? hydro_step_kernel<MODE, 3, 4, SRC, 2>
                              : hydro_step_kernel<MODE, 3, 6, SRC, 2>;
            smem = int(sizeof(Smem<T, 2>)) + extra;
            threads = kThreads;
        }
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return GAMER_E_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return GAMER_E_CUDA;
    if (want > 0 && want < per_sm && !special) per_sm = want;
    // Shared memory the SM does not give to these blocks stays L1 cache (for
    // the register spills above all): ask for the smallest carveout that holds
    // per_sm blocks.  The driver rounds a carveout percentage up to the next
    // capacity it supports; passing the floor of that capacity's own
    // percentage selects exactly it.
    const int pct = carveout_percent(int64_t(per_sm) * (smem + dev.smem_reserved),
                                     dev.smem_per_sm);
    if (pct < 100 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct) !=
            cudaSuccess)
        return GAMER_E_CUDA;
    const int64_t grid = std::min<int64_t>(N, int64_t(per_sm) * dev.sm_count);
    kern<<<dim3(unsigned(grid)), dim3(unsigned(threads)), smem, s>>>(in, out, face_flux, dt, dh,
                                                                     status, partials, N, kc,
                                                                     geo);
    return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
}

template <int MODE>
int hydro_advance(const typename Prec<MODE>::T* in, typename Prec<MODE>::T* out,
                  typename Prec<MODE>::T* face_flux, const double* dt, const double* dh,
                  uint32_t* status, double* partials, int64_t N, const gh_params* p,
                  void* stream) {
    const LevelGeom geo = {1, 1, 1, 0, 0, 0, 0, hydro_debug_drop_group(),
                           hydro_debug_wait_polls()};
    return hydro_launch<MODE, 0>(in, out, face_flux, dt, dh, status, partials, N, p, geo,
                                 stream);
}

template <int MODE>
int hydro_advance_level(const typename Prec<MODE>::T* level, typename Prec<MODE>::T* out,
                        typename Prec<MODE>::T* face_flux, int32_t gx, int32_t gy, int32_t gz,
                        int32_t bc, const double* dt, const double* dh, uint32_t* status,
                        double* partials, const gh_params* p, void* stream) {
    if (gx < 0 || gy < 0 || gz < 0 || (bc != 0 && bc != 1)) return GAMER_E_PARAM;
    if (int64_t(gx) * 16 > (1 << 30) || int64_t(gy) * 16 > (1 << 30) ||
        int64_t(gz) * 16 > (1 << 30))
        return GAMER_E_PARAM;
    // the gather's per-group plan holds level offsets within a z-layer of
    // groups in units of 16 cells as 32-bit integers
    if (int64_t(gx) * gy * 1280 + 2048 > INT32_MAX) return GAMER_E_PARAM;
    const LevelGeom geo = {gx, gy, gz, bc, 0, 0, hydro_debug_poison(), hydro_debug_drop_group(),
                           hydro_debug_wait_polls()};
    return hydro_launch<MODE, 1>(level, out, face_flux, dt, dh, status, partials,
                                 int64_t(gx) * gy * gz, p, geo, stream, gz);
}

// Layers z0 .. z0+nz-1 of the level from a window of zn layers starting at
// level layer zb (periodic wrap); every layer the stencil reads must be in it.
template <int MODE>
int hydro_advance_level_window(const typename Prec<MODE>::T* window, typename Prec<MODE>::T* out,
                               typename Prec<MODE>::T* face_flux, int32_t gx, int32_t gy,
                               int32_t gz, int32_t bc, int32_t zb, int32_t zn, int32_t z0,
                               int32_t nz, const double* dt, const double* dh, uint32_t* status,
                               double* partials, const gh_params* p, void* stream) {
    if (gx < 0 || gy < 0 || gz < 0 || (bc != 0 && bc != 1)) return GAMER_E_PARAM;
    if (int64_t(gx) * 16 > (1 << 30) || int64_t(gy) * 16 > (1 << 30) ||
        int64_t(gz) * 16 > (1 << 30))
        return GAMER_E_PARAM;
    if (int64_t(gx) * gy * 1280 + 2048 > INT32_MAX) return GAMER_E_PARAM;
    if (nz < 0 || z0 < 0 || int64_t(z0) + nz > gz || zb < 0 || zb >= (gz > 0 ? gz : 1) ||
        zn < 0 || zn > gz)
        return GAMER_E_PARAM;
    if (nz == 0 || gx == 0 || gy == 0) return GAMER_OK;
    // every layer read (z0 - 1 .. z0 + nz, wrapped or clamped) lies in the window
    for (int64_t z = int64_t(z0) - 1; z <= int64_t(z0) + nz; ++z) {
        int64_t zz = z;
        if (zz < 0 || zz >= gz) {
            if (bc == 1) continue;  // zero-gradient: the clamped layer is an end layer, read anyway
            zz = (zz + gz) % gz;
        }
        if ((zz - zb + gz) % gz >= zn) return GAMER_E_PARAM;
    }
    const LevelGeom geo = {gx, gy, gz,
                           bc, zb, z0,
                           hydro_debug_poison(), hydro_debug_drop_group(),
                           hydro_debug_wait_polls()};
    return hydro_launch<MODE, 1>(window, out, face_flux, dt, dh, status, partials,
                                 int64_t(gx) * gy * nz, p, geo, stream, zn);
}

}  // namespace gamer
