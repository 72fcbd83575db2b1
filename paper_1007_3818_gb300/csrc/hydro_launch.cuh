// hydro_launch.cuh -- argument validation and launch of the hydro step kernel.
#pragma once

#include "abi_common.h"
#include "hydro_kernel.cuh"

namespace gamer {

// Launch-shape override (0 = automatic: every SM filled to its occupancy).
int& hydro_ctas_per_sm_override(int mode);
// Code-shape variant of the FP32 kernel (0: inline Riemann solver, 1: one
// out-of-line copy); chosen by the autotuner.
int& hydro_variant();

template <int MODE>
int hydro_advance(const typename Prec<MODE>::T* in, typename Prec<MODE>::T* out,
                  typename Prec<MODE>::T* face_flux, const double* dt, const double* dh,
                  uint32_t* status, double* partials, int64_t N, const gh_params* p,
                  void* stream) {
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
    const size_t nin = size_t(N) * 40000 * sizeof(T), nout = size_t(N) * 20480 * sizeof(T);
    const size_t nff = face_flux ? size_t(N) * 7680 * sizeof(T) : 0;
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

    // variant: FP64 has one (1 CTA/SM); FP32 modes are built for 2 and 3 CTAs/SM
    const int want = hydro_ctas_per_sm_override(MODE);
    const int minb = (MODE == GAMER_MODE_F64) ? 1 : ((want == 2) ? 2 : 3);
    void (*kern)(const T*, T*, T*, const double*, const double*, uint32_t*, double*, int64_t,
                 KConst<T, P>);
    if constexpr (MODE == GAMER_MODE_F64) {
        kern = hydro_step_kernel<MODE, 1>;
    } else if constexpr (MODE == GAMER_MODE_F32) {
        kern = (minb == 2) ? hydro_step_kernel<MODE, 2>
                           : (hydro_variant() == 1 ? hydro_step_kernel<MODE, 3, 1>
                                                   : hydro_step_kernel<MODE, 3>);
    } else {
        kern = (minb == 2) ? hydro_step_kernel<MODE, 2> : hydro_step_kernel<MODE, 3>;
    }
    const int smem = int(sizeof(Smem<T>));
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
        return GAMER_E_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return GAMER_E_CUDA;
    if (want > 0 && want < per_sm) per_sm = want;
    const int64_t grid = std::min<int64_t>(N, int64_t(per_sm) * dev.sm_count);
    KConst<T, P> kc;
    kc.gamma = T(p->gamma);
    kc.gm1 = T(p->gamma - 1.0);
    kc.gm1p = P(p->gamma - 1.0);
    kc.limiter = p->limiter;
    kc.pfb = p->predictor_fallback;
    kern<<<dim3(unsigned(grid)), dim3(kThreads), smem, static_cast<cudaStream_t>(stream)>>>(
        in, out, face_flux, dt, dh, status, partials, N, kc);
    return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
}

}  // namespace gamer
