// abi_common.h -- host-side argument checks and device queries shared by the
// C-ABI entry points of the CUDA library.
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "gamer_gb300.h"

namespace gamer {

inline bool aligned(const void* p, size_t a) {
    return (reinterpret_cast<uintptr_t>(p) % a) == 0;
}

// [a, a + na) and [b, b + nb) (bytes) overlap; NULL ranges never overlap.
inline bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

inline int check_params(const gh_params* p) {
    if (!p) return GAMER_E_NULL;
    if (!std::isfinite(p->gamma) || !(p->gamma > 1.0)) return GAMER_E_PARAM;
    if (p->limiter < 0 || p->limiter > 2) return GAMER_E_PARAM;
    if (p->predictor_fallback != 0 && p->predictor_fallback != 1) return GAMER_E_PARAM;
    if ((p->flux_layout != 0 && p->flux_layout != 1) || (p->riemann != 0 && p->riemann != 1) ||
        (p->reconstruction != 0 && p->reconstruction != 1) || p->reserved != 0)
        return GAMER_E_PARAM;
    if (!std::isfinite(p->rho_floor) || p->rho_floor < 0.0 || !std::isfinite(p->p_floor) ||
        p->p_floor < 0.0)
        return GAMER_E_PARAM;
    return GAMER_OK;
}

struct DeviceInfo {
    int device = -1;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    int status = GAMER_E_CUDA;
};

// Properties of the current device (cached per device id).
DeviceInfo current_device();

inline int device_ok() {
    DeviceInfo d = current_device();
    return d.status;
}

}  // namespace gamer
