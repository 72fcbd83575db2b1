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
    int smem_per_sm = 0;     // shared memory an SM can give its blocks (bytes)
    int smem_reserved = 0;   // shared memory the system reserves per block (bytes)
    int status = GAMER_E_CUDA;
};

// Properties of the current device (cached per device id).
DeviceInfo current_device();

// Carveout preference (percent of smem_per_sm) for blocks that need `need`
// bytes of shared memory per SM in all: the floor of the percentage of the
// smallest shared-memory capacity of the sm_100 family (0, 8, 16, 32, 64,
// 100, 132, 164, 196 or 228 KB) that holds them, which the driver's
// rounding up maps back to that capacity; 100 when only the largest does.
inline int carveout_percent(int64_t need, int smem_per_sm) {
    static const int kCapacityKB[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
    if (smem_per_sm <= 0) return 100;
    for (int kb : kCapacityKB) {
        const int64_t cap = int64_t(kb) * 1024;
        if (cap >= need && cap < smem_per_sm) return int(100 * cap / smem_per_sm);
    }
    return 100;
}

inline int device_ok() {
    DeviceInfo d = current_device();
    return d.status;
}

}  // namespace gamer
