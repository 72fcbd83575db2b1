// abi.cu -- library-wide C-ABI utilities: error strings, device check,
// version, launch-shape overrides used by the autotuner.
#include <cuda_runtime.h>

#include <mutex>

#include "abi_common.h"

namespace gamer {

DeviceInfo current_device() {
    static std::mutex mu;
    static DeviceInfo cache[64];
    DeviceInfo d;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return d;
    if (dev < 64) {
        std::lock_guard<std::mutex> lock(mu);
        if (cache[dev].device == dev) return cache[dev];
    }
    d.device = dev;
    if (cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&d.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess) {
        d.status = GAMER_E_CUDA;
        return d;
    }
    // built for sm_103a only: family 10.x with the 10.3 feature set
    d.status = (d.cc_major == 10 && d.cc_minor == 3) ? GAMER_OK : GAMER_E_DEVICE;
    if (dev < 64) {
        std::lock_guard<std::mutex> lock(mu);
        cache[dev] = d;
    }
    return d;
}

int& hydro_debug_poison() {
    static int v = 0;
    return v;
}

int64_t& hydro_debug_drop_group() {
    static int64_t v = -1;
    return v;
}

uint32_t& hydro_debug_wait_polls() {
    static uint32_t v = 0;
    return v;
}

int& hydro_variant() {
    static int v = 0;
    return v;
}

int& hydro_ctas_per_sm_override(int mode) {
    static int v[4] = {0, 0, 0, 0};
    return v[(mode >= 0 && mode < 4) ? mode : 0];
}

}  // namespace gamer

extern "C" const char* gamer_strerror(int code) {
    switch (code) {
        case GAMER_OK: return "success";
        case GAMER_E_NULL: return "a required pointer is NULL";
        case GAMER_E_PARAM: return "bad size or parameter";
        case GAMER_E_ALIGN: return "misaligned pointer";
        case GAMER_E_CUDA: return "CUDA launch or configuration error";
        case GAMER_E_DEVICE: return "current device is not a compute capability 10.3 GPU (sm_103a)";
        case GAMER_E_OVERLAP: return "an output buffer overlaps another buffer";
        case GAMER_E_WORKSPACE: return "workspace missing or too small";
        case GAMER_E_TIMEOUT: return "a bounded wait gave up";
        default: return "unknown error code";
    }
}

extern "C" int gamer_device_check(void) { return gamer::device_ok(); }

extern "C" const char* gamer_version(void) {
    return "gamer-gb300 hydro 1.0 (sm_103a, MUSCL-Hancock + Roe)";
}

extern "C" int gamer_set_hydro_ctas_per_sm(int32_t mode, int32_t ctas_per_sm) {
    if (mode < 0 || mode > 3 || ctas_per_sm < 0 || ctas_per_sm > 16) return GAMER_E_PARAM;
    gamer::hydro_ctas_per_sm_override(mode) = ctas_per_sm;
    return GAMER_OK;
}

extern "C" int gamer_set_hydro_variant(int32_t variant) {
    if (variant < 0 || variant > 3) return GAMER_E_PARAM;
    gamer::hydro_variant() = variant;
    return GAMER_OK;
}

extern "C" int gamer_set_debug_poison(int32_t on) {
    if (on != 0 && on != 1) return GAMER_E_PARAM;
    gamer::hydro_debug_poison() = on;
    return GAMER_OK;
}

extern "C" int gamer_set_debug_drop_plane(int64_t group, int32_t wait_polls) {
    if (group < -1 || wait_polls < 0) return GAMER_E_PARAM;
    gamer::hydro_debug_drop_group() = group;
    gamer::hydro_debug_wait_polls() = uint32_t(wait_polls);
    return GAMER_OK;
}
