// reduce_dt.cu -- FP64 time step per AMR level and conservation totals from
// the per-group partials of the hydro step.  Two deterministic passes: each
// block reduces a fixed contiguous slice of groups into the caller's
// workspace, one block combines the slices in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "abi_common.h"

namespace gamer {
namespace {

constexpr int kRedThreads = 256;
constexpr int kMaxLevels = 64;

inline int64_t red_blocks(int64_t N) {
    return std::max<int64_t>(1, std::min<int64_t>(1024, (N + 1023) / 1024));
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// pass 1: block b reduces groups [b*chunk, min(N, (b+1)*chunk))
__global__ void __launch_bounds__(kRedThreads) dt_pass1(const double* __restrict__ part,
                                                        int64_t N, const int32_t* __restrict__ level,
                                                        int L, int64_t chunk,
                                                        double* __restrict__ ws) {
    __shared__ unsigned long long smax[kMaxLevels];
    __shared__ double ssum[kRedThreads / 32][5];
    for (int l = threadIdx.x; l < L; l += blockDim.x) smax[l] = 0ull;
    __syncthreads();
    const int64_t lo = int64_t(blockIdx.x) * chunk, hi = min(N, lo + chunk);
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t g = lo + threadIdx.x; g < hi; g += blockDim.x) {
        const double m = part[g * 6];
        int l = level ? level[g] : 0;
        l = (l < 0 || l >= L) ? 0 : l;
        // speeds are >= 0, so the IEEE bit pattern orders like the value; a
        // NaN (the partials of a group the step abandoned) has a larger bit
        // pattern than any speed and so wins the maximum
        if (m > 0.0 || m != m)
            atomicMax(&smax[l], static_cast<unsigned long long>(__double_as_longlong(m)));
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] += part[g * 6 + 1 + q];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double t = warp_sum(s[q]);
        if (lane == 0) ssum[warp][q] = t;
    }
    __syncthreads();
    double* out = ws + size_t(blockIdx.x) * (L + 5);
    for (int l = threadIdx.x; l < L; l += blockDim.x)
        out[l] = __longlong_as_double(static_cast<long long>(smax[l]));
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += ssum[w][threadIdx.x];
        out[L + threadIdx.x] = t;
    }
}

// pass 2: one block combines the B slices in order
__global__ void __launch_bounds__(kRedThreads) dt_pass2(const double* __restrict__ ws, int B,
                                                        int L, const double* __restrict__ dh_level,
                                                        double cfl, double* __restrict__ dt_out,
                                                        double* __restrict__ totals) {
    __shared__ double ssum[kRedThreads / 32][5];
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        double m = 0.0;
        for (int b = 0; b < B; ++b) {  // a NaN, once met, stays (fmax would drop it)
            const double x = ws[size_t(b) * (L + 5) + l];
            m = (x > m || x != x) ? x : m;
        }
        dt_out[l] = (m != m) ? m : (m > 0.0) ? cfl * dh_level[l] / m : 0.0;
    }
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < B; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] += ws[size_t(b) * (L + 5) + L + q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const double t = warp_sum(s[q]);
        if (lane == 0) ssum[warp][q] = t;
    }
    __syncthreads();
    if (totals && threadIdx.x < 5) {
        double t = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += ssum[w][threadIdx.x];
        totals[threadIdx.x] = t;
    }
}

// pass 3 (optional): per-group time step for the next step, dt_group[g] = dt_out[level[g]]
__global__ void __launch_bounds__(kRedThreads) dt_scatter(const double* __restrict__ dt_out,
                                                          const int32_t* __restrict__ level,
                                                          int L, int64_t N,
                                                          double* __restrict__ dt_group) {
    for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < N;
         g += int64_t(gridDim.x) * blockDim.x) {
        int l = level ? level[g] : 0;
        l = (l < 0 || l >= L) ? 0 : l;
        dt_group[g] = dt_out[l];
    }
}

}  // namespace
}  // namespace gamer

extern "C" size_t gamer_hydro_dt_workspace_bytes(int64_t N, int32_t n_levels) {
    if (N < 0 || n_levels < 1 || n_levels > gamer::kMaxLevels) return 0;
    return size_t(gamer::red_blocks(N)) * size_t(n_levels + 5) * sizeof(double);
}

extern "C" int gamer_hydro_dt(const double* partials, int64_t N, const int32_t* level,
                              int32_t n_levels, const double* dh_level, double cfl, double* dt_out,
                              double* totals, double* dt_group, void* workspace,
                              size_t workspace_bytes, void* stream) {
    using namespace gamer;
    if (N < 0 || n_levels < 1 || n_levels > kMaxLevels || !std::isfinite(cfl) || cfl <= 0.0)
        return GAMER_E_PARAM;
    if (!dh_level || !dt_out || (N > 0 && !partials)) return GAMER_E_NULL;
    if (!aligned(partials, 8) || !aligned(dh_level, 8) || !aligned(dt_out, 8) ||
        !aligned(totals, 8) || !aligned(level, 4) || !aligned(workspace, 8) ||
        !aligned(dt_group, 8))
        return GAMER_E_ALIGN;
    const size_t need = gamer_hydro_dt_workspace_bytes(N, n_levels);
    if (!workspace || workspace_bytes < need) return GAMER_E_WORKSPACE;
    const int rc = device_ok();
    if (rc != GAMER_OK) return rc;
    const int64_t B = red_blocks(N);
    const int64_t chunk = std::max<int64_t>(1, (N + B - 1) / B);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* ws = static_cast<double*>(workspace);
    dt_pass1<<<unsigned(B), kRedThreads, 0, s>>>(partials, N, level, n_levels, chunk, ws);
    dt_pass2<<<1, kRedThreads, 0, s>>>(ws, int(B), n_levels, dh_level, cfl, dt_out, totals);
    if (dt_group && N > 0) {
        const DeviceInfo d = current_device();
        const int64_t blocks = std::min<int64_t>((N + kRedThreads - 1) / kRedThreads,
                                                 int64_t(d.sm_count) * 8);
        dt_scatter<<<unsigned(blocks), kRedThreads, 0, s>>>(dt_out, level, n_levels, N, dt_group);
    }
    return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
}

// ---------------------------------------------------------------------------
// gamer_hydro_dt_noalloc: gamer_hydro_dt for callers that cannot allocate
// device memory.  Its scratch is this fixed file-scope device array (64 KiB,
// present on every GPU that loads the library until the process exits).
namespace gamer {
namespace {

constexpr size_t kNoAllocScratchBytes = 64 * 1024;
__device__ __align__(256) double g_dt_scratch[kNoAllocScratchBytes / sizeof(double)];

// Device address of g_dt_scratch on the current device (host code only sees
// a stand-in for the array, never its address).  Looked up on every call made
// outside stream capture, so a module reloaded after cudaDeviceReset is found
// again; during capture the address of the last lookup on this device is used
// (the first call on a device must come before any capture).
double* noalloc_scratch(int dev, cudaStream_t stream) {
    static std::mutex mu;
    static double* addr[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev] || cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_dt_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        addr[dev] = static_cast<double*>(p);
    }
    return addr[dev];
}

}  // namespace
}  // namespace gamer

extern "C" int gamer_hydro_dt_noalloc(const double* partials, int64_t N, const int32_t* level,
                                      int32_t n_levels, const double* dh_level, double cfl,
                                      double* dt_out, double* totals, double* dt_group,
                                      void* stream) {
    using namespace gamer;
    if (N < 0 || n_levels < 1 || n_levels > kMaxLevels) return GAMER_E_PARAM;
    const size_t need = gamer_hydro_dt_workspace_bytes(N, n_levels);
    if (need > kNoAllocScratchBytes) return GAMER_E_WORKSPACE;
    const DeviceInfo d = current_device();
    if (d.status != GAMER_OK) return d.status;
    double* scratch = noalloc_scratch(d.device, static_cast<cudaStream_t>(stream));
    if (!scratch) return GAMER_E_CUDA;
    return gamer_hydro_dt(partials, N, level, n_levels, dh_level, cfl, dt_out, totals, dt_group,
                          scratch, kNoAllocScratchBytes, stream);
}
