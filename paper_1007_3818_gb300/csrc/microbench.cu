// microbench.cu -- throughput probes that give the roofline denominators the
// hydro step is measured against: FP32 FMA, FP64 FMA, MUFU reciprocal and an
// HBM copy.  The caller times each launch with CUDA events.
#include <cuda_runtime.h>

#include "abi_common.h"

namespace gamer {
namespace {

constexpr int kChains = 8;

template <class T>
__global__ void __launch_bounds__(256) fma_probe(T* out, int iters, T b, T c) {
    T a[kChains];
#pragma unroll
    for (int s = 0; s < kChains; ++s) a[s] = T(threadIdx.x + s);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int s = 0; s < kChains; ++s) a[s] = fma(a[s], b, c);
    T acc = T(0);
#pragma unroll
    for (int s = 0; s < kChains; ++s) acc += a[s];
    if (acc == T(-1)) out[threadIdx.x] = acc;  // never true; keeps the chains alive
}

__global__ void __launch_bounds__(256) rcp_probe(float* out, int iters) {
    float a[kChains];
#pragma unroll
    for (int s = 0; s < kChains; ++s) a[s] = 1.0f + float(threadIdx.x + s);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int s = 0; s < kChains; ++s) asm volatile("rcp.approx.ftz.f32 %0, %0;" : "+f"(a[s]));
    float acc = 0.f;
#pragma unroll
    for (int s = 0; s < kChains; ++s) acc += a[s];
    if (acc == -1.f) out[threadIdx.x] = acc;
}

__global__ void __launch_bounds__(256) copy_probe(const float4* __restrict__ src,
                                                  float4* __restrict__ dst, int64_t n4) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n4;
         i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = src[i];
}

}  // namespace
}  // namespace gamer

// kind 0: FP32 FMA, 1: FP64 FMA, 2: MUFU rcp (each: grid of 8 CTAs x 256
// threads per SM, 8 chains x iters operations per thread; `buf` >= 1 KB);
// kind 3: copy of n floats from buf to buf + n (HBM read + write).
// Returns the number of operations (FMA/rcp) or bytes moved through *work.
extern "C" int gamer_microbench(int32_t kind, int64_t iters, void* buf, int64_t n, double* work,
                                void* stream) {
    using namespace gamer;
    if (!buf || !work) return GAMER_E_NULL;
    const DeviceInfo d = current_device();
    if (d.status != GAMER_OK) return d.status;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid = unsigned(d.sm_count) * 8u;
    if (kind >= 0 && kind <= 2) {
        if (iters <= 0 || iters > (1 << 30)) return GAMER_E_PARAM;
        if (kind == 0) fma_probe<float><<<grid, 256, 0, s>>>((float*)buf, int(iters), 0.999f, 1e-3f);
        if (kind == 1) fma_probe<double><<<grid, 256, 0, s>>>((double*)buf, int(iters), 0.999, 1e-3);
        if (kind == 2) rcp_probe<<<grid, 256, 0, s>>>((float*)buf, int(iters));
        *work = double(grid) * 256.0 * kChains * double(iters);
    } else if (kind == 3) {
        if (n <= 0 || n % 4 != 0 || !aligned(buf, 16)) return GAMER_E_PARAM;
        const float* src = static_cast<const float*>(buf);
        copy_probe<<<grid * 4, 256, 0, s>>>(reinterpret_cast<const float4*>(src),
                                            reinterpret_cast<float4*>(static_cast<float*>(buf) + n),
                                            n / 4);
        *work = double(n) * 8.0;
    } else {
        return GAMER_E_PARAM;
    }
    return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
}
