// ghost_fill.cu -- ghost-zone preparation for a uniform level (paper Sec. 2:
// the ghost-zone data each patch group needs before the hydro solver runs).
//
// One CTA per (group, variable) writes the 20^3 padded tile with 16-byte
// vector stores (4 floats / 2 doubles along x; tile rows are 80 / 160 bytes,
// so every row starts 16-byte aligned); each element is gathered from the
// owning group of the level (periodic wrap or clamp at the level boundary).
#include <cuda_runtime.h>

#include "abi_common.h"

namespace gamer {
namespace {

template <class T> struct Vec;
template <> struct Vec<float> { using V = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using V = double2; static constexpr int n = 2; };

__device__ __forceinline__ int wrap_coord(int X, int n, int bc) {
    if (bc == 0) {
        X = X % n;
        return X < 0 ? X + n : X;
    }
    return X < 0 ? 0 : (X >= n ? n - 1 : X);
}

template <class T>
__global__ void __launch_bounds__(256) fill_ghosts_kernel(const T* __restrict__ level,
                                                          T* __restrict__ in, int gx, int gy,
                                                          int gz, int bc) {
    using V = typename Vec<T>::V;
    constexpr int NV = Vec<T>::n;
    const int g = blockIdx.x / 5, v = blockIdx.x % 5;
    const int bx = g % gx, by = (g / gx) % gy, bz = g / (gx * gy);
    const int nx = 16 * gx, ny = 16 * gy, nz = 16 * gz;
    T* dst = in + (size_t(g) * 5 + v) * 8000;
    for (int e = threadIdx.x; e < 8000 / NV; e += blockDim.x) {
        const int c = e * NV;
        const int k = c / 400, j = (c / 20) % 20, i0 = c % 20;
        const int Z = wrap_coord(bz * 16 + k - 2, nz, bc);
        const int Y = wrap_coord(by * 16 + j - 2, ny, bc);
        const size_t rowbase = ((size_t(Z >> 4) * gy + (Y >> 4)) * gx) * 20480 +
                               size_t(v) * 4096 + size_t(Z & 15) * 256 + size_t(Y & 15) * 16;
        T vals[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const int X = wrap_coord(bx * 16 + i0 + t - 2, nx, bc);
            vals[t] = level[rowbase + size_t(X >> 4) * 20480 + (X & 15)];
        }
        V w;
        if constexpr (NV == 4) {
            w = make_float4(vals[0], vals[1], vals[2], vals[3]);
        } else {
            w = make_double2(vals[0], vals[1]);
        }
        reinterpret_cast<V*>(dst)[e] = w;
    }
}

template <class T>
int fill_ghosts(const T* level, T* in, int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                void* stream) {
    if (gx < 0 || gy < 0 || gz < 0 || (bc != 0 && bc != 1)) return GAMER_E_PARAM;
    const int64_t G = int64_t(gx) * gy * gz;
    if (G == 0) return GAMER_OK;
    if (!level || !in) return GAMER_E_NULL;
    if (int64_t(gx) * 16 > (1 << 30) || int64_t(gy) * 16 > (1 << 30) ||
        int64_t(gz) * 16 > (1 << 30) || G * 5 > 0x7fffffffLL)
        return GAMER_E_PARAM;
    if (!aligned(level, sizeof(T)) || !aligned(in, 16)) return GAMER_E_ALIGN;
    if (overlaps(level, size_t(G) * 20480 * sizeof(T), in, size_t(G) * 40000 * sizeof(T)))
        return GAMER_E_OVERLAP;
    const int rc = device_ok();
    if (rc != GAMER_OK) return rc;
    fill_ghosts_kernel<T><<<unsigned(G * 5), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        level, in, gx, gy, gz, bc);
    return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
}

}  // namespace
}  // namespace gamer

extern "C" int gamer_fill_ghosts_uniform_f32(const float* level, float* in, int32_t gx,
                                             int32_t gy, int32_t gz, int32_t bc, void* stream) {
    return gamer::fill_ghosts<float>(level, in, gx, gy, gz, bc, stream);
}

extern "C" int gamer_fill_ghosts_uniform_f64(const double* level, double* in, int32_t gx,
                                             int32_t gy, int32_t gz, int32_t bc, void* stream) {
    return gamer::fill_ghosts<double>(level, in, gx, gy, gz, bc, stream);
}
