// host_fill.cu -- ghost-zone preparation on the host CPU for levels that live
// in host memory (paper Sec. 2: the ghost data of each patch group are
// prepared by the CPU; here OpenMP threads over groups).  Pure copies: every
// cell of the 20^3 tile comes from the owning group of the level, with
// periodic wrap or zero-gradient clamp at the level boundary, row by row.
#include <omp.h>

#include <cstdint>
#include <cstring>

#include "gamer_gb300.h"

namespace gamer {
namespace {

inline int wrap_host(int X, int n, int bc) {
    if (bc == 0) {
        X %= n;
        return X < 0 ? X + n : X;
    }
    return X < 0 ? 0 : (X >= n ? n - 1 : X);
}

}  // namespace

// Fills tiles g in [g0, g1) of the level into out (tile g at out + (g - g0)).
// Per (k, j) row the source rows of all five variables are found once; each
// 20-cell row is the interior 16-cell run of its own group plus two 2-cell
// runs from the x neighbours (the same group when the level is one group wide).
template <class T>
void fill_tiles_host(const T* level, T* out, int gx, int gy, int gz, int bc, int64_t g0,
                     int64_t g1, int nthreads) {
    const int nx = 16 * gx, ny = 16 * gy, nz = 16 * gz;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t g = g0; g < g1; ++g) {
        const int bx = int(g % gx), by = int((g / gx) % gy), bz = int(g / (int64_t(gx) * gy));
        T* dst = out + (g - g0) * 40000;
        const int xl0 = wrap_host(bx * 16 - 2, nx, bc), xl1 = wrap_host(bx * 16 - 1, nx, bc);
        const int xr0 = wrap_host(bx * 16 + 16, nx, bc), xr1 = wrap_host(bx * 16 + 17, nx, bc);
        const int64_t gxl0 = xl0 >> 4, gxl1 = xl1 >> 4, gxr0 = xr0 >> 4, gxr1 = xr1 >> 4;
        const int oxl0 = xl0 & 15, oxl1 = xl1 & 15, oxr0 = xr0 & 15, oxr1 = xr1 & 15;
        for (int k = 0; k < 20; ++k) {
            const int Z = wrap_host(bz * 16 + k - 2, nz, bc);
            for (int j = 0; j < 20; ++j) {
                const int Y = wrap_host(by * 16 + j - 2, ny, bc);
                const int64_t rowg = (int64_t(Z >> 4) * gy + (Y >> 4)) * gx;
                const size_t rowoff = size_t(Z & 15) * 256 + size_t(Y & 15) * 16;
                const T* own = level + (rowg + bx) * 20480 + rowoff;
                const T* l0 = level + (rowg + gxl0) * 20480 + rowoff + oxl0;
                const T* l1 = level + (rowg + gxl1) * 20480 + rowoff + oxl1;
                const T* r0 = level + (rowg + gxr0) * 20480 + rowoff + oxr0;
                const T* r1 = level + (rowg + gxr1) * 20480 + rowoff + oxr1;
                T* d = dst + k * 400 + j * 20;
                for (int v = 0; v < 5; ++v) {
                    const size_t vo = size_t(v) * 4096;
                    T* dv = d + v * 8000;
                    dv[0] = l0[vo];
                    dv[1] = l1[vo];
                    std::memcpy(dv + 2, own + vo, 16 * sizeof(T));
                    dv[18] = r0[vo];
                    dv[19] = r1[vo];
                }
            }
        }
    }
}

template void fill_tiles_host<float>(const float*, float*, int, int, int, int, int64_t, int64_t,
                                     int);
template void fill_tiles_host<double>(const double*, double*, int, int, int, int, int64_t,
                                      int64_t, int);

namespace {

template <class T>
int fill_host(const T* level, T* in, int32_t gx, int32_t gy, int32_t gz, int32_t bc,
              int32_t nthreads) {
    if (gx < 0 || gy < 0 || gz < 0 || (bc != 0 && bc != 1)) return GAMER_E_PARAM;
    const int64_t G = int64_t(gx) * gy * gz;
    if (G == 0) return GAMER_OK;
    if (!level || !in) return GAMER_E_NULL;
    if (int64_t(gx) * 16 > (1 << 30) || int64_t(gy) * 16 > (1 << 30) ||
        int64_t(gz) * 16 > (1 << 30))
        return GAMER_E_PARAM;
    const uintptr_t a = reinterpret_cast<uintptr_t>(level), b = reinterpret_cast<uintptr_t>(in);
    if (a < b + size_t(G) * 40000 * sizeof(T) && b < a + size_t(G) * 20480 * sizeof(T))
        return GAMER_E_OVERLAP;
    if (nthreads < 1) nthreads = omp_get_max_threads();
    fill_tiles_host<T>(level, in, gx, gy, gz, bc, 0, G, nthreads);
    return GAMER_OK;
}

}  // namespace
}  // namespace gamer

extern "C" int gamer_fill_ghosts_uniform_host_f32(const float* level, float* in, int32_t gx,
                                                  int32_t gy, int32_t gz, int32_t bc,
                                                  int32_t nthreads) {
    return gamer::fill_host<float>(level, in, gx, gy, gz, bc, nthreads);
}

extern "C" int gamer_fill_ghosts_uniform_host_f64(const double* level, double* in, int32_t gx,
                                                  int32_t gy, int32_t gz, int32_t bc,
                                                  int32_t nthreads) {
    return gamer::fill_host<double>(level, in, gx, gy, gz, bc, nthreads);
}
