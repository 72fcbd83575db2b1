// amr.cu -- coarse-fine coupling after one coarse step and its fine sub-steps
// (the step that consumes the face fluxes the hydro step emits): the
// conservative flux fix-up of the coarse cells beside a fine region and the
// restriction of fine groups onto the coarse octants they cover.  The paper
// relies on GAMER's AMR structure for both without describing them; this is
// the standard refluxing of Berger & Colella (1989) for refinement ratio 2,
// with fine patch groups covering one coarse octant each.
//
// Both kernels do their arithmetic in FP64 with explicitly rounded operations
// (no contraction), in the same order as the definition, and round once to
// the storage type: the FP64 entry points reproduce the definition bit for
// bit, and a cell corrected by one record does so in FP32 as well.
#include <cstdint>

#include "abi_common.h"
#include "gamer_gb300.h"

namespace gamer {
namespace {

constexpr int kFixupThreads = 64;     // one thread per coarse face of a record's 8x8 quadrant
constexpr int kRestrictThreads = 256;

__device__ __forceinline__ bool face_ok(const gamer_cf_face& F, int64_t Nc, int64_t Nf) {
    return F.coarse >= 0 && F.coarse < Nc && F.fine >= 0 && F.fine < Nf && F.dir >= 0 &&
           F.dir <= 2 && F.plane >= 0 && F.plane <= 2 && (F.side == 0 || F.side == 1) &&
           F.quadrant >= 0 && F.quadrant <= 3 && !(F.side == 1 && F.plane == 0) &&
           !(F.side == 0 && F.plane == 2);
}

// Records of class cls = 2*dir + side only: within a class no two records
// touch the same coarse cell (a cell has one face per direction and side), so
// the six class launches are free of races and their order is fixed.
template <class T>
__global__ void __launch_bounds__(kFixupThreads)
    flux_fixup_kernel(T* __restrict__ coarse, const T* __restrict__ cflux,
                      const T* __restrict__ fflux, int n_sub, const double* __restrict__ dt,
                      const double* __restrict__ dh, int64_t Nc, int64_t Nf,
                      const gamer_cf_face* __restrict__ faces, int64_t n, int cls,
                      int32_t* __restrict__ bad) {
    const int t = threadIdx.x;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const gamer_cf_face F = faces[r];
        if (!face_ok(F, Nc, Nf)) {
            if (cls == 0 && t == 0 && bad) atomicAdd(bad, 1);
            continue;
        }
        if (2 * F.dir + F.side != cls) continue;
        const int a0 = (F.quadrant & 1) ? 8 : 0, b0 = (F.quadrant & 2) ? 8 : 0;
        const int a = a0 + (t >> 3), b = b0 + (t & 7);
        const int layer = F.side ? 8 * F.plane - 1 : 8 * F.plane;
        const int fface = 2 * F.dir + (F.side ? 0 : 1);  // the fine group's face
        int i, j, k;
        if (F.dir == 0) {
            k = a; j = b; i = layer;
        } else if (F.dir == 1) {
            k = a; i = b; j = layer;
        } else {
            j = a; i = b; k = layer;
        }
        const double lam = __ddiv_rn(dt[F.coarse], dh[F.coarse]);
        const double cnt = double(4 * n_sub);  // fine faces x sub-steps
        const T* Fc = cflux + (F.coarse * 9 + 3 * F.dir + F.plane) * int64_t(1280);
        T* U = coarse + F.coarse * int64_t(20480);
        const int A0 = 2 * (a - a0), B0 = 2 * (b - b0);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            double sum = 0.0;
            for (int s = 0; s < n_sub; ++s) {
                const T* Ff = fflux + ((s * Nf + F.fine) * 6 + fface) * int64_t(1280) + q * 256;
#pragma unroll
                for (int dA = 0; dA < 2; ++dA)
#pragma unroll
                    for (int dB = 0; dB < 2; ++dB)
                        sum = __dadd_rn(sum, double(Ff[(A0 + dA) * 16 + B0 + dB]));
            }
            const double mean = __ddiv_rn(sum, cnt);
            const double corr = __dmul_rn(lam, __dsub_rn(double(Fc[q * 256 + a * 16 + b]), mean));
            T& u = U[((q * 16 + k) * 16 + j) * 16 + i];
            const double un = F.side ? __dadd_rn(double(u), corr) : __dsub_rn(double(u), corr);
            u = T(un);
        }
    }
}

template <class T>
__global__ void __launch_bounds__(kRestrictThreads)
    restrict_kernel(const T* __restrict__ fine, T* __restrict__ coarse, int64_t Nc, int64_t Nf,
                    const gamer_cf_child* __restrict__ children, int64_t n,
                    int32_t* __restrict__ bad) {
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const gamer_cf_child C = children[r];
        if (!(C.coarse >= 0 && C.coarse < Nc && C.fine >= 0 && C.fine < Nf && C.octant >= 0 &&
              C.octant <= 7)) {
            if (threadIdx.x == 0 && bad) atomicAdd(bad, 1);
            continue;
        }
        const int ox = (C.octant & 1) ? 8 : 0, oy = (C.octant & 2) ? 8 : 0,
                  oz = (C.octant & 4) ? 8 : 0;
        const T* f = fine + C.fine * int64_t(20480);
        T* c = coarse + C.coarse * int64_t(20480);
        // 5 x 8^3 coarse cells, x fastest across the threads
        for (int it = threadIdx.x; it < 2560; it += kRestrictThreads) {
            const int i = it & 7, j = (it >> 3) & 7, k = (it >> 6) & 7, q = it >> 9;
            double sum = 0.0;
#pragma unroll
            for (int dk = 0; dk < 2; ++dk)
#pragma unroll
                for (int dj = 0; dj < 2; ++dj)
#pragma unroll
                    for (int di = 0; di < 2; ++di)
                        sum = __dadd_rn(
                            sum, double(f[((q * 16 + 2 * k + dk) * 16 + 2 * j + dj) * 16 + 2 * i +
                                          di]));
            c[((q * 16 + oz + k) * 16 + oy + j) * 16 + ox + i] = T(__dmul_rn(sum, 0.125));
        }
    }
}

int64_t grid_for(int64_t n) {
    DeviceInfo d = current_device();
    const int64_t cap = int64_t(d.sm_count > 0 ? d.sm_count : 1) * 16;
    return n < cap ? n : cap;
}

template <class T>
int flux_fixup(T* coarse, const T* cflux, const T* fflux, int32_t n_sub, const double* dt,
               const double* dh, int64_t Nc, int64_t Nf, const gamer_cf_face* faces, int64_t n,
               int32_t* bad, void* stream) {
    if (n < 0 || Nc < 0 || Nf < 0 || n_sub < 1) return GAMER_E_PARAM;
    if (n == 0) return GAMER_OK;
    if (!coarse || !cflux || !fflux || !dt || !dh || !faces) return GAMER_E_NULL;
    if (!aligned(coarse, sizeof(T)) || !aligned(cflux, sizeof(T)) ||
        !aligned(fflux, sizeof(T)) || !aligned(dt, 8) || !aligned(dh, 8) || !aligned(faces, 8) ||
        !aligned(bad, 4))
        return GAMER_E_ALIGN;
    const size_t nc = size_t(Nc) * 20480 * sizeof(T);
    const void* ins[5] = {cflux, fflux, dt, dh, faces};
    const size_t insz[5] = {size_t(Nc) * 11520 * sizeof(T),
                            size_t(n_sub) * size_t(Nf) * 7680 * sizeof(T), size_t(Nc) * 8,
                            size_t(Nc) * 8, size_t(n) * sizeof(gamer_cf_face)};
    for (int b = 0; b < 5; ++b)
        if (overlaps(coarse, nc, ins[b], insz[b]) || overlaps(bad, 4, ins[b], insz[b]))
            return GAMER_E_OVERLAP;
    if (overlaps(coarse, nc, bad, 4)) return GAMER_E_OVERLAP;
    DeviceInfo d = current_device();
    if (d.status != GAMER_OK) return d.status;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned grid = unsigned(grid_for(n));
    for (int cls = 0; cls < 6; ++cls)
        flux_fixup_kernel<T><<<grid, kFixupThreads, 0, s>>>(coarse, cflux, fflux, n_sub, dt, dh,
                                                            Nc, Nf, faces, n, cls, bad);
    return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
}

template <class T>
int restrict_groups(const T* fine, T* coarse, int64_t Nc, int64_t Nf,
                    const gamer_cf_child* children, int64_t n, int32_t* bad, void* stream) {
    if (n < 0 || Nc < 0 || Nf < 0) return GAMER_E_PARAM;
    if (n == 0) return GAMER_OK;
    if (!fine || !coarse || !children) return GAMER_E_NULL;
    if (!aligned(fine, sizeof(T)) || !aligned(coarse, sizeof(T)) || !aligned(children, 8) ||
        !aligned(bad, 4))
        return GAMER_E_ALIGN;
    const size_t nc = size_t(Nc) * 20480 * sizeof(T);
    if (overlaps(coarse, nc, fine, size_t(Nf) * 20480 * sizeof(T)) ||
        overlaps(coarse, nc, children, size_t(n) * sizeof(gamer_cf_child)) ||
        overlaps(coarse, nc, bad, 4))
        return GAMER_E_OVERLAP;
    DeviceInfo d = current_device();
    if (d.status != GAMER_OK) return d.status;
    restrict_kernel<T><<<unsigned(grid_for(n)), kRestrictThreads, 0,
                         static_cast<cudaStream_t>(stream)>>>(fine, coarse, Nc, Nf, children, n,
                                                              bad);
    return cudaGetLastError() == cudaSuccess ? GAMER_OK : GAMER_E_CUDA;
}

}  // namespace
}  // namespace gamer

extern "C" int gamer_flux_fixup_f32(float* coarse, const float* coarse_flux,
                                    const float* fine_flux, int32_t n_sub, const double* dt,
                                    const double* dh, int64_t Nc, int64_t Nf,
                                    const gamer_cf_face* faces, int64_t n_faces, int32_t* bad,
                                    void* stream) {
    return gamer::flux_fixup<float>(coarse, coarse_flux, fine_flux, n_sub, dt, dh, Nc, Nf, faces,
                                    n_faces, bad, stream);
}

extern "C" int gamer_flux_fixup_f64(double* coarse, const double* coarse_flux,
                                    const double* fine_flux, int32_t n_sub, const double* dt,
                                    const double* dh, int64_t Nc, int64_t Nf,
                                    const gamer_cf_face* faces, int64_t n_faces, int32_t* bad,
                                    void* stream) {
    return gamer::flux_fixup<double>(coarse, coarse_flux, fine_flux, n_sub, dt, dh, Nc, Nf,
                                     faces, n_faces, bad, stream);
}

extern "C" int gamer_restrict_f32(const float* fine, float* coarse, int64_t Nc, int64_t Nf,
                                  const gamer_cf_child* children, int64_t n_children,
                                  int32_t* bad, void* stream) {
    return gamer::restrict_groups<float>(fine, coarse, Nc, Nf, children, n_children, bad, stream);
}

extern "C" int gamer_restrict_f64(const double* fine, double* coarse, int64_t Nc, int64_t Nf,
                                  const gamer_cf_child* children, int64_t n_children,
                                  int32_t* bad, void* stream) {
    return gamer::restrict_groups<double>(fine, coarse, Nc, Nf, children, n_children, bad,
                                          stream);
}
