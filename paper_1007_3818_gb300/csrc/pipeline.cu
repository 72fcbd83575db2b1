// pipeline.cu -- host-resident batches streamed through the GPU: host->device
// copy, hydro step and device->host copy of successive batches overlap on
// three streams (the paper overlaps CPU ghost preparation, GPU solves and disk
// I/O the same way, Sec. 2 and Sec. 3).  The pipeline owns its device buffers
// (allocated once at creation); advance_host itself allocates nothing.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <new>

#include "abi_common.h"
#include "gamer_gb300.h"

extern "C" int gamer_hydro_advance_f32(const float*, float*, float*, const double*, const double*,
                                       uint32_t*, double*, int64_t, const gh_params*, void*);
extern "C" int gamer_hydro_advance_mixed(const float*, float*, float*, const double*,
                                         const double*, uint32_t*, double*, int64_t,
                                         const gh_params*, void*);
extern "C" int gamer_hydro_advance_f64(const double*, double*, double*, const double*,
                                       const double*, uint32_t*, double*, int64_t,
                                       const gh_params*, void*);

namespace {

constexpr int kSets = 3;  // buffer sets in flight

struct BufSet {
    void* in = nullptr;
    void* out = nullptr;
    void* ff = nullptr;
    double* dt = nullptr;
    double* dh = nullptr;
    uint32_t* status = nullptr;
    double* partials = nullptr;
    cudaEvent_t h2d_done = nullptr, comp_done = nullptr, d2h_done = nullptr;
    bool used = false;
};

}  // namespace

struct gamer_pipeline {
    // pinned host staging of ghost-padded tiles for level steps (allocated on
    // the first gamer_pipeline_level_step_host call)
    void* staging[3] = {nullptr, nullptr, nullptr};
    double* stage_dt = nullptr;  // pinned [2][batch]: dt, dh of a level step
    int mode = 0;
    int64_t batch = 0;
    int with_flux = 0;
    size_t esz = 4;
    int device = -1;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    BufSet set[kSets];
    double timeout_s = 60.0;
};

namespace {

void release(gamer_pipeline* pl) {
    if (!pl) return;
    for (auto& st : pl->staging)
        if (st) cudaFreeHost(st);
    if (pl->stage_dt) cudaFreeHost(pl->stage_dt);
    for (auto& b : pl->set) {
        cudaFree(b.in);
        cudaFree(b.out);
        cudaFree(b.ff);
        cudaFree(b.dt);
        cudaFree(b.dh);
        cudaFree(b.status);
        cudaFree(b.partials);
        if (b.h2d_done) cudaEventDestroy(b.h2d_done);
        if (b.comp_done) cudaEventDestroy(b.comp_done);
        if (b.d2h_done) cudaEventDestroy(b.d2h_done);
    }
    if (pl->s_h2d) cudaStreamDestroy(pl->s_h2d);
    if (pl->s_comp) cudaStreamDestroy(pl->s_comp);
    if (pl->s_d2h) cudaStreamDestroy(pl->s_d2h);
    delete pl;
}

// Waits for `ev` by polling with a deadline (never blocks indefinitely).
int wait_event(cudaEvent_t ev, double timeout_s) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return GAMER_OK;
        if (e != cudaErrorNotReady) return GAMER_E_CUDA;
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return GAMER_E_TIMEOUT;
    }
}

}  // namespace

extern "C" int gamer_pipeline_create(int32_t mode, int64_t batch_groups, int32_t with_flux,
                                     gamer_pipeline** out) {
    using namespace gamer;
    if (!out) return GAMER_E_NULL;
    *out = nullptr;
    if (mode < 0 || mode > 2 || batch_groups < 1 || batch_groups > (int64_t(1) << 24))
        return GAMER_E_PARAM;
    const DeviceInfo d = current_device();
    if (d.status != GAMER_OK) return d.status;
    gamer_pipeline* pl = new (std::nothrow) gamer_pipeline();
    if (!pl) return GAMER_E_CUDA;
    pl->mode = mode;
    pl->batch = batch_groups;
    pl->with_flux = with_flux ? 1 : 0;
    pl->esz = (mode == GAMER_MODE_F64) ? 8 : 4;
    pl->device = d.device;
    bool ok = cudaStreamCreateWithFlags(&pl->s_h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pl->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&pl->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
    const size_t B = size_t(batch_groups);
    for (auto& b : pl->set) {
        if (!ok) break;
        ok = cudaMalloc(&b.in, B * 40000 * pl->esz) == cudaSuccess &&
             cudaMalloc(&b.out, B * 20480 * pl->esz) == cudaSuccess &&
             (!pl->with_flux || cudaMalloc(&b.ff, B * 9 * 1280 * pl->esz) == cudaSuccess) &&
             cudaMalloc(&b.dt, B * 8) == cudaSuccess && cudaMalloc(&b.dh, B * 8) == cudaSuccess &&
             cudaMalloc(&b.status, B * 4) == cudaSuccess &&
             cudaMalloc(&b.partials, B * 48) == cudaSuccess &&
             cudaEventCreateWithFlags(&b.h2d_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&b.comp_done, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&b.d2h_done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        release(pl);
        cudaGetLastError();
        return GAMER_E_CUDA;
    }
    *out = pl;
    return GAMER_OK;
}

extern "C" int gamer_pipeline_destroy(gamer_pipeline* pl) {
    if (!pl) return GAMER_E_NULL;
    cudaStreamSynchronize(pl->s_h2d);
    cudaStreamSynchronize(pl->s_comp);
    cudaStreamSynchronize(pl->s_d2h);
    release(pl);
    return GAMER_OK;
}

extern "C" int gamer_pipeline_advance_host(gamer_pipeline* pl, const void* in_host,
                                           void* out_host, void* face_flux_host,
                                           const double* dt_host, const double* dh_host,
                                           uint32_t* status_host, double* partials_host, int64_t N,
                                           const gh_params* p) {
    using namespace gamer;
    if (!pl) return GAMER_E_NULL;
    if (N < 0) return GAMER_E_PARAM;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    if (N == 0) return GAMER_OK;
    if (!in_host || !out_host || !dt_host || !dh_host) return GAMER_E_NULL;
    if (face_flux_host && !pl->with_flux) return GAMER_E_PARAM;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != pl->device) return GAMER_E_DEVICE;
    const size_t e = pl->esz;
    const size_t ffg = size_t(p->flux_layout ? 9 : 6) * 1280;  // face-flux values per group
    const char* hin = static_cast<const char*>(in_host);
    char* hout = static_cast<char*>(out_host);
    char* hff = static_cast<char*>(face_flux_host);
    const int64_t nb = (N + pl->batch - 1) / pl->batch;
    for (int64_t b = 0; b < nb; ++b) {
        BufSet& S = pl->set[b % kSets];
        const int64_t g0 = b * pl->batch;
        const int64_t n = std::min<int64_t>(pl->batch, N - g0);
        // the set's previous copies back to the host must be done before reuse
        if (S.used && cudaStreamWaitEvent(pl->s_h2d, S.d2h_done, 0) != cudaSuccess)
            return GAMER_E_CUDA;
        bool ok = cudaMemcpyAsync(S.in, hin + size_t(g0) * 40000 * e, size_t(n) * 40000 * e,
                                  cudaMemcpyHostToDevice, pl->s_h2d) == cudaSuccess &&
                  cudaMemcpyAsync(S.dt, dt_host + g0, size_t(n) * 8, cudaMemcpyHostToDevice,
                                  pl->s_h2d) == cudaSuccess &&
                  cudaMemcpyAsync(S.dh, dh_host + g0, size_t(n) * 8, cudaMemcpyHostToDevice,
                                  pl->s_h2d) == cudaSuccess &&
                  cudaEventRecord(S.h2d_done, pl->s_h2d) == cudaSuccess &&
                  cudaStreamWaitEvent(pl->s_comp, S.h2d_done, 0) == cudaSuccess;
        if (!ok) return GAMER_E_CUDA;
        void* ff = (hff && S.ff) ? S.ff : nullptr;
        if (pl->mode == GAMER_MODE_F32)
            rc = gamer_hydro_advance_f32((const float*)S.in, (float*)S.out, (float*)ff, S.dt, S.dh,
                                         S.status, S.partials, n, p, pl->s_comp);
        else if (pl->mode == GAMER_MODE_MIXED)
            rc = gamer_hydro_advance_mixed((const float*)S.in, (float*)S.out, (float*)ff, S.dt,
                                           S.dh, S.status, S.partials, n, p, pl->s_comp);
        else
            rc = gamer_hydro_advance_f64((const double*)S.in, (double*)S.out, (double*)ff, S.dt,
                                         S.dh, S.status, S.partials, n, p, pl->s_comp);
        if (rc != GAMER_OK) return rc;
        ok = cudaEventRecord(S.comp_done, pl->s_comp) == cudaSuccess &&
             cudaStreamWaitEvent(pl->s_d2h, S.comp_done, 0) == cudaSuccess &&
             cudaMemcpyAsync(hout + size_t(g0) * 20480 * e, S.out, size_t(n) * 20480 * e,
                             cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        if (ok && ff)
            ok = cudaMemcpyAsync(hff + size_t(g0) * ffg * e, S.ff, size_t(n) * ffg * e,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        if (ok && status_host)
            ok = cudaMemcpyAsync(status_host + g0, S.status, size_t(n) * 4,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        if (ok && partials_host)
            ok = cudaMemcpyAsync(partials_host + g0 * 6, S.partials, size_t(n) * 48,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        ok = ok && cudaEventRecord(S.d2h_done, pl->s_d2h) == cudaSuccess;
        if (!ok) return GAMER_E_CUDA;
        S.used = true;
    }
    // results are in host memory when the last device->host copies are done
    const BufSet& last = pl->set[(nb - 1) % kSets];
    return wait_event(last.d2h_done, pl->timeout_s);
}

namespace gamer {
template <class T>
void fill_tiles_host(const T* level, T* out, int gx, int gy, int gz, int bc, int64_t g0,
                     int64_t g1, int nthreads);
}

extern "C" int gamer_pipeline_level_step_host(gamer_pipeline* pl, const void* level_in_host,
                                              void* level_out_host, int32_t gx, int32_t gy,
                                              int32_t gz, int32_t bc, double dt, double dh,
                                              uint32_t* status_host, double* partials_host,
                                              const gh_params* p, int32_t nthreads) {
    using namespace gamer;
    if (!pl) return GAMER_E_NULL;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    if (gx < 0 || gy < 0 || gz < 0 || (bc != 0 && bc != 1)) return GAMER_E_PARAM;
    const int64_t G = int64_t(gx) * gy * gz;
    if (G == 0) return GAMER_OK;
    if (!level_in_host || !level_out_host) return GAMER_E_NULL;
    if (level_in_host == level_out_host) return GAMER_E_OVERLAP;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != pl->device) return GAMER_E_DEVICE;
    const size_t e = pl->esz;
    const size_t tile_bytes = size_t(pl->batch) * 40000 * e;
    if (!pl->staging[0]) {
        for (auto& st : pl->staging)
            if (cudaHostAlloc(&st, tile_bytes, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                return GAMER_E_CUDA;
            }
        if (cudaHostAlloc(reinterpret_cast<void**>(&pl->stage_dt), size_t(pl->batch) * 16,
                          cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return GAMER_E_CUDA;
        }
    }
    // every group of the level takes the same dt and dh
    for (int64_t i = 0; i < pl->batch; ++i) {
        pl->stage_dt[i] = dt;
        pl->stage_dt[pl->batch + i] = dh;
    }
    const double* hdt = pl->stage_dt;
    const double* hdh = pl->stage_dt + pl->batch;
    char* hout = static_cast<char*>(level_out_host);
    const int64_t nb = (G + pl->batch - 1) / pl->batch;
    for (int64_t b = 0; b < nb; ++b) {
        BufSet& S = pl->set[b % kSets];
        char* stg = static_cast<char*>(pl->staging[b % kSets]);
        const int64_t g0 = b * pl->batch;
        const int64_t n = std::min<int64_t>(pl->batch, G - g0);
        // the staging buffer is refilled only once its previous copy has left
        if (S.used && (rc = wait_event(S.h2d_done, pl->timeout_s)) != GAMER_OK) return rc;
        // host ghost preparation of this batch overlaps the GPU work queued before it
        if (pl->mode == GAMER_MODE_F64)
            fill_tiles_host<double>(static_cast<const double*>(level_in_host),
                                    reinterpret_cast<double*>(stg), gx, gy, gz, bc, g0, g0 + n,
                                    nthreads);
        else
            fill_tiles_host<float>(static_cast<const float*>(level_in_host),
                                   reinterpret_cast<float*>(stg), gx, gy, gz, bc, g0, g0 + n,
                                   nthreads);
        if (S.used && cudaStreamWaitEvent(pl->s_h2d, S.d2h_done, 0) != cudaSuccess)
            return GAMER_E_CUDA;
        bool ok = cudaMemcpyAsync(S.in, stg, size_t(n) * 40000 * e, cudaMemcpyHostToDevice,
                                  pl->s_h2d) == cudaSuccess &&
                  cudaMemcpyAsync(S.dt, hdt, size_t(n) * 8, cudaMemcpyHostToDevice,
                                  pl->s_h2d) == cudaSuccess &&
                  cudaMemcpyAsync(S.dh, hdh, size_t(n) * 8, cudaMemcpyHostToDevice,
                                  pl->s_h2d) == cudaSuccess &&
                  cudaEventRecord(S.h2d_done, pl->s_h2d) == cudaSuccess &&
                  cudaStreamWaitEvent(pl->s_comp, S.h2d_done, 0) == cudaSuccess;
        if (!ok) return GAMER_E_CUDA;
        if (pl->mode == GAMER_MODE_F32)
            rc = gamer_hydro_advance_f32((const float*)S.in, (float*)S.out, nullptr, S.dt, S.dh,
                                         S.status, S.partials, n, p, pl->s_comp);
        else if (pl->mode == GAMER_MODE_MIXED)
            rc = gamer_hydro_advance_mixed((const float*)S.in, (float*)S.out, nullptr, S.dt,
                                           S.dh, S.status, S.partials, n, p, pl->s_comp);
        else
            rc = gamer_hydro_advance_f64((const double*)S.in, (double*)S.out, nullptr, S.dt,
                                         S.dh, S.status, S.partials, n, p, pl->s_comp);
        if (rc != GAMER_OK) return rc;
        ok = cudaEventRecord(S.comp_done, pl->s_comp) == cudaSuccess &&
             cudaStreamWaitEvent(pl->s_d2h, S.comp_done, 0) == cudaSuccess &&
             cudaMemcpyAsync(hout + size_t(g0) * 20480 * e, S.out, size_t(n) * 20480 * e,
                             cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        if (ok && status_host)
            ok = cudaMemcpyAsync(status_host + g0, S.status, size_t(n) * 4,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        if (ok && partials_host)
            ok = cudaMemcpyAsync(partials_host + g0 * 6, S.partials, size_t(n) * 48,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        ok = ok && cudaEventRecord(S.d2h_done, pl->s_d2h) == cudaSuccess;
        if (!ok) return GAMER_E_CUDA;
        S.used = true;
    }
    return wait_event(pl->set[(nb - 1) % kSets].d2h_done, pl->timeout_s);
}

extern "C" int gamer_pipeline_set_timeout(gamer_pipeline* pl, double seconds) {
    if (!pl) return GAMER_E_NULL;
    if (!(seconds > 0.0)) return GAMER_E_PARAM;
    pl->timeout_s = seconds;
    return GAMER_OK;
}
