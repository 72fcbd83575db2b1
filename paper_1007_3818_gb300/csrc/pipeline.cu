// pipeline.cu -- host-resident data streamed through the GPU: host->device
// copy, hydro step and device->host copy of successive batches overlap on
// three streams (the paper overlaps CPU ghost preparation, GPU solves and disk
// I/O the same way, Sec. 2 and Sec. 3).  Tile batches use the buffers
// allocated at creation; a host-resident level is streamed in z-slabs of its
// 16^3 interiors with a one-layer halo on each side, the ghost zones being
// gathered on the device (window buffers allocated on first use).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <climits>
#include <chrono>
#include <cstring>
#include <new>
#include <thread>

#include "abi_common.h"
#include "gamer_gb300.h"

extern "C" int gamer_hydro_advance_f32(const float*, float*, float*, const double*, const double*,
                                       uint32_t*, double*, int64_t, const gh_params*, void*);
extern "C" int gamer_hydro_advance_mixed(const float*, float*, float*, const double*,
                                         const double*, uint32_t*, double*, int64_t,
                                         const gh_params*, void*);
extern "C" int gamer_hydro_advance_ff(const float*, float*, float*, const double*,
                                         const double*, uint32_t*, double*, int64_t,
                                         const gh_params*, void*);
extern "C" int gamer_hydro_advance_f64(const double*, double*, double*, const double*,
                                       const double*, uint32_t*, double*, int64_t,
                                       const gh_params*, void*);
extern "C" int gamer_hydro_advance_level_window_f32(const float*, float*, float*, int32_t, int32_t,
                                                    int32_t, int32_t, int32_t, int32_t, int32_t,
                                                    int32_t, const double*, const double*,
                                                    uint32_t*, double*, const gh_params*, void*);
extern "C" int gamer_hydro_advance_level_window_mixed(const float*, float*, float*, int32_t,
                                                      int32_t, int32_t, int32_t, int32_t, int32_t,
                                                      int32_t, int32_t, const double*,
                                                      const double*, uint32_t*, double*,
                                                      const gh_params*, void*);
extern "C" int gamer_hydro_advance_level_window_ff(const float*, float*, float*, int32_t,
                                                      int32_t, int32_t, int32_t, int32_t, int32_t,
                                                      int32_t, int32_t, const double*,
                                                      const double*, uint32_t*, double*,
                                                      const gh_params*, void*);
extern "C" int gamer_hydro_advance_level_window_f64(const double*, double*, double*, int32_t,
                                                    int32_t, int32_t, int32_t, int32_t, int32_t,
                                                    int32_t, int32_t, const double*,
                                                    const double*, uint32_t*, double*,
                                                    const gh_params*, void*);

extern "C" size_t gamer_hydro_dt_workspace_bytes(int64_t N, int32_t n_levels);
extern "C" int gamer_hydro_dt(const double* partials, int64_t N, const int32_t* level,
                              int32_t n_levels, const double* dh_level, double cfl, double* dt_out,
                              double* totals, double* dt_group, void* workspace,
                              size_t workspace_bytes, void* stream);

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
    // z-slab window of a host-resident level (level steps only)
    void* win = nullptr;
    void* wout = nullptr;
    double* wdt = nullptr;
    uint32_t* wstatus = nullptr;
    double* wpartials = nullptr;
    size_t win_cap = 0, wout_cap = 0, wn_cap = 0;  // bytes, bytes, groups
};

}  // namespace

struct gamer_pipeline {
    double* stage_dt = nullptr;  // pinned [2][n]: dt, dh of a level step
    size_t stage_n = 0;
    // device copy of a whole level (levels that fit): input, output, dt/dh,
    // status, partials; allocated on first use, grown when needed
    void* lev_in = nullptr;
    void* lev_out = nullptr;
    double* lev_dt = nullptr;
    uint32_t* lev_status = nullptr;
    double* lev_partials = nullptr;
    size_t lev_cap = 0;  // groups
    cudaEvent_t lev_ev[3] = {nullptr, nullptr, nullptr};
    int level_mode = 0;  // 0 automatic, 1 device copy of the level, 2 slab windows
    int64_t h2d_bytes = 0, d2h_bytes = 0;  // copied by the last call
    int mode = 0;
    int64_t batch = 0;
    int with_flux = 0;
    size_t esz = 4;
    int device = -1;
    cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
    BufSet set[kSets];
    double timeout_s = 60.0;
    // multi-step runs (level_run_host): device input and output levels by
    // step parity, per-group dt and dh, status of the step and its OR over
    // the steps, partials, dh and the dt of every step, dt workspace, and
    // events [parity][in, out][slab] for the copies of each slab
    void* run_in[2] = {nullptr, nullptr};
    void* run_out[2] = {nullptr, nullptr};
    double* run_dt = nullptr;        // [2][G]: dt, dh per group
    uint32_t* run_status = nullptr;  // [2][G]: this step, OR over the steps
    double* run_partials = nullptr;  // [G][6]
    double* run_aux = nullptr;       // [1 + steps]: dh, then the dt of each step
    void* run_ws = nullptr;
    size_t run_ws_bytes = 0, run_cap = 0, run_level_bytes = 0, run_aux_cap = 0;
    cudaEvent_t* run_ev = nullptr;   // [2][2][run_ev_slabs]
    int32_t run_ev_slabs = 0;
    cudaEvent_t run_comp[2] = {nullptr, nullptr};
    cudaEvent_t run_end = nullptr;
    // a call returned GAMER_E_TIMEOUT with work still queued on the streams:
    // the next call first waits (bounded) for the streams to drain
    bool stuck = false;
};

namespace {

void release_run(gamer_pipeline* pl) {
    for (int i = 0; i < 2; ++i) {
        cudaFree(pl->run_in[i]);
        cudaFree(pl->run_out[i]);
        pl->run_in[i] = pl->run_out[i] = nullptr;
    }
    cudaFree(pl->run_dt);
    cudaFree(pl->run_status);
    cudaFree(pl->run_partials);
    cudaFree(pl->run_aux);
    cudaFree(pl->run_ws);
    pl->run_dt = pl->run_partials = pl->run_aux = nullptr;
    pl->run_status = nullptr;
    pl->run_ws = nullptr;
    pl->run_ws_bytes = pl->run_cap = pl->run_level_bytes = pl->run_aux_cap = 0;
    if (pl->run_ev) {
        for (int32_t i = 0; i < 4 * pl->run_ev_slabs; ++i)
            if (pl->run_ev[i]) cudaEventDestroy(pl->run_ev[i]);
        delete[] pl->run_ev;
        pl->run_ev = nullptr;
    }
    pl->run_ev_slabs = 0;
    for (auto& ev : pl->run_comp)
        if (ev) cudaEventDestroy(ev);
    pl->run_comp[0] = pl->run_comp[1] = nullptr;
    if (pl->run_end) cudaEventDestroy(pl->run_end);
    pl->run_end = nullptr;
}

void release(gamer_pipeline* pl) {
    if (!pl) return;
    release_run(pl);
    if (pl->stage_dt) cudaFreeHost(pl->stage_dt);
    cudaFree(pl->lev_in);
    cudaFree(pl->lev_out);
    cudaFree(pl->lev_dt);
    cudaFree(pl->lev_status);
    cudaFree(pl->lev_partials);
    for (auto& ev : pl->lev_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& b : pl->set) {
        cudaFree(b.in);
        cudaFree(b.out);
        cudaFree(b.ff);
        cudaFree(b.dt);
        cudaFree(b.dh);
        cudaFree(b.status);
        cudaFree(b.partials);
        cudaFree(b.win);
        cudaFree(b.wout);
        cudaFree(b.wdt);
        cudaFree(b.wstatus);
        cudaFree(b.wpartials);
        if (b.h2d_done) cudaEventDestroy(b.h2d_done);
        if (b.comp_done) cudaEventDestroy(b.comp_done);
        if (b.d2h_done) cudaEventDestroy(b.d2h_done);
    }
    if (pl->s_h2d) cudaStreamDestroy(pl->s_h2d);
    if (pl->s_comp) cudaStreamDestroy(pl->s_comp);
    if (pl->s_d2h) cudaStreamDestroy(pl->s_d2h);
    delete pl;
}

// Polls `ready` (cudaSuccess / cudaErrorNotReady / error) with a deadline
// (never blocks indefinitely); after the first polls it sleeps 50 us between
// them, so a long wait leaves the host core to other work.
template <class Q>
int poll_until(Q ready, double timeout_s) {
    const auto t0 = std::chrono::steady_clock::now();
    for (int n = 0;; ++n) {
        const cudaError_t e = ready();
        if (e == cudaSuccess) return GAMER_OK;
        if (e != cudaErrorNotReady) return GAMER_E_CUDA;
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > timeout_s) return GAMER_E_TIMEOUT;
        if (n >= 64) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Waits for `ev` on pipeline pl; a timeout leaves pl marked stuck.
int wait_event(gamer_pipeline* pl, cudaEvent_t ev, double timeout_s) {
    const int rc = poll_until([ev] { return cudaEventQuery(ev); }, timeout_s);
    if (rc == GAMER_E_TIMEOUT) pl->stuck = true;
    return rc;
}

// Start of every call on pl: after a timed-out call, wait (bounded) until
// the pipeline's three streams are idle, so that no copy of the earlier call
// is still due to land in host memory; GAMER_E_TIMEOUT (nothing enqueued) if
// they are not.
int unstick(gamer_pipeline* pl) {
    if (!pl->stuck) return GAMER_OK;
    for (cudaStream_t s : {pl->s_h2d, pl->s_comp, pl->s_d2h}) {
        const int rc = poll_until([s] { return cudaStreamQuery(s); }, pl->timeout_s);
        if (rc != GAMER_OK) return rc;
    }
    pl->stuck = false;
    return GAMER_OK;
}

void CUDART_CB sleep_host(void* seconds) {
    const double s = *static_cast<double*>(seconds);
    std::this_thread::sleep_for(std::chrono::duration<double>(s));
    delete static_cast<double*>(seconds);
}

}  // namespace

extern "C" int gamer_pipeline_create(int32_t mode, int64_t batch_groups, int32_t with_flux,
                                     gamer_pipeline** out) {
    using namespace gamer;
    if (!out) return GAMER_E_NULL;
    *out = nullptr;
    if (mode < 0 || mode > 3 || batch_groups < 1 || batch_groups > (int64_t(1) << 24))
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
    if (const int st = unstick(pl); st != GAMER_OK) return st;
    if (N < 0) return GAMER_E_PARAM;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    pl->h2d_bytes = pl->d2h_bytes = 0;
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
    // bytes this call moves: tiles, dt and dh in; states, fluxes, status, partials out
    pl->h2d_bytes = N * (40000 * int64_t(e) + 16);
    pl->d2h_bytes = N * (20480 * int64_t(e) + (hff ? int64_t(ffg) * int64_t(e) : 0) +
                         (status_host ? 4 : 0) + (partials_host ? 48 : 0));
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
        else if (pl->mode == GAMER_MODE_FF)
            rc = gamer_hydro_advance_ff((const float*)S.in, (float*)S.out, (float*)ff, S.dt,
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
    return wait_event(pl, last.d2h_done, pl->timeout_s);
}

namespace {

// (Re)allocates a set's window buffers for win_bytes of input and n groups.
bool ensure_window(BufSet& S, size_t win_bytes, size_t n, size_t esz) {
    if (S.win_cap < win_bytes) {
        cudaFree(S.win);
        S.win = nullptr;
        S.win_cap = 0;
        if (cudaMalloc(&S.win, win_bytes) != cudaSuccess) return false;
        S.win_cap = win_bytes;
    }
    if (S.wn_cap < n) {
        cudaFree(S.wout);
        cudaFree(S.wdt);
        cudaFree(S.wstatus);
        cudaFree(S.wpartials);
        S.wout = S.wdt = nullptr;
        S.wstatus = nullptr;
        S.wpartials = nullptr;
        S.wn_cap = S.wout_cap = 0;
        if (cudaMalloc(&S.wout, n * 20480 * esz) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&S.wdt), n * 16) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&S.wstatus), n * 4) != cudaSuccess ||
            cudaMalloc(reinterpret_cast<void**>(&S.wpartials), n * 48) != cudaSuccess)
            return false;
        S.wn_cap = n;
        S.wout_cap = n * 20480 * esz;
    }
    return true;
}

// Whether a level of G groups (level_bytes of interiors) is advanced from a
// device copy of the whole level: when that copy exists already or its input
// and output fit in 80 % of the free device memory.  Allocates it if so.
bool level_resident(gamer_pipeline* pl, int64_t G, size_t level_bytes) {
    if (pl->level_mode == 2) return false;
    if (pl->lev_cap >= size_t(G)) return true;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t need = 2 * level_bytes + size_t(G) * (16 + 4 + 48);
    if (pl->level_mode == 0 && double(need) > 0.8 * double(free_b)) return false;
    cudaFree(pl->lev_in);
    cudaFree(pl->lev_out);
    cudaFree(pl->lev_dt);
    cudaFree(pl->lev_status);
    cudaFree(pl->lev_partials);
    pl->lev_in = pl->lev_out = nullptr;
    pl->lev_dt = pl->lev_partials = nullptr;
    pl->lev_status = nullptr;
    pl->lev_cap = 0;
    bool ok = cudaMalloc(&pl->lev_in, level_bytes) == cudaSuccess &&
              cudaMalloc(&pl->lev_out, level_bytes) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&pl->lev_dt), size_t(G) * 16) == cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&pl->lev_status), size_t(G) * 4) ==
                  cudaSuccess &&
              cudaMalloc(reinterpret_cast<void**>(&pl->lev_partials), size_t(G) * 48) ==
                  cudaSuccess;
    for (auto& ev : pl->lev_ev)
        ok = ok && (ev || cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    pl->lev_cap = size_t(G);
    return true;
}

// Level step from the device copy: slab s (layers z0 .. z0+nz-1) is copied in
// on the h2d stream; its kernel, on the compute stream, waits for its own
// copy and the next slab's (the layer above) and for the periodic wrap layer,
// which goes first; its results go back on the d2h stream.  Every layer
// crosses the link once (plus the wrap layer).
int level_step_resident(gamer_pipeline* pl, const char* hin, char* hout, int32_t gx, int32_t gy,
                        int32_t gz, int32_t bc, int32_t L, uint32_t* status_host,
                        double* partials_host, const gh_params* p) {
    using namespace gamer;
    const size_t e = pl->esz;
    const int64_t layer = int64_t(gx) * gy;
    const int64_t G = layer * gz;
    const size_t layer_bytes = size_t(layer) * 20480 * e;
    char* din = static_cast<char*>(pl->lev_in);
    char* dout = static_cast<char*>(pl->lev_out);
    // dt, dh of every group: one copy of the pinned staging (filled by the caller)
    if (cudaMemcpyAsync(pl->lev_dt, pl->stage_dt, size_t(G) * 8, cudaMemcpyHostToDevice,
                        pl->s_h2d) != cudaSuccess ||
        cudaMemcpyAsync(pl->lev_dt + G, pl->stage_dt + G, size_t(G) * 8,
                        cudaMemcpyHostToDevice, pl->s_h2d) != cudaSuccess)
        return GAMER_E_CUDA;
    pl->h2d_bytes += 16 * G;
    const int32_t nslab = (gz + L - 1) / L;
    // the periodic wrap layer below slab 0 first
    if (bc == 0 && nslab > 1) {
        if (cudaMemcpyAsync(din + size_t(gz - 1) * layer_bytes, hin + size_t(gz - 1) * layer_bytes,
                            layer_bytes, cudaMemcpyHostToDevice, pl->s_h2d) != cudaSuccess)
            return GAMER_E_CUDA;
        pl->h2d_bytes += int64_t(layer_bytes);
    }
    auto copy_in = [&](int32_t s) -> bool {
        const int32_t z0 = s * L, nz = std::min<int32_t>(L, gz - z0);
        size_t off = size_t(z0) * layer_bytes, bytes = size_t(nz) * layer_bytes;
        if (bc == 0 && nslab > 1 && s == nslab - 1) bytes -= layer_bytes;  // wrap layer: sent
        pl->h2d_bytes += int64_t(bytes);
        return (bytes == 0 || cudaMemcpyAsync(din + off, hin + off, bytes, cudaMemcpyHostToDevice,
                                              pl->s_h2d) == cudaSuccess) &&
               cudaEventRecord(pl->lev_ev[s % 3], pl->s_h2d) == cudaSuccess;
    };
    if (!copy_in(0)) return GAMER_E_CUDA;
    int rc = GAMER_OK;
    for (int32_t s = 0; s < nslab; ++s) {
        // the kernel of slab s reads the first layer of slab s + 1
        if (s + 1 < nslab && !copy_in(s + 1)) return GAMER_E_CUDA;
        const cudaEvent_t need = pl->lev_ev[(s + 1 < nslab ? s + 1 : s) % 3];
        if (cudaStreamWaitEvent(pl->s_comp, need, 0) != cudaSuccess) return GAMER_E_CUDA;
        const int32_t z0 = s * L, nz = std::min<int32_t>(L, gz - z0);
        const int64_t g0 = int64_t(z0) * layer, n = int64_t(nz) * layer;
        char* o = dout + size_t(g0) * 20480 * e;
        if (pl->mode == GAMER_MODE_F32)
            rc = gamer_hydro_advance_level_window_f32(
                (const float*)din, (float*)o, nullptr, gx, gy, gz, bc, 0, gz, z0, nz,
                pl->lev_dt + g0, pl->lev_dt + G + g0, pl->lev_status + g0,
                pl->lev_partials + g0 * 6, p, pl->s_comp);
        else if (pl->mode == GAMER_MODE_MIXED)
            rc = gamer_hydro_advance_level_window_mixed(
                (const float*)din, (float*)o, nullptr, gx, gy, gz, bc, 0, gz, z0, nz,
                pl->lev_dt + g0, pl->lev_dt + G + g0, pl->lev_status + g0,
                pl->lev_partials + g0 * 6, p, pl->s_comp);
        else if (pl->mode == GAMER_MODE_FF)
            rc = gamer_hydro_advance_level_window_ff(
                (const float*)din, (float*)o, nullptr, gx, gy, gz, bc, 0, gz, z0, nz,
                pl->lev_dt + g0, pl->lev_dt + G + g0, pl->lev_status + g0,
                pl->lev_partials + g0 * 6, p, pl->s_comp);
        else
            rc = gamer_hydro_advance_level_window_f64(
                (const double*)din, (double*)o, nullptr, gx, gy, gz, bc, 0, gz, z0, nz,
                pl->lev_dt + g0, pl->lev_dt + G + g0, pl->lev_status + g0,
                pl->lev_partials + g0 * 6, p, pl->s_comp);
        if (rc != GAMER_OK) return rc;
        BufSet& S = pl->set[s % kSets];
        bool ok = cudaEventRecord(S.comp_done, pl->s_comp) == cudaSuccess &&
                  cudaStreamWaitEvent(pl->s_d2h, S.comp_done, 0) == cudaSuccess &&
                  cudaMemcpyAsync(hout + size_t(g0) * 20480 * e, o, size_t(n) * 20480 * e,
                                  cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        pl->d2h_bytes += n * 20480 * int64_t(e);
        if (ok && status_host) {
            ok = cudaMemcpyAsync(status_host + g0, pl->lev_status + g0, size_t(n) * 4,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
            pl->d2h_bytes += 4 * n;
        }
        if (ok && partials_host) {
            ok = cudaMemcpyAsync(partials_host + g0 * 6, pl->lev_partials + g0 * 6,
                                 size_t(n) * 48, cudaMemcpyDeviceToHost, pl->s_d2h) ==
                 cudaSuccess;
            pl->d2h_bytes += 48 * n;
        }
        ok = ok && cudaEventRecord(S.d2h_done, pl->s_d2h) == cudaSuccess;
        if (!ok) return GAMER_E_CUDA;
        S.used = true;
    }
    return wait_event(pl, pl->set[(nslab - 1) % kSets].d2h_done, pl->timeout_s);
}

}  // namespace

// A host-resident level in z-slabs of L layers (L*gx*gy ~ the batch size):
// each slab's window -- its layers plus the layer below and above (periodic
// wrap or zero-gradient clamp) -- goes to the device in at most two copies,
// the window kernel advances the slab with the ghost zones gathered on the
// device, and the slab's results come back; three slabs are in flight.
extern "C" int gamer_pipeline_level_step_host(gamer_pipeline* pl, const void* level_in_host,
                                              void* level_out_host, int32_t gx, int32_t gy,
                                              int32_t gz, int32_t bc, double dt, double dh,
                                              uint32_t* status_host, double* partials_host,
                                              const gh_params* p, int32_t /*nthreads*/) {
    using namespace gamer;
    if (!pl) return GAMER_E_NULL;
    if (const int st = unstick(pl); st != GAMER_OK) return st;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    if (gx < 0 || gy < 0 || gz < 0 || (bc != 0 && bc != 1)) return GAMER_E_PARAM;
    pl->h2d_bytes = pl->d2h_bytes = 0;
    const int64_t layer = int64_t(gx) * gy;
    const int64_t G = layer * gz;
    if (G == 0) return GAMER_OK;
    if (!level_in_host || !level_out_host) return GAMER_E_NULL;
    if (level_in_host == level_out_host) return GAMER_E_OVERLAP;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != pl->device) return GAMER_E_DEVICE;
    const size_t e = pl->esz;
    const size_t layer_bytes = size_t(layer) * 20480 * e;
    const int32_t L = int32_t(std::max<int64_t>(1, std::min<int64_t>(pl->batch / layer, gz)));
    const int32_t zn_max = std::min<int32_t>(L + 2, gz);
    const size_t n_max = size_t(L) * size_t(layer);
    const bool resident = level_resident(pl, G, layer_bytes * size_t(gz));
    // pinned dt, dh staging: [2][cnt], cnt = the groups of one copy
    const size_t cnt = resident ? size_t(G) : n_max;
    if (pl->stage_n < cnt) {
        if (pl->stage_dt) cudaFreeHost(pl->stage_dt);
        pl->stage_dt = nullptr;
        pl->stage_n = 0;
        if (cudaHostAlloc(reinterpret_cast<void**>(&pl->stage_dt), cnt * 16,
                          cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return GAMER_E_CUDA;
        }
        pl->stage_n = cnt;
    }
    // every group of the level takes the same dt and dh
    for (size_t i = 0; i < cnt; ++i) {
        pl->stage_dt[i] = dt;
        pl->stage_dt[cnt + i] = dh;
    }
    const char* hin = static_cast<const char*>(level_in_host);
    char* hout = static_cast<char*>(level_out_host);
    const int32_t nslab = (gz + L - 1) / L;
    if (resident)
        return level_step_resident(pl, hin, hout, gx, gy, gz, bc, L, status_host,
                                   partials_host, p);
    for (int32_t sl = 0; sl < nslab; ++sl) {
        BufSet& S = pl->set[sl % kSets];
        const int32_t z0 = sl * L, nz = std::min<int32_t>(L, gz - z0);
        const int64_t n = int64_t(nz) * layer;
        int32_t zb, zn;
        if (bc == 0) {
            zn = std::min<int32_t>(nz + 2, gz);
            zb = (zn == gz) ? 0 : (z0 - 1 + gz) % gz;
        } else {
            const int32_t lo = std::max<int32_t>(z0 - 1, 0), hi = std::min<int32_t>(z0 + nz, gz - 1);
            zb = lo;
            zn = hi - lo + 1;
        }
        // the set's buffers are reused only once its previous results have left
        if (S.used && (rc = wait_event(pl, S.d2h_done, pl->timeout_s)) != GAMER_OK) return rc;
        if (!ensure_window(S, size_t(zn_max) * layer_bytes, n_max, e)) {
            cudaGetLastError();
            return GAMER_E_CUDA;
        }
        // window layers zb .. zb+zn-1 (mod gz): one copy, or two across the wrap
        const int32_t first = std::min<int32_t>(zn, gz - zb);
        bool ok = cudaMemcpyAsync(S.win, hin + size_t(zb) * layer_bytes, size_t(first) * layer_bytes,
                                  cudaMemcpyHostToDevice, pl->s_h2d) == cudaSuccess;
        if (ok && first < zn)
            ok = cudaMemcpyAsync(static_cast<char*>(S.win) + size_t(first) * layer_bytes, hin,
                                 size_t(zn - first) * layer_bytes, cudaMemcpyHostToDevice,
                                 pl->s_h2d) == cudaSuccess;
        ok = ok &&
             cudaMemcpyAsync(S.wdt, pl->stage_dt, size_t(n) * 8, cudaMemcpyHostToDevice,
                             pl->s_h2d) == cudaSuccess &&
             cudaMemcpyAsync(S.wdt + n, pl->stage_dt + n_max, size_t(n) * 8,
                             cudaMemcpyHostToDevice, pl->s_h2d) == cudaSuccess &&
             cudaEventRecord(S.h2d_done, pl->s_h2d) == cudaSuccess &&
             cudaStreamWaitEvent(pl->s_comp, S.h2d_done, 0) == cudaSuccess;
        if (!ok) return GAMER_E_CUDA;
        pl->h2d_bytes += int64_t(zn) * int64_t(layer_bytes) + 16 * n;
        if (pl->mode == GAMER_MODE_F32)
            rc = gamer_hydro_advance_level_window_f32(
                (const float*)S.win, (float*)S.wout, nullptr, gx, gy, gz, bc, zb, zn, z0, nz,
                S.wdt, S.wdt + n, S.wstatus, S.wpartials, p, pl->s_comp);
        else if (pl->mode == GAMER_MODE_MIXED)
            rc = gamer_hydro_advance_level_window_mixed(
                (const float*)S.win, (float*)S.wout, nullptr, gx, gy, gz, bc, zb, zn, z0, nz,
                S.wdt, S.wdt + n, S.wstatus, S.wpartials, p, pl->s_comp);
        else if (pl->mode == GAMER_MODE_FF)
            rc = gamer_hydro_advance_level_window_ff(
                (const float*)S.win, (float*)S.wout, nullptr, gx, gy, gz, bc, zb, zn, z0, nz,
                S.wdt, S.wdt + n, S.wstatus, S.wpartials, p, pl->s_comp);
        else
            rc = gamer_hydro_advance_level_window_f64(
                (const double*)S.win, (double*)S.wout, nullptr, gx, gy, gz, bc, zb, zn, z0, nz,
                S.wdt, S.wdt + n, S.wstatus, S.wpartials, p, pl->s_comp);
        if (rc != GAMER_OK) return rc;
        const int64_t g0 = int64_t(z0) * layer;
        ok = cudaEventRecord(S.comp_done, pl->s_comp) == cudaSuccess &&
             cudaStreamWaitEvent(pl->s_d2h, S.comp_done, 0) == cudaSuccess &&
             cudaMemcpyAsync(hout + size_t(g0) * 20480 * e, S.wout, size_t(n) * 20480 * e,
                             cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
        pl->d2h_bytes += n * 20480 * int64_t(e);
        if (ok && status_host) {
            ok = cudaMemcpyAsync(status_host + g0, S.wstatus, size_t(n) * 4,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
            pl->d2h_bytes += 4 * n;
        }
        if (ok && partials_host) {
            ok = cudaMemcpyAsync(partials_host + g0 * 6, S.wpartials, size_t(n) * 48,
                                 cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess;
            pl->d2h_bytes += 48 * n;
        }
        ok = ok && cudaEventRecord(S.d2h_done, pl->s_d2h) == cudaSuccess;
        if (!ok) return GAMER_E_CUDA;
        S.used = true;
    }
    return wait_event(pl, pl->set[(nslab - 1) % kSets].d2h_done, pl->timeout_s);
}

namespace {

__global__ void status_or_kernel(uint32_t* __restrict__ acc, const uint32_t* __restrict__ st,
                                 int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x)
        acc[i] |= st[i];
}

// Device buffers and events of a run over G groups (level_bytes per level),
// nslab slabs and nsteps steps; grown when a run needs more.
bool ensure_run(gamer_pipeline* pl, int64_t G, size_t level_bytes, int32_t nslab,
                int32_t nsteps) {
    if (pl->run_cap < size_t(G) || pl->run_level_bytes < level_bytes) {
        release_run(pl);
        bool ok = true;
        for (int i = 0; i < 2 && ok; ++i)
            ok = cudaMalloc(&pl->run_in[i], level_bytes) == cudaSuccess &&
                 cudaMalloc(&pl->run_out[i], level_bytes) == cudaSuccess;
        const size_t ws = gamer_hydro_dt_workspace_bytes(G, 1);
        ok = ok &&
             cudaMalloc(reinterpret_cast<void**>(&pl->run_dt), size_t(G) * 16) == cudaSuccess &&
             cudaMalloc(reinterpret_cast<void**>(&pl->run_status), size_t(G) * 8) ==
                 cudaSuccess &&
             cudaMalloc(reinterpret_cast<void**>(&pl->run_partials), size_t(G) * 48) ==
                 cudaSuccess &&
             ws > 0 && cudaMalloc(&pl->run_ws, ws) == cudaSuccess;
        for (auto& ev : pl->run_comp)
            ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&pl->run_end, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            release_run(pl);
            return false;
        }
        pl->run_ws_bytes = ws;
        pl->run_cap = size_t(G);
        pl->run_level_bytes = level_bytes;
    }
    if (pl->run_aux_cap < size_t(nsteps) + 1) {
        cudaFree(pl->run_aux);
        pl->run_aux = nullptr;
        pl->run_aux_cap = 0;
        if (cudaMalloc(reinterpret_cast<void**>(&pl->run_aux), (size_t(nsteps) + 1) * 8) !=
            cudaSuccess)
            return false;
        pl->run_aux_cap = size_t(nsteps) + 1;
    }
    if (pl->run_ev_slabs < nslab) {
        if (pl->run_ev) {
            for (int32_t i = 0; i < 4 * pl->run_ev_slabs; ++i)
                if (pl->run_ev[i]) cudaEventDestroy(pl->run_ev[i]);
            delete[] pl->run_ev;
        }
        pl->run_ev_slabs = 0;
        pl->run_ev = new (std::nothrow) cudaEvent_t[4 * size_t(nslab)]();
        if (!pl->run_ev) return false;
        for (int32_t i = 0; i < 4 * nslab; ++i)
            if (cudaEventCreateWithFlags(&pl->run_ev[i], cudaEventDisableTiming) != cudaSuccess)
                return false;
        pl->run_ev_slabs = nslab;
    }
    return true;
}

int advance_window(const gamer_pipeline* pl, const void* din, void* out, int32_t gx, int32_t gy,
                   int32_t gz, int32_t bc, int32_t z0, int32_t nz, const double* dt,
                   const double* dh, uint32_t* status, double* partials, const gh_params* p) {
    if (pl->mode == GAMER_MODE_F32)
        return gamer_hydro_advance_level_window_f32((const float*)din, (float*)out, nullptr, gx,
                                                    gy, gz, bc, 0, gz, z0, nz, dt, dh, status,
                                                    partials, p, pl->s_comp);
    if (pl->mode == GAMER_MODE_MIXED)
        return gamer_hydro_advance_level_window_mixed((const float*)din, (float*)out, nullptr,
                                                      gx, gy, gz, bc, 0, gz, z0, nz, dt, dh,
                                                      status, partials, p, pl->s_comp);
    if (pl->mode == GAMER_MODE_FF)
        return gamer_hydro_advance_level_window_ff((const float*)din, (float*)out, nullptr, gx,
                                                   gy, gz, bc, 0, gz, z0, nz, dt, dh, status,
                                                   partials, p, pl->s_comp);
    return gamer_hydro_advance_level_window_f64((const double*)din, (double*)out, nullptr, gx, gy,
                                                gz, bc, 0, gz, z0, nz, dt, dh, status, partials,
                                                p, pl->s_comp);
}

}  // namespace

// nsteps steps of a host level between two host buffers.  Step n's slabs go
// in the order n, n+1, ... (mod the slab count), so that its first slabs read
// what step n-1 sent back first; copies in of step n wait only for step
// n-1's copies out of the same slabs, and both link directions stay busy
// across steps.  The dt of step n >= 1 is reduced on the device from step
// n-1's partials (gamer_hydro_dt), on the compute stream.
extern "C" int gamer_pipeline_level_run_host(gamer_pipeline* pl, void* level0, void* level1,
                                             int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                             int32_t nsteps, double dt0, double dh, double cfl,
                                             double* dt_host, uint32_t* status_host,
                                             double* partials_host, const gh_params* p) {
    using namespace gamer;
    if (!pl) return GAMER_E_NULL;
    if (const int st = unstick(pl); st != GAMER_OK) return st;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    if (gx < 0 || gy < 0 || gz < 0 || (bc != 0 && bc != 1) || nsteps < 0) return GAMER_E_PARAM;
    if (!(std::isfinite(dt0) && dt0 >= 0.0) || !(std::isfinite(dh) && dh > 0.0) ||
        !(std::isfinite(cfl) && cfl > 0.0))
        return GAMER_E_PARAM;
    if (int64_t(gx) * 16 > (1 << 30) || int64_t(gy) * 16 > (1 << 30) ||
        int64_t(gz) * 16 > (1 << 30) || int64_t(gx) * gy * 1280 + 2048 > INT32_MAX)
        return GAMER_E_PARAM;
    pl->h2d_bytes = pl->d2h_bytes = 0;
    const int64_t layer = int64_t(gx) * gy;
    const int64_t G = layer * gz;
    if (G == 0 || nsteps == 0) return GAMER_OK;
    if (!level0 || !level1) return GAMER_E_NULL;
    const size_t e = pl->esz;
    const size_t layer_bytes = size_t(layer) * 20480 * e;
    const size_t level_bytes = layer_bytes * size_t(gz);
    if (overlaps(level0, level_bytes, level1, level_bytes)) return GAMER_E_OVERLAP;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != pl->device) return GAMER_E_DEVICE;
    const int32_t L = int32_t(std::max<int64_t>(1, std::min<int64_t>(pl->batch / layer, gz)));
    const int32_t nslab = (gz + L - 1) / L;
    if (!ensure_run(pl, G, level_bytes, nslab, nsteps)) {
        cudaGetLastError();
        return GAMER_E_CUDA;
    }
    // dt0 and dh of every group through the pinned staging
    if (pl->stage_n < size_t(G)) {
        if (pl->stage_dt) cudaFreeHost(pl->stage_dt);
        pl->stage_dt = nullptr;
        pl->stage_n = 0;
        if (cudaHostAlloc(reinterpret_cast<void**>(&pl->stage_dt), size_t(G) * 16,
                          cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return GAMER_E_CUDA;
        }
        pl->stage_n = size_t(G);
    }
    const size_t cnt = pl->stage_n;
    for (int64_t i = 0; i < G; ++i) {
        pl->stage_dt[i] = dt0;
        pl->stage_dt[cnt + i] = dh;
    }
    // the previous call's copies out of the staging are complete (it returned
    // after its last copy), so the staging may be rewritten here
    bool ok = cudaMemcpyAsync(pl->run_dt, pl->stage_dt, size_t(G) * 8, cudaMemcpyHostToDevice,
                              pl->s_h2d) == cudaSuccess &&
              cudaMemcpyAsync(pl->run_dt + G, pl->stage_dt + cnt, size_t(G) * 8,
                              cudaMemcpyHostToDevice, pl->s_h2d) == cudaSuccess &&
              cudaMemcpyAsync(pl->run_aux, pl->stage_dt + cnt, 8, cudaMemcpyHostToDevice,
                              pl->s_h2d) == cudaSuccess &&
              cudaMemcpyAsync(pl->run_aux + 1, pl->stage_dt, 8, cudaMemcpyHostToDevice,
                              pl->s_h2d) == cudaSuccess &&
              cudaMemsetAsync(pl->run_status + G, 0, size_t(G) * 4, pl->s_comp) == cudaSuccess;
    if (!ok) return GAMER_E_CUDA;
    pl->h2d_bytes += 16 * G + 16;
    char* hbuf[2] = {static_cast<char*>(level0), static_cast<char*>(level1)};
    const DeviceInfo d = current_device();
    const unsigned or_blocks =
        unsigned(std::min<int64_t>((G + 255) / 256, int64_t(d.sm_count > 0 ? d.sm_count : 1) * 8));
    for (int32_t n = 0; n < nsteps; ++n) {
        const int par = n & 1;
        const char* hin = hbuf[par];
        char* hout = hbuf[par ^ 1];
        char* din = static_cast<char*>(pl->run_in[par]);
        char* dout = static_cast<char*>(pl->run_out[par]);
        cudaEvent_t* ev_in = pl->run_ev + size_t(par * 2 + 0) * pl->run_ev_slabs;
        cudaEvent_t* ev_out = pl->run_ev + size_t(par * 2 + 1) * pl->run_ev_slabs;
        cudaEvent_t* prev_out = pl->run_ev + size_t((par ^ 1) * 2 + 1) * pl->run_ev_slabs;
        const int32_t r = n % nslab;  // first slab of this step
        // copies in.  This parity's device input was last read by step n-2's
        // kernels; the host input of a slab is step n-1's output of it.
        if (n >= 2 && cudaStreamWaitEvent(pl->s_h2d, pl->run_comp[par], 0) != cudaSuccess)
            return GAMER_E_CUDA;
        // the layer below slab r first (periodic wrap, or r > 0): it is the
        // top layer of the last slab in this step's order, r - 1
        const bool below = nslab > 1 && (bc == 0 || r > 0);
        const int32_t sbelow = (r + nslab - 1) % nslab;
        if (below) {
            const size_t off = size_t((int64_t(r) * L + gz - 1) % gz) * layer_bytes;
            ok = (n == 0 || cudaStreamWaitEvent(pl->s_h2d, prev_out[sbelow], 0) == cudaSuccess) &&
                 cudaMemcpyAsync(din + off, hin + off, layer_bytes, cudaMemcpyHostToDevice,
                                 pl->s_h2d) == cudaSuccess;
            if (!ok) return GAMER_E_CUDA;
            pl->h2d_bytes += int64_t(layer_bytes);
        }
        for (int32_t i = 0; i < nslab; ++i) {
            const int32_t s = (r + i) % nslab;
            const int32_t z0 = s * L, nz = std::min<int32_t>(L, gz - z0);
            const int32_t cz = (below && s == sbelow) ? nz - 1 : nz;
            const size_t off = size_t(z0) * layer_bytes, bytes = size_t(cz) * layer_bytes;
            ok = (n == 0 || cudaStreamWaitEvent(pl->s_h2d, prev_out[s], 0) == cudaSuccess) &&
                 (bytes == 0 || cudaMemcpyAsync(din + off, hin + off, bytes,
                                                cudaMemcpyHostToDevice, pl->s_h2d) ==
                                    cudaSuccess) &&
                 cudaEventRecord(ev_in[i], pl->s_h2d) == cudaSuccess;
            if (!ok) return GAMER_E_CUDA;
            pl->h2d_bytes += int64_t(bytes);
        }
        // this step's dt: dt0, or reduced from step n-1's partials
        if (n >= 1) {
            rc = gamer_hydro_dt(pl->run_partials, G, nullptr, 1, pl->run_aux, cfl,
                                pl->run_aux + 1 + n, nullptr, pl->run_dt, pl->run_ws,
                                pl->run_ws_bytes, pl->s_comp);
            if (rc != GAMER_OK) return rc;
        }
        for (int32_t i = 0; i < nslab; ++i) {
            const int32_t s = (r + i) % nslab;
            const int32_t z0 = s * L, nz = std::min<int32_t>(L, gz - z0);
            const int64_t g0 = int64_t(z0) * layer, ng = int64_t(nz) * layer;
            // its layers and the layer above are in copies 0 .. i+1; its
            // output slot was last read by step n-2's copy out
            ok = cudaStreamWaitEvent(pl->s_comp, ev_in[std::min(i + 1, nslab - 1)], 0) ==
                     cudaSuccess &&
                 (n < 2 || cudaStreamWaitEvent(pl->s_comp, ev_out[s], 0) == cudaSuccess);
            if (!ok) return GAMER_E_CUDA;
            rc = advance_window(pl, din, dout + size_t(g0) * 20480 * e, gx, gy, gz, bc, z0, nz,
                                pl->run_dt + g0, pl->run_dt + G + g0, pl->run_status + g0,
                                pl->run_partials + g0 * 6, p);
            if (rc != GAMER_OK) return rc;
            // the slab's kernel -> its copy out (only the set's event is used)
            const cudaEvent_t done = pl->set[i % kSets].comp_done;
            ok = cudaEventRecord(done, pl->s_comp) == cudaSuccess &&
                 cudaStreamWaitEvent(pl->s_d2h, done, 0) == cudaSuccess &&
                 cudaMemcpyAsync(hout + size_t(z0) * layer_bytes, dout + size_t(z0) * layer_bytes,
                                 size_t(nz) * layer_bytes, cudaMemcpyDeviceToHost,
                                 pl->s_d2h) == cudaSuccess &&
                 cudaEventRecord(ev_out[s], pl->s_d2h) == cudaSuccess;
            if (!ok) return GAMER_E_CUDA;
            pl->d2h_bytes += ng * 20480 * int64_t(e);
        }
        status_or_kernel<<<or_blocks, 256, 0, pl->s_comp>>>(pl->run_status + G, pl->run_status,
                                                           G);
        if (cudaGetLastError() != cudaSuccess ||
            cudaEventRecord(pl->run_comp[par], pl->s_comp) != cudaSuccess)
            return GAMER_E_CUDA;
    }
    // the run's dt sequence, status bits OR-ed over the steps, last partials
    ok = cudaStreamWaitEvent(pl->s_d2h, pl->run_comp[(nsteps - 1) & 1], 0) == cudaSuccess &&
         (!dt_host || cudaMemcpyAsync(dt_host, pl->run_aux + 1, size_t(nsteps) * 8,
                                      cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess) &&
         (!status_host || cudaMemcpyAsync(status_host, pl->run_status + G, size_t(G) * 4,
                                          cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess) &&
         (!partials_host || cudaMemcpyAsync(partials_host, pl->run_partials, size_t(G) * 48,
                                            cudaMemcpyDeviceToHost, pl->s_d2h) == cudaSuccess) &&
         cudaEventRecord(pl->run_end, pl->s_d2h) == cudaSuccess;
    if (!ok) return GAMER_E_CUDA;
    pl->d2h_bytes += (dt_host ? 8 * int64_t(nsteps) : 0) + (status_host ? 4 * G : 0) +
                     (partials_host ? 48 * G : 0);
    return wait_event(pl, pl->run_end, pl->timeout_s * nsteps);
}

extern "C" int gamer_pipeline_last_bytes(const gamer_pipeline* pl, int64_t* h2d, int64_t* d2h) {
    if (!pl || !h2d || !d2h) return GAMER_E_NULL;
    *h2d = pl->h2d_bytes;
    *d2h = pl->d2h_bytes;
    return GAMER_OK;
}

extern "C" int gamer_pipeline_debug_hold(gamer_pipeline* pl, double seconds) {
    if (!pl) return GAMER_E_NULL;
    if (!(std::isfinite(seconds) && seconds >= 0.0 && seconds <= 60.0)) return GAMER_E_PARAM;
    double* arg = new (std::nothrow) double(seconds);
    if (!arg) return GAMER_E_CUDA;
    cudaEvent_t ev = pl->set[0].h2d_done;  // reused: no call is in flight here
    if (cudaLaunchHostFunc(pl->s_h2d, sleep_host, arg) != cudaSuccess) {
        delete arg;
        cudaGetLastError();
        return GAMER_E_CUDA;
    }
    if (cudaEventRecord(ev, pl->s_h2d) != cudaSuccess ||
        cudaStreamWaitEvent(pl->s_comp, ev, 0) != cudaSuccess ||
        cudaStreamWaitEvent(pl->s_d2h, ev, 0) != cudaSuccess) {
        cudaGetLastError();
        return GAMER_E_CUDA;
    }
    return GAMER_OK;
}

extern "C" int gamer_pipeline_set_timeout(gamer_pipeline* pl, double seconds) {
    if (!pl) return GAMER_E_NULL;
    if (!(seconds > 0.0)) return GAMER_E_PARAM;
    pl->timeout_s = seconds;
    return GAMER_OK;
}

extern "C" int gamer_pipeline_set_level_mode(gamer_pipeline* pl, int32_t mode) {
    if (!pl) return GAMER_E_NULL;
    if (mode < 0 || mode > 2) return GAMER_E_PARAM;
    pl->level_mode = mode;
    if (mode == 2) {  // give the device copy back
        cudaFree(pl->lev_in);
        cudaFree(pl->lev_out);
        cudaFree(pl->lev_dt);
        cudaFree(pl->lev_status);
        cudaFree(pl->lev_partials);
        pl->lev_in = pl->lev_out = nullptr;
        pl->lev_dt = pl->lev_partials = nullptr;
        pl->lev_status = nullptr;
        pl->lev_cap = 0;
    }
    return GAMER_OK;
}
