// level_graph.cu -- one CUDA graph for the device-resident step of a uniform
// level: ghost fill -> MUSCL-Hancock/Roe step -> dt / conservation reduction
// (whose per-group dt feeds the next step); without a tiles buffer the ghost
// fill is fused into the step kernel.  A graph advances level_a into
// level_b; the caller alternates it with the graph of the swapped buffers, so
// a run of steps needs no host involvement and no per-kernel launch overhead.
#include <cuda_runtime.h>

#include <new>

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

struct gamer_level_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int enqueue_step(int mode, const void* cur, void* nxt, void* tiles, void* ff, double* dt_group,
                 const double* dh_group, uint32_t* status, double* partials, int gx, int gy,
                 int gz, int bc, const gh_params* p, const double* dh_level, double* dt_level,
                 double* totals, void* ws, size_t ws_bytes, cudaStream_t s) {
    const int64_t G = int64_t(gx) * gy * gz;
    int rc;
    if (!tiles) {  // fused ghost gather: one kernel reads the level directly
        if (mode == GAMER_MODE_F32)
            rc = gamer_hydro_advance_level_f32((const float*)cur, (float*)nxt, (float*)ff, gx, gy,
                                               gz, bc, dt_group, dh_group, status, partials, p, s);
        else if (mode == GAMER_MODE_MIXED)
            rc = gamer_hydro_advance_level_mixed((const float*)cur, (float*)nxt, (float*)ff, gx,
                                                 gy, gz, bc, dt_group, dh_group, status, partials,
                                                 p, s);
        else if (mode == GAMER_MODE_FF)
            rc = gamer_hydro_advance_level_ff((const float*)cur, (float*)nxt, (float*)ff, gx, gy,
                                              gz, bc, dt_group, dh_group, status, partials, p, s);
        else
            rc = gamer_hydro_advance_level_f64((const double*)cur, (double*)nxt, (double*)ff, gx,
                                               gy, gz, bc, dt_group, dh_group, status, partials,
                                               p, s);
        if (rc != GAMER_OK) return rc;
        return gamer_hydro_dt(partials, G, nullptr, 1, dh_level, p->cfl, dt_level, totals,
                              dt_group, ws, ws_bytes, s);
    }
    if (mode == GAMER_MODE_F64)
        rc = gamer_fill_ghosts_uniform_f64((const double*)cur, (double*)tiles, gx, gy, gz, bc, s);
    else
        rc = gamer_fill_ghosts_uniform_f32((const float*)cur, (float*)tiles, gx, gy, gz, bc, s);
    if (rc != GAMER_OK) return rc;
    if (mode == GAMER_MODE_F32)
        rc = gamer_hydro_advance_f32((const float*)tiles, (float*)nxt, (float*)ff, dt_group,
                                     dh_group, status, partials, G, p, s);
    else if (mode == GAMER_MODE_MIXED)
        rc = gamer_hydro_advance_mixed((const float*)tiles, (float*)nxt, (float*)ff, dt_group,
                                       dh_group, status, partials, G, p, s);
    else if (mode == GAMER_MODE_FF)
        rc = gamer_hydro_advance_ff((const float*)tiles, (float*)nxt, (float*)ff, dt_group,
                                    dh_group, status, partials, G, p, s);
    else
        rc = gamer_hydro_advance_f64((const double*)tiles, (double*)nxt, (double*)ff, dt_group,
                                     dh_group, status, partials, G, p, s);
    if (rc != GAMER_OK) return rc;
    return gamer_hydro_dt(partials, G, nullptr, 1, dh_level, p->cfl, dt_level, totals, dt_group,
                          ws, ws_bytes, s);
}

}  // namespace

extern "C" int gamer_level_graph_create(int32_t mode, void* level_a, void* level_b, void* tiles,
                                        void* face_flux, double* dt_group,
                                        const double* dh_group, uint32_t* status,
                                        double* partials, int32_t gx, int32_t gy, int32_t gz,
                                        int32_t bc, const gh_params* p, const double* dh_level,
                                        double* dt_level, double* totals, void* workspace,
                                        size_t workspace_bytes, gamer_level_graph** out) {
    using namespace gamer;
    if (!out) return GAMER_E_NULL;
    *out = nullptr;
    if (mode < 0 || mode > 3 || gx < 1 || gy < 1 || gz < 1) return GAMER_E_PARAM;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    if (!(std::isfinite(p->cfl) && p->cfl > 0.0)) return GAMER_E_PARAM;
    if (!level_a || !level_b || !dt_group || !dh_group || !partials || !dh_level || !dt_level)
        return GAMER_E_NULL;
    const DeviceInfo d = current_device();
    if (d.status != GAMER_OK) return d.status;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GAMER_E_CUDA;
    gamer_level_graph* h = new (std::nothrow) gamer_level_graph();
    if (!h) {
        cudaStreamDestroy(s);
        return GAMER_E_CUDA;
    }
    rc = GAMER_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = GAMER_E_CUDA;
    } else {
        rc = enqueue_step(mode, level_a, level_b, tiles, face_flux, dt_group, dh_group, status,
                          partials, gx, gy, gz, bc, p, dh_level, dt_level, totals, workspace,
                          workspace_bytes, s);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rc == GAMER_OK && e != cudaSuccess) rc = GAMER_E_CUDA;
        h->graph = g;
        if (rc == GAMER_OK && cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess)
            rc = GAMER_E_CUDA;
    }
    cudaStreamDestroy(s);
    if (rc != GAMER_OK) {
        if (h->exec) cudaGraphExecDestroy(h->exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        delete h;
        cudaGetLastError();
        return rc;
    }
    *out = h;
    return GAMER_OK;
}

namespace {

// One step of an uneven AMR batch: dt per level from the partials of the
// previous step, scattered to the groups, then the persistent step of all N
// groups (whose partials feed the next step).
int enqueue_batch_step(int mode, const void* in, void* out, void* ff, double* dt_group,
                       const double* dh_group, const int32_t* level, int32_t n_levels,
                       uint32_t* status, double* partials, int64_t N, const gh_params* p,
                       const double* dh_level, double* dt_level, double* totals, void* ws,
                       size_t ws_bytes, cudaStream_t s) {
    int rc = gamer_hydro_dt(partials, N, level, n_levels, dh_level, p->cfl, dt_level, totals,
                            dt_group, ws, ws_bytes, s);
    if (rc != GAMER_OK) return rc;
    if (mode == GAMER_MODE_F32)
        return gamer_hydro_advance_f32((const float*)in, (float*)out, (float*)ff, dt_group,
                                       dh_group, status, partials, N, p, s);
    if (mode == GAMER_MODE_MIXED)
        return gamer_hydro_advance_mixed((const float*)in, (float*)out, (float*)ff, dt_group,
                                         dh_group, status, partials, N, p, s);
    if (mode == GAMER_MODE_FF)
        return gamer_hydro_advance_ff((const float*)in, (float*)out, (float*)ff, dt_group,
                                      dh_group, status, partials, N, p, s);
    return gamer_hydro_advance_f64((const double*)in, (double*)out, (double*)ff, dt_group,
                                   dh_group, status, partials, N, p, s);
}

// Captures `enqueue` (a callable taking the capture stream) into a new graph
// handle.
template <class F>
int capture(F enqueue, gamer_level_graph** out) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return GAMER_E_CUDA;
    gamer_level_graph* h = new (std::nothrow) gamer_level_graph();
    if (!h) {
        cudaStreamDestroy(s);
        return GAMER_E_CUDA;
    }
    int rc = GAMER_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = GAMER_E_CUDA;
    } else {
        rc = enqueue(s);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (rc == GAMER_OK && e != cudaSuccess) rc = GAMER_E_CUDA;
        h->graph = g;
        if (rc == GAMER_OK && cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess)
            rc = GAMER_E_CUDA;
    }
    cudaStreamDestroy(s);
    if (rc != GAMER_OK) {
        if (h->exec) cudaGraphExecDestroy(h->exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        delete h;
        cudaGetLastError();
        return rc;
    }
    *out = h;
    return GAMER_OK;
}

}  // namespace

extern "C" int gamer_batch_graph_create(int32_t mode, const void* in, void* out, void* face_flux,
                                        double* dt_group, const double* dh_group,
                                        const int32_t* level, int32_t n_levels, uint32_t* status,
                                        double* partials, int64_t N, const gh_params* p,
                                        const double* dh_level, double* dt_level, double* totals,
                                        void* workspace, size_t workspace_bytes,
                                        gamer_level_graph** out_graph) {
    using namespace gamer;
    if (!out_graph) return GAMER_E_NULL;
    *out_graph = nullptr;
    if (mode < 0 || mode > 3 || N < 1 || n_levels < 1 || n_levels > 64) return GAMER_E_PARAM;
    int rc = check_params(p);
    if (rc != GAMER_OK) return rc;
    if (!(std::isfinite(p->cfl) && p->cfl > 0.0)) return GAMER_E_PARAM;
    if (!in || !out || !dt_group || !dh_group || !partials || !dh_level || !dt_level)
        return GAMER_E_NULL;
    if (workspace_bytes < gamer_hydro_dt_workspace_bytes(N, n_levels) || !workspace)
        return GAMER_E_WORKSPACE;
    const DeviceInfo d = current_device();
    if (d.status != GAMER_OK) return d.status;
    return capture(
        [&](cudaStream_t s) {
            return enqueue_batch_step(mode, in, out, face_flux, dt_group, dh_group, level,
                                      n_levels, status, partials, N, p, dh_level, dt_level,
                                      totals, workspace, workspace_bytes, s);
        },
        out_graph);
}

extern "C" int gamer_level_graph_launch(gamer_level_graph* h, void* stream) {
    if (!h || !h->exec) return GAMER_E_NULL;
    return cudaGraphLaunch(h->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? GAMER_OK
               : GAMER_E_CUDA;
}

extern "C" int gamer_level_graph_destroy(gamer_level_graph* h) {
    if (!h) return GAMER_E_NULL;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    delete h;
    return GAMER_OK;
}
