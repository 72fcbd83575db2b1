/*
 * gamer_gb300.h -- C ABI of the GB300 (sm_103a) MUSCL-Hancock + Roe patch-group
 * hydro step.
 *
 * The operation (paper Sec. 2, "Extension I: hydrodynamic solver"): advance
 * each AMR patch group by one time step with the MUSCL-Hancock method and
 * Roe's Riemann solver -- spatial data reconstruction, half-step prediction,
 * Riemann solver, full-step update -- as an unsplit finite-volume scheme with a
 * five-point stencil per direction.  A patch group is 16^3 cells; with the
 * two-cell ghost shell that stencil needs its input is 20^3 cells.  The ghost
 * data are prepared outside the solver (paper Sec. 2: "the operation of
 * preparing the ghost-zone data"); gamer_fill_ghosts_uniform_* does that on
 * the device for a uniform level.  Groups are independent within a step, so a
 * batch of N groups of uneven AMR levels (each its own dt and dh) is one call.
 *
 * Conventions shared by every entry point:
 *  - Array pointers are caller-owned DEVICE memory unless a function says
 *    otherwise; the library never allocates, frees or synchronises on the
 *    device path.  Work is enqueued on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream) and runs asynchronously.
 *  - Layouts are C-contiguous, x fastest.  Conserved variables are ordered
 *    (rho, rho*vx, rho*vy, rho*vz, E).
 *  - Return codes: 0 success; negative GAMER_E* codes below.  Nothing is
 *    launched when a call returns an error.  Per-group numerical events never
 *    fail a call: they are reported in status[g] (GAMER_ST_* bits).
 *  - N == 0 is a no-op returning 0.
 *  - Device code never traps: bad data produce status bits, not faults.
 */
#ifndef GAMER_GB300_H
#define GAMER_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define GAMER_OK 0
#define GAMER_E_NULL (-1)        /* a required pointer is NULL                        */
#define GAMER_E_PARAM (-2)       /* bad size or parameter (N < 0, gamma <= 1, ...)      */
#define GAMER_E_ALIGN (-3)       /* misaligned pointer                                  */
#define GAMER_E_CUDA (-4)        /* CUDA launch / configuration error                  */
#define GAMER_E_DEVICE (-5)      /* current device is not compute capability 10.x      */
#define GAMER_E_OVERLAP (-6)     /* an output buffer overlaps an input buffer          */
#define GAMER_E_WORKSPACE (-7)   /* workspace missing or too small                     */
#define GAMER_E_TIMEOUT (-8)     /* a bounded host wait gave up (pipeline)             */

/* ---- per-group status bits (status[g]) ---- */
#define GAMER_ST_PREDICTOR_FALLBACK 0x1u /* a cell's half-step states were replaced (first order) */
#define GAMER_ST_HLLE_FALLBACK      0x2u /* a face used HLLE instead of Roe                       */
#define GAMER_ST_NONPOSITIVE_OUT    0x4u /* an updated cell has rho <= 0 or p <= 0 (or NaN)       */
#define GAMER_ST_BAD_INPUT          0x8u /* non-finite read input, or dt < 0 / dh <= 0 / non-finite */
#define GAMER_ST_INTERNAL_TIMEOUT  0x10u /* a bounded on-chip wait gave up; outputs are invalid:
                                            the CTA stops, so this group and every later
                                            group it owned carry the bit, get NaN partials
                                            and keep whatever out / face_flux held        */
#define GAMER_ST_FLOOR             0x20u /* a density or pressure floor changed an updated cell   */

/* ---- precision modes ---- */
#define GAMER_MODE_F32 0   /* FP32 storage and arithmetic                                     */
#define GAMER_MODE_MIXED 1 /* FP32 storage/arithmetic; pressure E - |m|^2/(2 rho) in FP64 where
                              the kinetic energy is more than half of E (high Mach)       */
#define GAMER_MODE_F64 2   /* FP64 storage and arithmetic                                     */
#define GAMER_MODE_FF 3    /* FP32 storage/arithmetic, pressure recovery in float-float        */

/* ---- scheme parameters ---- */
typedef struct gh_params {
    double gamma;               /* ratio of specific heats; finite and > 1                  */
    double cfl;                 /* Courant number; used only by gamer_hydro_dt's callers    */
    int32_t limiter;            /* slope limiter: 0 van Leer (default), 1 minmod, 2 MC      */
    int32_t predictor_fallback; /* 0: cell average (default), 1: un-evolved face states   */
    int32_t flux_layout;        /* face_flux per group: 0 = the six group faces [6][5][16][16]
                                   (default); 1 = nine planes [9][5][16][16], three per
                                   direction at 0, 8 and 16 cells (x: 0,1,2; y: 3,4,5;
                                   z: 6,7,8), which adds the patch boundaries inside the
                                   group for the coarse-fine flux fix-up                   */
    int32_t riemann;            /* Riemann solver: 0 Roe with Harten-Hyman entropy fix and
                                   HLLE fallback (default; the paper's), 1 HLLC (a scheme
                                   variant: exact on isolated contact and shear waves)     */
    double rho_floor;           /* finite, >= 0; 0 = off (default): an updated density below
                                   it is raised to it, momentum kept                         */
    double p_floor;             /* finite, >= 0; 0 = off (default): where the updated density
                                   is positive and the pressure below p_floor, the total
                                   energy becomes |m|^2/(2 rho) + p_floor/(gamma - 1)
                                   (at least 4 eps |m|^2/(2 rho), eps of the storage type) */
    int32_t reconstruction;     /* slopes limited in 0: the primitive variables (default;
                                   the paper's reading), 1: the characteristic variables
                                   of each direction (a scheme variant)                    */
    int32_t reserved;           /* must be 0                                                */
} gh_params;

/*
 * gamer_hydro_advance_{f32,mixed,f64}: one MUSCL-Hancock + Roe step of N
 * independent patch groups (paper Sec. 2: reconstruction, half-step
 * prediction, Riemann solver, full-step update; unsplit; Roe's solver with
 * Harten's entropy fix and an HLLE fallback for negative density or
 * pressure).
 *
 *   in        [N][5][20][20][20] conserved state with the 2-cell ghost shell;
 *             16-byte aligned.  The 8 corner 2x2x2 blocks and the depth-2
 *             edge cells are never read.
 *   out       [N][5][16][16][16] updated interior; element aligned; must not
 *             overlap in.
 *   face_flux [N][6][5][16][16] raw numerical flux F (not multiplied by dt)
 *             through the six group faces, in the order -x, +x, -y, +y, -z, +z;
 *             the two in-face indices are [k][j] for x faces, [k][i] for y
 *             faces, [j][i] for z faces.  With p->flux_layout = 1,
 *             [N][9][5][16][16]: per direction the planes at 0, 8 and 16
 *             cells (the group faces and the patch boundary between them), in
 *             the order x0, x8, x16, y0, y8, y16, z0, z8, z16.  For the AMR
 *             coarse-fine flux fix-up (gamer_flux_fixup_*).  May be NULL.
 *   dt, dh    [N] time step and cell width of each group (FP64).
 *   status    [N] GAMER_ST_* bits, or NULL.
 *   partials  [N][6] FP64: { max over updated cells of max_d |v_d| + c,
 *             sum rho, sum rho vx, sum rho vy, sum rho vz, sum E } of the
 *             updated state, or NULL.  Input of gamer_hydro_dt.
 *   N         number of groups (>= 0).
 *   p         scheme parameters (host pointer).
 *   stream    cudaStream_t.
 * _f32, _mixed and _ff take float arrays, _f64 double arrays.  In _mixed mode
 * FP64 is used only where stability needs it: a recovery of the pressure from
 * the conserved state is done in FP64 where |m|^2/(2 rho) > E/2 (high-Mach
 * cells, where E - rho v^2/2 cancels) and in FP32 elsewhere, with gamma - 1
 * held as a float pair so that it brings no rounding bias (there the result
 * is within a few ulps of the FP64 recovery); a test rho E - |m|^2/2 > 0 is
 * decided in FP32 when the FP32 difference is larger than 2^-20 (|rho E| +
 * |m|^2/2), so certainly of the right sign, and in FP64 otherwise; everything
 * else is FP32 (the group reductions are FP64 in every mode).  _ff
 * does the same recoveries (and the rho E - |m|^2/2 > 0 tests) in float-float
 * FP32 arithmetic: |m|^2 exact by FMA products and TwoSum, 1/rho refined to
 * about 2^-46, E - |m|^2/(2 rho) by TwoSum -- as accurate as the FP64 recovery
 * for FP32 states while |m|^2/(2 rho) < 2^22 p, at FP32 speed (a test whose
 * FP32 sign is certain is decided in FP32, with the same outcome).
 */
int gamer_hydro_advance_f32(const float* in, float* out, float* face_flux, const double* dt,
                            const double* dh, uint32_t* status, double* partials, int64_t N,
                            const gh_params* p, void* stream);
int gamer_hydro_advance_mixed(const float* in, float* out, float* face_flux, const double* dt,
                              const double* dh, uint32_t* status, double* partials, int64_t N,
                              const gh_params* p, void* stream);
int gamer_hydro_advance_ff(const float* in, float* out, float* face_flux, const double* dt,
                              const double* dh, uint32_t* status, double* partials, int64_t N,
                              const gh_params* p, void* stream);
int gamer_hydro_advance_f64(const double* in, double* out, double* face_flux, const double* dt,
                            const double* dh, uint32_t* status, double* partials, int64_t N,
                            const gh_params* p, void* stream);

/*
 * gamer_hydro_advance_level_{f32,mixed,f64}: the same step for every group of
 * a uniform level, with the ghost-zone preparation fused into the solver: each
 * group's 20^3 input is gathered plane by plane from its own 16^3 interior and
 * its neighbours' (periodic or zero-gradient boundaries, as
 * gamer_fill_ghosts_uniform_*), so no 20^3 tiles are written or read.
 *   level     [G][5][16][16][16], G = gx*gy*gz, group id (z*gy + y)*gx + x;
 *             16-byte aligned; must not overlap out (every group reads its
 *             neighbours' interiors).
 *   out, face_flux, dt, dh, status, partials: as gamer_hydro_advance_* with
 *             N = G.
 *   bc        0 periodic, 1 zero-gradient.
 * Returns GAMER_E_PARAM for negative extents, bc not 0 or 1, an extent above
 * 2^26 groups, or more than (2^31 - 2048) / 1280 (about 1.68 million) groups
 * in one z-layer (gx*gy).
 * Results equal gamer_fill_ghosts_uniform_* followed by gamer_hydro_advance_*
 * bit for bit.
 */
int gamer_hydro_advance_level_f32(const float* level, float* out, float* face_flux, int32_t gx,
                                  int32_t gy, int32_t gz, int32_t bc, const double* dt,
                                  const double* dh, uint32_t* status, double* partials,
                                  const gh_params* p, void* stream);
int gamer_hydro_advance_level_mixed(const float* level, float* out, float* face_flux,
                                    int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                    const double* dt, const double* dh, uint32_t* status,
                                    double* partials, const gh_params* p, void* stream);
int gamer_hydro_advance_level_ff(const float* level, float* out, float* face_flux,
                                    int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                    const double* dt, const double* dh, uint32_t* status,
                                    double* partials, const gh_params* p, void* stream);
int gamer_hydro_advance_level_f64(const double* level, double* out, double* face_flux,
                                  int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                  const double* dt, const double* dh, uint32_t* status,
                                  double* partials, const gh_params* p, void* stream);

/*
 * gamer_hydro_advance_level_window_{f32,mixed,f64}: as
 * gamer_hydro_advance_level_* for the z-layers z0 .. z0+nz-1 of a gx*gy*gz
 * level of which the device holds only a window: zn consecutive layers
 * (layer = gx*gy groups, group order as in the level), the first being level
 * layer zb, the following ones zb+1, ... modulo gz (periodic wrap).  For
 * streaming a level through device memory in slabs (paper Sec. 3: out-of-core
 * computation); every layer the step reads (z0-1 .. z0+nz, wrapped for bc 0,
 * clamped for bc 1) must be in the window.
 *   window    [zn][gy][gx][5][16][16][16] device memory, 16-byte aligned.
 *   out, face_flux, dt, dh, status, partials: as gamer_hydro_advance_* with
 *             N = gx*gy*nz (group g is level group g + z0*gx*gy).
 * Returns GAMER_E_PARAM for extents as gamer_hydro_advance_level_*, for
 * z0 < 0, nz < 0, z0 + nz > gz, zb outside [0, gz), zn outside [0, gz], or a
 * needed layer missing from the window; nz = 0 is a no-op.
 */
int gamer_hydro_advance_level_window_f32(const float* window, float* out, float* face_flux,
                                         int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                         int32_t zb, int32_t zn, int32_t z0, int32_t nz,
                                         const double* dt, const double* dh, uint32_t* status,
                                         double* partials, const gh_params* p, void* stream);
int gamer_hydro_advance_level_window_mixed(const float* window, float* out, float* face_flux,
                                           int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                           int32_t zb, int32_t zn, int32_t z0, int32_t nz,
                                           const double* dt, const double* dh, uint32_t* status,
                                           double* partials, const gh_params* p, void* stream);
int gamer_hydro_advance_level_window_ff(const float* window, float* out, float* face_flux,
                                           int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                           int32_t zb, int32_t zn, int32_t z0, int32_t nz,
                                           const double* dt, const double* dh, uint32_t* status,
                                           double* partials, const gh_params* p, void* stream);
int gamer_hydro_advance_level_window_f64(const double* window, double* out, double* face_flux,
                                         int32_t gx, int32_t gy, int32_t gz, int32_t bc,
                                         int32_t zb, int32_t zn, int32_t z0, int32_t nz,
                                         const double* dt, const double* dh, uint32_t* status,
                                         double* partials, const gh_params* p, void* stream);

/*
 * gamer_fill_ghosts_uniform_{f32,f64}: ghost-zone preparation for a uniform
 * level (paper Sec. 2: the ghost-zone data each patch needs before the solver
 * runs).  level[G][5][16][16][16] holds the interiors of G = gx*gy*gz groups,
 * group id (z*gy + y)*gx + x; writes in[G][5][20][20][20], every one of the
 * 8000 cells (corners too) from the group itself or its neighbours.
 * bc: 0 periodic, 1 zero-gradient (outflow: nearest interior cell of the
 * level).  level and in must not overlap.  level element aligned, in
 * 16-byte aligned (16-byte vector stores).
 */
int gamer_fill_ghosts_uniform_f32(const float* level, float* in, int32_t gx, int32_t gy,
                                  int32_t gz, int32_t bc, void* stream);
int gamer_fill_ghosts_uniform_f64(const double* level, double* in, int32_t gx, int32_t gy,
                                  int32_t gz, int32_t bc, void* stream);

/*
 * gamer_hydro_dt: time step per AMR level and conservation totals, in FP64,
 * from the per-group partials of gamer_hydro_advance_* (the CFL condition of
 * the explicit scheme and the global sums the paper's code reduces over MPI):
 *   dt_out[l]   = cfl * dh_level[l] / max_{g : level[g] == l} partials[g][0]
 *                 (0 when no group of level l has a positive signal speed)
 *   totals[5]   = sum over all groups of partials[g][1..5]      (may be NULL)
 *   dt_group[g] = dt_out[level[g]], the next step's dt per group (may be NULL)
 * A NaN speed in the partials (a group the step abandoned, see
 * GAMER_ST_INTERNAL_TIMEOUT) makes its level's dt NaN.
 * level [N] int32 in [0, n_levels) or NULL (all groups in level 0);
 * 1 <= n_levels <= 64; cfl finite and > 0.  dh_level [n_levels], dt_out
 * [n_levels], totals [5], dt_group [N] are device arrays.  The reduction is
 * deterministic (fixed order).  It needs device scratch memory of
 * gamer_hydro_dt_workspace_bytes(N, n_levels) bytes, 8-byte aligned, owned by
 * the caller (0 is returned for invalid sizes).
 */
size_t gamer_hydro_dt_workspace_bytes(int64_t N, int32_t n_levels);
int gamer_hydro_dt(const double* partials, int64_t N, const int32_t* level, int32_t n_levels,
                   const double* dh_level, double cfl, double* dt_out, double* totals,
                   double* dt_group, void* workspace, size_t workspace_bytes, void* stream);

/*
 * gamer_hydro_dt_noalloc: gamer_hydro_dt without a workspace argument, for
 * callers that cannot allocate device memory -- for example a host AMR code
 * whose device memory is all owned by its own allocator and that hands this
 * library only the arrays it already holds, or a binding from a language with
 * no access to a CUDA allocator.  The paper has no counterpart; this is an
 * interface convenience.  The scratch is a fixed 64 KiB array in the library's
 * device memory (held on every GPU that loads the library until the process
 * exits), so the call allocates nothing.  It accepts the sizes whose workspace,
 * gamer_hydro_dt_workspace_bytes(N, n_levels), fits in 64 KiB -- every N up to
 * 64 Ki groups, and every N for n_levels <= 3 -- and returns GAMER_E_WORKSPACE
 * for larger ones.  Arguments, results and other errors are those of
 * gamer_hydro_dt.  The call looks up the scratch array's device address
 * (with the device current) every time it is made outside stream capture, so
 * it keeps working after cudaDeviceReset; during a capture it uses the address
 * of its last lookup on that device, so make the first call on a device
 * before any stream capture.  All calls share the one array and every call rewrites
 * the part it reads, so nothing needs clearing between calls; calls whose GPU
 * work overlaps (different streams, no ordering between them) race on it.
 */
int gamer_hydro_dt_noalloc(const double* partials, int64_t N, const int32_t* level,
                           int32_t n_levels, const double* dh_level, double cfl, double* dt_out,
                           double* totals, double* dt_group, void* stream);

/*
 * Device-resident uniform-level step as one CUDA graph (ghost fill -> hydro
 * step -> dt reduction, no host round trip).
 * gamer_level_graph_create captures, on a private stream, one step:
 * level_a -> (ghost fill into tiles) -> hydro step -> level_b, followed by
 * gamer_hydro_dt, whose dt_group output is the dt[] input of the next step.
 * A run of steps alternates this graph with the one created with level_a and
 * level_b swapped.  All pointers are caller-owned device arrays sized for
 * G = gx*gy*gz groups: level_a, level_b [G][5][16]^3 of the mode's element
 * type; tiles [G][5][20]^3 for a separate ghost-fill kernel, or NULL to fuse
 * the ghost gather into the step kernel (gamer_hydro_advance_level_*);
 * face_flux [G][6][5][16][16] or NULL; dt_group,
 * dh_group [G]; status [G] or NULL; partials [G][6]; dh_level, dt_level [1];
 * totals [5] or NULL; workspace of gamer_hydro_dt_workspace_bytes(G, 1) bytes.
 * dt_group must hold the first step's dt before the first launch.
 * p->cfl is the Courant number of the dt reduction.  The buffers must outlive
 * the graph.  gamer_level_graph_launch enqueues the step on `stream`.
 */
typedef struct gamer_level_graph gamer_level_graph;
int gamer_level_graph_create(int32_t mode, void* level_a, void* level_b, void* tiles,
                             void* face_flux, double* dt_group, const double* dh_group,
                             uint32_t* status, double* partials, int32_t gx, int32_t gy,
                             int32_t gz, int32_t bc, const gh_params* p, const double* dh_level,
                             double* dt_level, double* totals, void* workspace,
                             size_t workspace_bytes, gamer_level_graph** out);
int gamer_level_graph_launch(gamer_level_graph* g, void* stream);
int gamer_level_graph_destroy(gamer_level_graph* g);

/*
 * gamer_batch_graph_create: one step of a batch of N patch groups from uneven
 * AMR levels (each group with its own dt and dh; paper Sec. 2: patches of all
 * levels are batched to the GPU solver) as one CUDA graph: the time step of
 * every level from the partials of the previous step (gamer_hydro_dt with the
 * level map; dt_group[g] = dt_level[level[g]]), then one persistent launch of
 * gamer_hydro_advance_<mode> over all N groups, whose partials feed the next
 * replay.  Launched with gamer_level_graph_launch, destroyed with
 * gamer_level_graph_destroy.  A replay equals the two calls made directly, bit
 * for bit.
 *   in [N][5][20]^3 ghost-padded tiles, out [N][5][16]^3, face_flux as
 *   gamer_hydro_advance_* or NULL, dt_group [N] (written by the reduction),
 *   dh_group [N], level [N] int32 in [0, n_levels) or NULL, status [N] or NULL,
 *   partials [N][6] (must hold the partials of the state the first replay
 *   starts from, e.g. from a zero-dt step), dh_level and dt_level [n_levels],
 *   totals [5] or NULL, workspace of gamer_hydro_dt_workspace_bytes(N,
 *   n_levels) bytes.  All device memory, outliving the graph; mode
 *   GAMER_MODE_*; p->cfl is the Courant number.  Returns GAMER_E_PARAM for N <
 *   1, n_levels outside 1..64 or a bad mode / parameter, GAMER_E_WORKSPACE for
 *   a short workspace, and the errors of the captured calls.
 */
int gamer_batch_graph_create(int32_t mode, const void* in, void* out, void* face_flux,
                             double* dt_group, const double* dh_group, const int32_t* level,
                             int32_t n_levels, uint32_t* status, double* partials, int64_t N,
                             const gh_params* p, const double* dh_level, double* dt_level,
                             double* totals, void* workspace, size_t workspace_bytes,
                             gamer_level_graph** out_graph);

/*
 * Streamed host pipeline (the paper overlaps CPU, GPU and disk work, Sec. 2
 * and Sec. 3; here host->device copies, hydro steps and device->host copies
 * of successive batches overlap on three streams).
 * gamer_pipeline_create allocates three device buffer sets of batch_groups
 * groups each for precision `mode` (with face-flux buffers if with_flux).
 * gamer_pipeline_advance_host advances N groups held in HOST memory:
 * in_host [N][5][20]^3, out_host [N][5][16]^3, face_flux_host [N][6][5][16][16]
 * or NULL, dt_host, dh_host [N], status_host [N] or NULL, partials_host [N][6]
 * or NULL -- the same layouts as gamer_hydro_advance_*, element type by mode.
 * Host buffers should be page-locked (pinned) for the copies to overlap.  The
 * call returns when all results are in host memory; it waits with a deadline
 * (gamer_pipeline_set_timeout, default 60 s) and returns GAMER_E_TIMEOUT if
 * the GPU has not finished by then.  It allocates nothing.  One pipeline must
 * not be used by two host threads at once.
 *
 * After GAMER_E_TIMEOUT (here or in any gamer_pipeline_* call that copies),
 * that call's copies may still be queued: they will still read its host
 * inputs and write its host outputs.  Keep those buffers alive and untouched
 * until a later call on the pipeline returns GAMER_OK or
 * gamer_pipeline_destroy returns (it waits for the pipeline's streams).  Every
 * call on a pipeline whose previous call timed out first waits, up to the
 * timeout, for the pipeline's streams to drain, and returns GAMER_E_TIMEOUT
 * again, with nothing enqueued, if they have not.
 */
typedef struct gamer_pipeline gamer_pipeline;
int gamer_pipeline_create(int32_t mode, int64_t batch_groups, int32_t with_flux,
                          gamer_pipeline** out);
int gamer_pipeline_advance_host(gamer_pipeline* pl, const void* in_host, void* out_host,
                                void* face_flux_host, const double* dt_host,
                                const double* dh_host, uint32_t* status_host,
                                double* partials_host, int64_t N, const gh_params* p);
int gamer_pipeline_set_timeout(gamer_pipeline* pl, double seconds);
/* Test facility (not part of the scheme): holds the pipeline's three streams
 * for `seconds` (0 .. 60) with a host callback that sleeps, so that the next
 * call's bounded wait can be made to run out without any GPU-side wait. */
int gamer_pipeline_debug_hold(gamer_pipeline* pl, double seconds);

/*
 * gamer_pipeline_level_step_host: one step of a uniform level that lives in
 * HOST memory, streamed through the device in z-slabs (paper Sec. 3: a
 * problem larger than device memory processed piece by piece, transfers
 * overlapped with computation).  A slab is L layers of gx*gy groups, L*gx*gy
 * about the pipeline's batch size (at least one layer).  For each slab the 16^3
 * interiors of its layers and of the layer below and above (periodic wrap or,
 * for bc 1, the level's end layers) go to the device in at most two copies;
 * the slab is advanced by gamer_hydro_advance_level_window_* with the ghost
 * zones gathered on the device; its results come back into level_out_host.
 * Three slabs are in flight on the pipeline's three streams.  The host does
 * no ghost preparation: nthreads is ignored.
 * level_in_host, level_out_host [G][5][16]^3 (G = gx*gy*gz, element type by
 * mode, distinct, pinned for overlap); bc 0 periodic, 1 zero-gradient; one dt,
 * dh for the level; status_host [G] and partials_host [G][6] may be NULL.
 * The first call (and a call on a level whose slabs need more room) allocates
 * the device window buffers (held until gamer_pipeline_destroy).  Bounded
 * waits as for gamer_pipeline_advance_host; no face fluxes.
 *
 * When the level's input and output fit in 80 % of the free device memory
 * (or level mode 1 is set), the pipeline keeps a device copy of the whole
 * level instead (allocated once, held until destroy or level mode 2): each
 * slab of layers is copied in once, its kernel waits for its own copy and
 * the next slab's (the layer above) -- the periodic wrap layer goes first --
 * and its results go back while the next slabs are copied and advanced, so
 * every layer crosses the link once per step.
 *
 * gamer_pipeline_last_bytes: host->device and device->host bytes the last
 * advance_host, level_step_host or level_run_host call on this pipeline copied.
 *
 * gamer_pipeline_set_level_mode: 0 automatic (default), 1 always the device
 * copy of the level, 2 always slab windows with halo layers (frees the copy).
 */
int gamer_pipeline_level_step_host(gamer_pipeline* pl, const void* level_in_host,
                                   void* level_out_host, int32_t gx, int32_t gy, int32_t gz,
                                   int32_t bc, double dt, double dh, uint32_t* status_host,
                                   double* partials_host, const gh_params* p, int32_t nthreads);
int gamer_pipeline_last_bytes(const gamer_pipeline* pl, int64_t* h2d, int64_t* d2h);
int gamer_pipeline_set_level_mode(gamer_pipeline* pl, int32_t mode);

/*
 * gamer_pipeline_level_run_host: nsteps steps of a uniform level that lives in
 * HOST memory (paper Sec. 3: transfers overlapped with computation, here also
 * from one step to the next).  Step n reads level[n % 2] and writes
 * level[(n + 1) % 2] (level0, level1: [G][5][16]^3 host arrays, G =
 * gx*gy*gz, element type by mode, not overlapping, pinned for overlap); the
 * final state is in level[nsteps % 2].  Every step copies its input to the
 * device and its result back, in z-slabs of L layers as
 * gamer_pipeline_level_step_host with a device copy of the level; step n
 * takes its slabs in the order n, n+1, ... (mod the slab count), so a slab's
 * copy in waits only for the previous step's copy out of the same slab, and
 * the next step's copies in overlap this step's copies out.
 * Time step: dt0 (finite, >= 0) for step 0, e.g. from the partials of a
 * previous call; for n >= 1, cfl * dh / max_g partials[g][0] of step n-1
 * (gamer_hydro_dt on the device, the FP64 formula a host would use).
 * dh finite > 0, cfl finite > 0, nsteps >= 0, bc 0 periodic or 1
 * zero-gradient, extents as gamer_hydro_advance_level_*.
 *   dt_host       [nsteps] the dt of every step, or NULL.
 *   status_host   [G] GAMER_ST_* bits OR-ed over the steps, or NULL.
 *   partials_host [G][6] partials of the last step, or NULL.
 * Device memory: four copies of the level (input and output per step
 * parity) and per-group scratch, allocated on first use and held until
 * gamer_pipeline_destroy; GAMER_E_CUDA when they do not fit.  One bounded
 * wait at the end (the pipeline timeout times nsteps).  gamer_pipeline_last_bytes
 * reports the call's total bytes.
 */
int gamer_pipeline_level_run_host(gamer_pipeline* pl, void* level0, void* level1, int32_t gx,
                                  int32_t gy, int32_t gz, int32_t bc, int32_t nsteps, double dt0,
                                  double dh, double cfl, double* dt_host, uint32_t* status_host,
                                  double* partials_host, const gh_params* p);

/*
 * gamer_fill_ghosts_uniform_host_{f32,f64}: gamer_fill_ghosts_uniform_* on
 * HOST arrays, run by nthreads CPU threads (<= 0: all).  Synchronous.
 */
int gamer_fill_ghosts_uniform_host_f32(const float* level, float* in, int32_t gx, int32_t gy,
                                       int32_t gz, int32_t bc, int32_t nthreads);
int gamer_fill_ghosts_uniform_host_f64(const double* level, double* in, int32_t gx, int32_t gy,
                                       int32_t gz, int32_t bc, int32_t nthreads);
int gamer_pipeline_destroy(gamer_pipeline* pl);

/*
 * Host memory for the host-resident levels of gamer_pipeline_* (paper Sec. 3
 * keeps out-of-core data in host memory): gamer_host_alloc maps `bytes`
 * (rounded up to the transparent-huge-page size), asks for huge-page backing,
 * faults every page in with nthreads host threads (<= 0: all; the memory is
 * zero-filled) and page-locks it for CUDA (cudaHostRegister), so that device
 * copies from and to it run asynchronously at full link speed.  Huge pages
 * keep the translations that the copies walk few whatever the state of the
 * host's free memory.  Synchronous; returns GAMER_E_PARAM for 0 or more than
 * 2^46 bytes, GAMER_E_CUDA when the mapping or the registration fails.
 * gamer_host_free releases a pointer gamer_host_alloc returned (GAMER_E_PARAM
 * for any other); no device work may still use it.
 */
int gamer_host_alloc(size_t bytes, int32_t nthreads, void** out);
int gamer_host_free(void* ptr);

/* Message for a GAMER_E* return code (static string). */
const char* gamer_strerror(int code);

/* 0 when the current CUDA device can run this library (compute capability
 * 10.x, built for sm_103a), else GAMER_E_DEVICE or GAMER_E_CUDA. */
int gamer_device_check(void);

/* Library build identification (static string). */
const char* gamer_version(void);

/* Launch shape of gamer_hydro_advance_<mode> (mode = GAMER_MODE_*): CTAs per
 * SM of the persistent grid.  The FP32 modes come in two builds, sized for 2
 * CTAs per SM (no register spills) and for 3 (more warps per SM); 2 selects
 * the first, 0 or 3 the second (default).  FP64 always runs 1 CTA per SM.
 * Larger values are capped at what fits.  Used by the autotuner.
 * Process-wide and unsynchronised: every later launch of any host thread
 * reads it, so change it only while no other thread is launching steps. */
int gamer_set_hydro_ctas_per_sm(int32_t mode, int32_t ctas_per_sm);

/* Code shape of the hydro kernel: 0 = one problem at a time per thread, 160
 * threads per group (default); 1 = as 0 with one out-of-line copy of the
 * Riemann solver (FP32 3-CTA tile build only); 2 = two interleaved problems per
 * thread (z-face states in shared memory, branch-free Roe path, compile-time
 * limiter; 2 CTAs per SM in FP32, 1 in FP64; tile path only); 3 = 320 threads
 * per group, one owned column or face-slab cell per thread (2 CTAs per SM in
 * the FP32-storage modes, 1 in FP64), tile and level paths.  Where a variant does not
 * exist for a call (mode, path, HLLC or characteristic limiting) the default
 * shape runs.  Used by the autotuner; process-wide and unsynchronised like
 * gamer_set_hydro_ctas_per_sm. */
int gamer_set_hydro_variant(int32_t variant);

/* Debug facility (not part of the scheme): with on = 1, every later launch of
 * the level kernels (gamer_hydro_advance_level_*, _level_window_*) fills each
 * shared-memory input slot with NaN before gathering a plane into it (one
 * extra CTA barrier per plane), so a stencil read of a cell the gather does
 * not copy turns the results into NaN.  Results are unchanged when the gather
 * covers every cell read.  Process-wide; 0 (default) turns it off.  Returns
 * GAMER_E_PARAM for other values. */
int gamer_set_debug_poison(int32_t on);

/* Failure-detection test facility (not part of the scheme): with group >= 0,
 * every later launch of gamer_hydro_advance_* (default code shape) and of the
 * level kernels never issues the copy of input plane 5 of that group, so the
 * CTA's bounded wait for it runs out and its give-up path runs
 * (GAMER_ST_INTERNAL_TIMEOUT, see there) -- no fault, no hang.  wait_polls > 0
 * bounds every on-chip wait of those launches to that many polls (0: the
 * default bound, about 4 million).  group = -1 and wait_polls = 0 restore
 * normal operation.  Process-wide and unsynchronised; GAMER_E_PARAM for group
 * < -1 or wait_polls < 0. */
int gamer_set_debug_drop_plane(int64_t group, int32_t wait_polls);

/*
 * AMR coarse-fine coupling after one coarse step and its fine sub-steps: the
 * step that consumes the face fluxes of gamer_hydro_advance_*.  The paper
 * relies on GAMER's AMR structure (Sec. 1) without describing this coupling;
 * it is the conservative refluxing of Berger & Colella (1989) for refinement
 * ratio 2, where one fine patch group (16^3 fine cells) covers one octant
 * (8^3 cells) of a coarse patch group, so every coarse-fine interface lies on
 * a coarse group's flux plane at 0, 8 or 16 cells (flux_layout 1).
 *
 * gamer_cf_face: the 8x8 coarse faces of quadrant `quadrant` (bit 0: in-plane
 * index a from 8, bit 1: b from 8; [a][b] = [k][j] for x planes, [k][i] for y,
 * [j][i] for z) of plane `plane` (0, 1, 2 = 0, 8, 16 cells) along `dir` (0 x,
 * 1 y, 2 z) of coarse group `coarse`, covered by one face of fine group
 * `fine`.  side 1: the fine region lies on the + side of the corrected coarse
 * cells (layer 8*plane - 1; the fine group's -dir face); side 0: on their -
 * side (layer 8*plane; its +dir face).  Valid: plane >= 1 for side 1,
 * plane <= 1 for side 0.
 * gamer_cf_child: fine group `fine` covers octant `octant` (bit 0: x from 8,
 * bit 1: y, bit 2: z) of coarse group `coarse`; reserved = 0.
 */
typedef struct gamer_cf_face {
    int64_t coarse, fine;
    int32_t dir, plane, side, quadrant;
} gamer_cf_face;
typedef struct gamer_cf_child {
    int64_t coarse, fine;
    int32_t octant, reserved;
} gamer_cf_child;

/*
 * gamer_flux_fixup_{f32,f64}: each coarse cell beside a fine region gets
 *   U += s * (dt/dh)[coarse] * (F_c - <F_f>),  s = +1 (side 1) or -1 (side 0),
 * F_c its face flux from the coarse step and <F_f> the mean of the 2x2 fine
 * face fluxes over the n_sub equal fine sub-steps.  In place on the coarse
 * groups' updated state; applied class by class (2*dir + side = 0..5), so a
 * cell beside fine regions on several sides is corrected in that fixed order.
 * Arithmetic in FP64, rounded once per class to the storage type (mixed mode
 * uses _f32).
 *   coarse       [Nc][5][16][16][16] updated coarse state (in/out).
 *   coarse_flux  [Nc][9][5][16][16] the coarse step's face fluxes, flux_layout 1.
 *   fine_flux    [n_sub][Nf][6][5][16][16] the fine sub-steps' face fluxes.
 *   dt, dh       [Nc] the coarse groups' step and cell width (FP64).
 *   faces        [n_faces] records (device memory, 8-byte aligned).
 *   bad          device int32 or NULL: incremented once per invalid record
 *                (out-of-range index or field); such records are skipped.
 * All arrays are device memory; coarse must not overlap any input.  Returns
 * GAMER_OK, GAMER_E_PARAM (negative sizes, n_sub < 1), GAMER_E_NULL,
 * GAMER_E_ALIGN, GAMER_E_OVERLAP, GAMER_E_CUDA.  Asynchronous on `stream`.
 *
 * gamer_restrict_{f32,f64}: every coarse cell of a covered octant becomes the
 * mean of its 2x2x2 fine cells (FP64 sum in z, y, x order, times 1/8, rounded
 * once).  fine [Nf][5][16]^3, coarse [Nc][5][16]^3 (output; must not overlap
 * fine or the records), children [n_children] (device memory), bad as above.
 */
int gamer_flux_fixup_f32(float* coarse, const float* coarse_flux, const float* fine_flux,
                         int32_t n_sub, const double* dt, const double* dh, int64_t Nc,
                         int64_t Nf, const gamer_cf_face* faces, int64_t n_faces, int32_t* bad,
                         void* stream);
int gamer_flux_fixup_f64(double* coarse, const double* coarse_flux, const double* fine_flux,
                         int32_t n_sub, const double* dt, const double* dh, int64_t Nc,
                         int64_t Nf, const gamer_cf_face* faces, int64_t n_faces, int32_t* bad,
                         void* stream);
int gamer_restrict_f32(const float* fine, float* coarse, int64_t Nc, int64_t Nf,
                       const gamer_cf_child* children, int64_t n_children, int32_t* bad,
                       void* stream);
int gamer_restrict_f64(const double* fine, double* coarse, int64_t Nc, int64_t Nf,
                       const gamer_cf_child* children, int64_t n_children, int32_t* bad,
                       void* stream);

/* Throughput probes for the roofline denominators (not part of the scheme).
 * kind 0: FP32 FMA, 1: FP64 FMA, 2: FP32 MUFU reciprocal -- a grid of
 * 8 x 256 threads per SM, 8 dependent chains of `iters` operations per thread;
 * buf: device scratch of >= 8 KB.  kind 3: copies n floats from buf to buf + n
 * (buf holds 2n floats, 16-byte aligned, n a multiple of 4).  *work (host)
 * receives the operation count (kinds 0-2) or bytes read + written (kind 3).
 * The caller times the launch on `stream`. */
int gamer_microbench(int32_t kind, int64_t iters, void* buf, int64_t n, double* work,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GAMER_GB300_H */
