/*
 * gamer_oracle.h -- C interface of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no source with the CUDA library (its own header, its own types).
 *
 * Method: one unsplit MUSCL-Hancock finite-volume step with Roe's approximate
 * Riemann solver (paper Sec. 2: "spatial data reconstruction, half-step
 * prediction, Riemann solver, full-step update", unsplit, Roe's solver, a
 * five-point stencil per direction; the scheme itself is the one of the cited
 * textbook, Toro 2009, with Roe 1981).  Every detail the paper leaves open is
 * fixed by a documented reading (see the comments in gamer_oracle.cpp).
 *
 * Array layouts (all row-major, x fastest):
 *   box input   in [5][nz+4][ny+4][nx+4]   conserved (rho, mx, my, mz, E), 2 ghosts/side
 *   box output  out[5][nz][ny][nx]
 *   face fluxes six blocks, in order -x,+x,-y,+y,-z,+z:
 *               x faces [5][nz][ny], y faces [5][nz][nx], z faces [5][ny][nx]
 *   patch group = the box with nx = ny = nz = 16 (20^3 input, 16^3 output,
 *               face flux [6][5][16][16]).
 */
#ifndef GAMER_ORACLE_H
#define GAMER_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double gamma;            /* ratio of specific heats, > 1                       */
    int32_t limiter;         /* 0 van Leer (harmonic), 1 minmod, 2 monotonised central */
    int32_t predictor_fallback; /* 0: cell average, 1: un-evolved reconstruction   */
    double rho_floor;        /* >= 0; 0 = off: updated rho below it is raised to it  */
    double p_floor;          /* >= 0; 0 = off: updated p below it is raised to it   */
    int32_t flux_layout;     /* 0: six box faces; 1: nine planes, three per direction
                                at 0, n/2 and n cells (n even)                       */
    int32_t riemann;         /* 0: Roe with HLLE fallback (the paper's); 1: HLLC     */
    int32_t reconstruction;  /* slopes limited in 0: primitive variables (the paper's
                                reading), 1: characteristic variables                */
} oracle_params;

/* status bits (per box / per group) */
#define ORACLE_ST_PREDICTOR_FALLBACK 1u
#define ORACLE_ST_HLLE_FALLBACK      2u
#define ORACLE_ST_NONPOSITIVE_OUT    4u
#define ORACLE_ST_BAD_INPUT          8u
#define ORACLE_ST_FLOOR             32u

/* One step on a general ghost-padded box.  face_flux, status, partials may be
 * NULL.  partials[6] = { max over cells of max_d|v_d| + c, sum rho, sum mx,
 * sum my, sum mz, sum E } over the updated cells.  Returns 0, or -1 on a bad
 * argument (null array, n < 1, gamma <= 1, unknown limiter). */
int oracle_advance_box(const double* in, int nx, int ny, int nz, double* out,
                       double* face_flux, double dt, double dh, const oracle_params* p,
                       uint32_t* status, double* partials);

/* N independent 16^3 patch groups: in[N][5][20][20][20], out[N][5][16][16][16],
 * face_flux[N][6 or 9][5][16][16] (or NULL), dt[N], dh[N], status[N] (or NULL),
 * partials[N][6] (or NULL).  nthreads > 1 spreads groups over OpenMP threads. */
int oracle_advance_groups(const double* in, double* out, double* face_flux,
                          const double* dt, const double* dh, int64_t N,
                          const oracle_params* p, uint32_t* status, double* partials,
                          int nthreads);

/* Uniform-level ghost fill: level[G][5][16][16][16] with G = gx*gy*gz groups,
 * group id = (z*gy + y)*gx + x; writes in[G][5][20][20][20] (all 8000 cells,
 * corners included).  bc 0 = periodic, 1 = zero-gradient (outflow). */
int oracle_fill_ghosts_uniform(const double* level, int gx, int gy, int gz, int bc,
                               double* in);

/* Time step and conservation totals from per-group partials[N][6]:
 * dt_out[l] = cfl * dh_level[l] / max_{g in level l} partials[g][0]
 * (0 when that maximum is not positive); totals[5] = sum_g partials[g][1..5].
 * level may be NULL (all groups in level 0). */
int oracle_hydro_dt(const double* partials, int64_t N, const int32_t* level,
                    int32_t n_levels, const double* dh_level, double cfl,
                    double* dt_out, double* totals);

/* ---- AMR coarse-fine coupling after a coarse step and its fine sub-steps ----
 * Geometry: refinement ratio 2; a fine patch group (16^3 fine cells) covers one
 * octant (8^3 cells) of a coarse patch group, so coarse-fine interfaces lie on
 * the coarse groups' flux planes at 0, 8 or 16 cells (flux_layout 1).
 *
 * One interface record: the 8x8 coarse faces of quadrant `quadrant` (bit 0: in-
 * plane index a from 8, bit 1: b from 8; [a][b] = [k][j] for x planes, [k][i]
 * for y, [j][i] for z) of plane `plane` (0, 1, 2) along `dir` of coarse group
 * `coarse`, covered by one face of fine group `fine`.  side 1: the fine region
 * lies on the + side of the corrected coarse cells (layer 8*plane - 1; the fine
 * group's -dir face); side 0: on their - side (layer 8*plane; its +dir face). */
typedef struct {
    int64_t coarse, fine;
    int32_t dir, plane, side, quadrant;
} oracle_cf_face;

/* Flux fix-up (refluxing, Berger & Colella 1989): each coarse cell beside a
 * fine region gets U += s * (dt/dh)_coarse * (F_c - <F_f>), s = +1 for side 1
 * and -1 for side 0, F_c its coarse face flux (coarse_flux [Nc][9][5][16][16])
 * and <F_f> the mean of the 2x2 fine face fluxes over the n_sub equal sub-steps
 * (fine_flux [n_sub][Nf][6][5][16][16]).  Records are applied class by class
 * (2*dir + side = 0..5), each class in record order.  Returns the number of
 * invalid records (skipped) or -1 on a bad argument. */
int64_t oracle_flux_fixup(double* coarse, const double* coarse_flux, const double* fine_flux,
                          int n_sub, const double* dt, const double* dh, int64_t Nc, int64_t Nf,
                          const oracle_cf_face* faces, int64_t n);

/* One child record: fine group `fine` covers octant `octant` (bit 0: x from 8,
 * bit 1: y, bit 2: z) of coarse group `coarse`. */
typedef struct {
    int64_t coarse, fine;
    int32_t octant, reserved;
} oracle_cf_child;

/* Restriction: each coarse cell of a covered octant becomes the mean of its
 * 2x2x2 fine cells (conservative average).  fine [Nf][5][16]^3, coarse
 * [Nc][5][16]^3.  Returns the number of invalid records or -1. */
int64_t oracle_restrict(const double* fine, double* coarse, int64_t Nc, int64_t Nf,
                        const oracle_cf_child* children, int64_t n);

/* ---- pieces, exposed for unit pins ---- */
void oracle_prim_from_cons(const double U[5], double gamma, double W[5]);
void oracle_cons_from_prim(const double W[5], double gamma, double U[5]);
void oracle_euler_flux(int dir, const double W[5], double E, double F[5]);
double oracle_limiter(int id, double a, double b);
/* Characteristic-limited slope of the primitive state Wc (rho, vx, vy, vz, p)
 * along dir from its neighbours Wl, Wr (scheme variant). */
void oracle_char_slopes(int dir, const double Wl[5], const double Wc[5], const double Wr[5],
                        double gamma, int limiter, double slope[5]);
/* HLLC flux (scheme variant) in direction dir from conserved L/R states. */
void oracle_hllc_flux(int dir, const double UL[5], const double UR[5], double gamma, double F[5]);
/* Roe flux in direction dir from conserved L/R states; returns 1 when the HLLE
 * fallback replaced it, else 0.  entropy_fix = 0 switches the fix off (pins). */
int oracle_roe_flux(int dir, const double UL[5], const double UR[5], double gamma,
                    int entropy_fix, double F[5]);
void oracle_hlle_flux(int dir, const double UL[5], const double UR[5], double gamma,
                      double F[5]);

/* Exact Riemann solver (textbook Newton iteration for p*).  star[4] = {p*, u*,
 * rho*_L, rho*_R}.  Returns number of Newton iterations, or -1 on failure
 * (vacuum generation). */
int oracle_exact_riemann_star(double rl, double ul, double pl, double rr, double ur,
                              double pr, double gamma, double star[4]);
/* Samples the self-similar solution at xi = x/t; W[3] = {rho, u, p}. */
void oracle_exact_riemann_sample(double rl, double ul, double pl, double rr, double ur,
                                 double pr, double gamma, double xi, double W[3]);

/* Operation tally of one 16^3-group step (the same code run on a counting
 * scalar).  counts[6] = {add/sub, mul, div, sqrt, compare/min/max/abs, cells}.
 * Returns 0 on success. */
int oracle_count_ops_group(const double* in, double dt, double dh, const oracle_params* p,
                           double counts[6]);

/* Operation tally of one piece of the scheme on the counting scalar, for pins
 * of the tally against hand counts: piece 0 prim(a), 1 cons(a), 2 the Euler
 * flux along dir of primitive a with total energy b[0], 3 the configured
 * (default van Leer) limiter of a[0], b[0], 4 one Roe flux along dir of the
 * conserved states a, b (entropy fix on), 5 the admissibility test of the
 * conserved state a.  counts[5] = {add/sub, mul, div, sqrt, compare}.
 * Returns 0, or -1 on a bad argument. */
int oracle_count_ops_piece(int piece, int dir, const double* a, const double* b, double gamma,
                           double counts[5]);

#ifdef __cplusplus
}
#endif
#endif
