// gamer_oracle.cpp -- plain FP64 CPU oracle of the MUSCL-Hancock + Roe hydro step.
//
// TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
// CPU-baseline leg load this library; the CUDA product path never does, and the
// two share no source.  Built with -O2 -ffp-contract=off so that every operation
// is rounded as written.
//
// What it computes (paper Sec. 2): one unsplit finite-volume step of the
// MUSCL-Hancock method (Toro 2009) with Roe's Riemann solver (Roe 1981), in the
// four stages the paper names -- spatial data reconstruction, half-step
// prediction, Riemann solver, full-step update -- on a box with a two-cell ghost
// shell (the paper's five-point stencil per direction).  The paper gives no
// formulas; the readings taken where it is silent are marked READING below and
// are the ones this repository's design notes list:
//   R1 reconstruction of the primitive variables (rho, u, v, w, p), per component;
//   R2 slope limiter: van Leer harmonic 2ab/(a+b) if ab > 0 else 0 (default),
//      minmod and monotonised central as options;
//   R3 half-step: Toro's conservative evolution of the boundary-extrapolated
//      values, one common increment 0.5*dt/dh * sum_d [F_d(U^{d,-}) - F_d(U^{d,+})]
//      added to all six face states (unsplit), directions summed x, y, z;
//   R4 predictor fallback: if any of the six evolved face states has rho <= 0
//      or p <= 0, all six are replaced by the cell average (option 1: by the
//      un-evolved reconstructed states);
//   R5 Roe flux in a rotated frame (normal, t1, t2) = cyclic (x,y,z), wave
//      strengths from primitive jumps;
//   R6 entropy fix on the two acoustic waves: Harten's smoothing
//      |l| -> (l^2 + d^2)/(2d) when |l| < d, with the Harten-Hyman width
//      d = max(0, l~ - l(left state of the wave), l(right state) - l~), the
//      wave's side states being U_L and U*_L (wave 1), U*_R and U_R (wave 5);
//   R7 HLLE fallback (Einfeldt speeds) when the Roe sound speed squared is not
//      positive or either Roe intermediate state has rho <= 0 or p <= 0;
//      without a Roe sound speed, Davis's bounds over both states;
//   R9 no density or pressure floors;
//   R11 face fluxes emitted as the raw physical flux used by the update.
#include "gamer_oracle.h"

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdlib>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Counting scalar: the same scheme source instantiated on this type tallies the
// arithmetic it performs (used for the algorithmic-flop figure of a step).
struct Tally {
    double add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0;
};
thread_local Tally g_tally;

struct Cnt {
    double v;
    Cnt() : v(0.0) {}
    Cnt(double x) : v(x) {}  // NOLINT: implicit on purpose (literals)
};
inline Cnt operator+(Cnt a, Cnt b) { g_tally.add += 1; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_tally.add += 1; return Cnt(a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_tally.mul += 1; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_tally.div += 1; return Cnt(a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline bool operator<(Cnt a, Cnt b) { g_tally.cmp += 1; return a.v < b.v; }
inline bool operator>(Cnt a, Cnt b) { g_tally.cmp += 1; return a.v > b.v; }
inline bool operator<=(Cnt a, Cnt b) { g_tally.cmp += 1; return a.v <= b.v; }
inline bool operator>=(Cnt a, Cnt b) { g_tally.cmp += 1; return a.v >= b.v; }

inline double val(double x) { return x; }
inline double val(Cnt x) { return x.v; }
inline double r_sqrt(double x) { return std::sqrt(x); }
inline Cnt r_sqrt(Cnt x) { g_tally.sqrt += 1; return Cnt(std::sqrt(x.v)); }

template <class R> inline R r_abs(R x) { return (x < R(0.0)) ? -x : x; }
template <class R> inline R r_max(R a, R b) { return (a > b) ? a : b; }
template <class R> inline R r_min(R a, R b) { return (a < b) ? a : b; }

// ---------------------------------------------------------------------------
template <class R>
struct Scheme {
    R gamma;
    R gm1;  // gamma - 1
    int limiter;
    int pred_fallback;
    R rho_floor = R(0.0);  // 0: off
    R p_floor = R(0.0);    // 0: off
    int flux_layout = 0;   // 0: six box faces, 1: nine planes
    int solver = 0;        // Riemann solver: 0 Roe (with HLLE fallback), 1 HLLC
    int recon = 0;         // slopes limited in 0: primitive, 1: characteristic variables

    // Conserved -> primitive.  p = (gamma-1) (E - 0.5 |m|^2 / rho).
    void prim(const R U[5], R W[5]) const {
        W[0] = U[0];
        W[1] = U[1] / U[0];
        W[2] = U[2] / U[0];
        W[3] = U[3] / U[0];
        R ke = R(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
        W[4] = gm1 * (U[4] - ke);
    }
    R pressure(const R U[5]) const {
        R ke = R(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
        return gm1 * (U[4] - ke);
    }
    // Primitive -> conserved.  E = p/(gamma-1) + 0.5 rho |v|^2.
    void cons(const R W[5], R U[5]) const {
        U[0] = W[0];
        U[1] = W[0] * W[1];
        U[2] = W[0] * W[2];
        U[3] = W[0] * W[3];
        U[4] = W[4] / gm1 + R(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
    }
    // Physical Euler flux in direction d from primitive W and total energy E.
    static void flux(int d, const R W[5], R E, R F[5]) {
        R un = W[1 + d];
        R m = W[0] * un;
        F[0] = m;
        F[1] = m * W[1];
        F[2] = m * W[2];
        F[3] = m * W[3];
        F[1 + d] = F[1 + d] + W[4];
        F[4] = (E + W[4]) * un;
    }
    // READING R21 (scheme variant): slopes limited in the characteristic
    // variables of the primitive Euler system along direction d, at the cell's
    // own state (rho, u_n, u_t1, u_t2, p; c^2 = gamma p / rho):
    //   left eigenvectors  l1 = (0, -rho/(2c), 0, 0, 1/(2c^2)), l2 = (1, 0, 0, 0, -1/c^2),
    //                      l3 = e_t1, l4 = e_t2, l5 = (0, rho/(2c), 0, 0, 1/(2c^2));
    //   right eigenvectors r1 = (1, -c/rho, 0, 0, c^2), r2 = e_rho, r3 = e_t1,
    //                      r4 = e_t2, r5 = (1, c/rho, 0, 0, c^2).
    // Each characteristic component is limited from its left and right
    // differences and the slope is projected back; where c^2 <= 0 the
    // primitive slopes are used.
    void char_slopes(int d, const R Wl[5], const R Wc[5], const R Wr[5], R sl[5]) const {
        const R c2 = gamma * Wc[4] / Wc[0];
        if (!(c2 > R(0.0))) {
            for (int q = 0; q < 5; ++q) sl[q] = limit(Wc[q] - Wl[q], Wr[q] - Wc[q]);
            return;
        }
        const int n = 1 + d, t1 = 1 + (d + 1) % 3, t2 = 1 + (d + 2) % 3;
        const R c = r_sqrt(c2);
        R dl[5], dr[5];
        for (int q = 0; q < 5; ++q) {
            dl[q] = Wc[q] - Wl[q];
            dr[q] = Wr[q] - Wc[q];
        }
        R al[5], ar[5];
        const R* dW[2] = {dl, dr};
        R* a[2] = {al, ar};
        for (int s = 0; s < 2; ++s) {
            a[s][0] = R(0.5) * (dW[s][4] / c2 - Wc[0] * dW[s][n] / c);
            a[s][1] = dW[s][0] - dW[s][4] / c2;
            a[s][2] = dW[s][t1];
            a[s][3] = dW[s][t2];
            a[s][4] = R(0.5) * (dW[s][4] / c2 + Wc[0] * dW[s][n] / c);
        }
        R da[5];
        for (int k = 0; k < 5; ++k) da[k] = limit(al[k], ar[k]);
        sl[0] = da[0] + da[1] + da[4];
        sl[n] = c / Wc[0] * (da[4] - da[0]);
        sl[t1] = da[2];
        sl[t2] = da[3];
        sl[4] = c2 * (da[0] + da[4]);
    }

    // READING R2: limited slope from the left and right differences.
    R limit(R a, R b) const {
        if (!(a * b > R(0.0))) return R(0.0);
        if (limiter == 1) {  // minmod
            return (a > R(0.0)) ? r_min(a, b) : r_max(a, b);
        }
        if (limiter == 2) {  // monotonised central
            R s = (a > R(0.0)) ? R(1.0) : R(-1.0);
            R m = r_min(R(2.0) * r_abs(a), R(2.0) * r_abs(b));
            m = r_min(m, R(0.5) * r_abs(a + b));
            return s * m;
        }
        return R(2.0) * a * b / (a + b);  // van Leer harmonic
    }
    bool positive(const R U[5]) const {
        return (U[0] > R(0.0)) && (pressure(U) > R(0.0));
    }

    // READING R7: HLLE flux with Einfeldt speed estimates.  When the Roe state
    // is usable (have_roe) its speeds widen the bounds u_L - c_L, u_R + c_R;
    // without it, Davis's bounds over both states, which keep S_L < S_R also
    // in a supersonic collision (u_L - c_L > 0 > u_R + c_R).
    void hlle(const R UL[5], const R UR[5], const R FL[5], const R FR[5], R uL, R cL, R uR,
              R cR, bool have_roe, R uT, R cT, R F[5]) const {
        R sl = uL - cL;
        R sr = uR + cR;
        if (have_roe) {
            sl = r_min(sl, uT - cT);
            sr = r_max(sr, uT + cT);
        } else {
            sl = r_min(sl, uR - cR);
            sr = r_max(sr, uL + cL);
        }
        R bm = r_min(sl, R(0.0));
        R bp = r_max(sr, R(0.0));
        for (int i = 0; i < 5; ++i)
            F[i] = (bp * FL[i] - bm * FR[i] + bp * bm * (UR[i] - UL[i])) / (bp - bm);
    }

    // READINGS R5-R7: Roe flux through a face normal to direction d.
    // Returns true when the HLLE fallback was used.
    bool roe(int d, const R UL[5], const R UR[5], bool efix, R F[5]) const {
        R WL[5], WR[5], FL[5], FR[5];
        prim(UL, WL);
        prim(UR, WR);
        flux(d, WL, UL[4], FL);
        flux(d, WR, UR[4], FR);
        const int n = 1 + d, t1 = 1 + (d + 1) % 3, t2 = 1 + (d + 2) % 3;
        R uL = WL[n], vL = WL[t1], wL = WL[t2];
        R uR = WR[n], vR = WR[t1], wR = WR[t2];
        R cL = r_sqrt(gamma * WL[4] / WL[0]);
        R cR = r_sqrt(gamma * WR[4] / WR[0]);
        R HL = (UL[4] + WL[4]) / WL[0];
        R HR = (UR[4] + WR[4]) / WR[0];
        // Roe averages
        R rr = r_sqrt(WR[0] / WL[0]);
        R uT = (uL + rr * uR) / (R(1.0) + rr);
        R vT = (vL + rr * vR) / (R(1.0) + rr);
        R wT = (wL + rr * wR) / (R(1.0) + rr);
        R HT = (HL + rr * HR) / (R(1.0) + rr);
        R q2 = uT * uT + vT * vT + wT * wT;
        R cT2 = gm1 * (HT - R(0.5) * q2);
        if (!(cT2 > R(0.0))) {
            hlle(UL, UR, FL, FR, uL, cL, uR, cR, false, R(0.0), R(0.0), F);
            return true;
        }
        R cT = r_sqrt(cT2);
        R rT = rr * WL[0];
        // wave strengths from the primitive jumps
        R dr = WR[0] - WL[0];
        R du = uR - uL;
        R dv = vR - vL;
        R dw = wR - wL;
        R dp = WR[4] - WL[4];
        R a1 = (dp - rT * cT * du) / (R(2.0) * cT2);
        R a2 = dr - dp / cT2;
        R a3 = rT * dv;
        R a4 = rT * dw;
        R a5 = (dp + rT * cT * du) / (R(2.0) * cT2);
        // right eigenvectors (rotated frame: rho, m_n, m_t1, m_t2, E)
        R K1[5] = {R(1.0), uT - cT, vT, wT, HT - uT * cT};
        R K5[5] = {R(1.0), uT + cT, vT, wT, HT + uT * cT};
        // READING R7: positivity of the two Roe intermediate states
        R ULr[5] = {UL[0], UL[n], UL[t1], UL[t2], UL[4]};
        R URr[5] = {UR[0], UR[n], UR[t1], UR[t2], UR[4]};
        R S1[5], S4[5];
        for (int i = 0; i < 5; ++i) {
            S1[i] = ULr[i] + a1 * K1[i];
            S4[i] = URr[i] - a5 * K5[i];
        }
        if (!positive(S1) || !positive(S4)) {
            hlle(UL, UR, FL, FR, uL, cL, uR, cR, true, uT, cT, F);
            return true;
        }
        // eigenvalues; READING R6: Harten's smoothing of |lambda| on the two
        // acoustic waves with the Harten-Hyman width taken from the states on
        // either side of each wave: (U_L, U*_L) for wave 1, (U*_R, U_R) for wave 5.
        R l1 = uT - cT, l5 = uT + cT;
        R e1 = r_abs(l1), e2 = r_abs(uT), e5 = r_abs(l5);
        if (efix) {
            R W1[5], W4[5];
            prim(S1, W1);
            prim(S4, W4);
            R l1s = W1[1] - r_sqrt(gamma * W1[4] / W1[0]);  // lambda_1 of U*_L
            R l5s = W4[1] + r_sqrt(gamma * W4[4] / W4[0]);  // lambda_5 of U*_R
            R d1 = r_max(R(0.0), r_max(l1 - (uL - cL), l1s - l1));
            if (e1 < d1) e1 = (l1 * l1 + d1 * d1) / (R(2.0) * d1);
            R d5 = r_max(R(0.0), r_max(l5 - l5s, (uR + cR) - l5));
            if (e5 < d5) e5 = (l5 * l5 + d5 * d5) / (R(2.0) * d5);
        }
        // dissipation sum_k |lambda_k| alpha_k K_k, waves in order 1..5
        // (K2 = (1, u, v, w, q2/2), K3 = (0,0,1,0,v), K4 = (0,0,0,1,w))
        R s1 = e1 * a1, s2 = e2 * a2, s3 = e2 * a3, s4 = e2 * a4, s5 = e5 * a5;
        R D[5];
        D[0] = s1 + s2 + s5;
        D[1] = s1 * K1[1] + s2 * uT + s5 * K5[1];
        D[2] = s1 * vT + s2 * vT + s3 + s5 * vT;
        D[3] = s1 * wT + s2 * wT + s4 + s5 * wT;
        D[4] = s1 * K1[4] + s2 * (R(0.5) * q2) + s3 * vT + s4 * wT + s5 * K5[4];
        R Du[5];
        Du[0] = D[0];
        Du[n] = D[1];
        Du[t1] = D[2];
        Du[t2] = D[3];
        Du[4] = D[4];
        for (int i = 0; i < 5; ++i) F[i] = R(0.5) * (FL[i] + FR[i]) - R(0.5) * Du[i];
        return false;
    }

    // READING R20 (scheme variant): HLLC flux through a face normal to
    // direction d (Toro 2009, Sec. 10.4).  Wave-speed bounds as the HLLE of
    // R7 (Einfeldt's with the Roe speeds, Davis's when c~^2 <= 0); contact
    // speed S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R)) /
    // (rho_L (S_L - u_L) - rho_R (S_R - u_R)); star states
    // U*_K = rho_K (S_K - u_K) / (S_K - S*) (1, S*, v_K, w_K,
    // E_K / rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))); the flux is
    // F_L, F_L + S_L (U*_L - U_L), F_R + S_R (U*_R - U_R) or F_R by where the
    // face lies in the fan.
    void hllc(int d, const R UL[5], const R UR[5], R F[5]) const {
        R WL[5], WR[5], FL[5], FR[5];
        prim(UL, WL);
        prim(UR, WR);
        flux(d, WL, UL[4], FL);
        flux(d, WR, UR[4], FR);
        const int n = 1 + d, t1 = 1 + (d + 1) % 3, t2 = 1 + (d + 2) % 3;
        R cL = r_sqrt(gamma * WL[4] / WL[0]);
        R cR = r_sqrt(gamma * WR[4] / WR[0]);
        R rr = r_sqrt(WR[0] / WL[0]);
        R uT = (WL[n] + rr * WR[n]) / (R(1.0) + rr);
        R vT = (WL[t1] + rr * WR[t1]) / (R(1.0) + rr);
        R wT = (WL[t2] + rr * WR[t2]) / (R(1.0) + rr);
        R HT = ((UL[4] + WL[4]) / WL[0] + rr * (UR[4] + WR[4]) / WR[0]) / (R(1.0) + rr);
        R cT2 = gm1 * (HT - R(0.5) * (uT * uT + vT * vT + wT * wT));
        R sl = WL[n] - cL, sr = WR[n] + cR;
        if (cT2 > R(0.0)) {
            sl = r_min(sl, uT - r_sqrt(cT2));
            sr = r_max(sr, uT + r_sqrt(cT2));
        } else {
            sl = r_min(sl, WR[n] - cR);
            sr = r_max(sr, WL[n] + cL);
        }
        R ss = (WR[4] - WL[4] + WL[0] * WL[n] * (sl - WL[n]) - WR[0] * WR[n] * (sr - WR[n])) /
               (WL[0] * (sl - WL[n]) - WR[0] * (sr - WR[n]));
        if (sl >= R(0.0)) {
            for (int i = 0; i < 5; ++i) F[i] = FL[i];
            return;
        }
        if (sr <= R(0.0)) {
            for (int i = 0; i < 5; ++i) F[i] = FR[i];
            return;
        }
        const bool left = ss >= R(0.0);
        const R* U = left ? UL : UR;
        const R* W = left ? WL : WR;
        const R* FK = left ? FL : FR;
        const R sK = left ? sl : sr;
        const R fac = W[0] * (sK - W[n]) / (sK - ss);
        R Us[5];
        Us[0] = fac;
        Us[n] = fac * ss;
        Us[t1] = fac * W[t1];
        Us[t2] = fac * W[t2];
        Us[4] = fac * (U[4] / W[0] + (ss - W[n]) * (ss + W[4] / (W[0] * (sK - W[n]))));
        for (int i = 0; i < 5; ++i) F[i] = FK[i] + sK * (Us[i] - U[i]);
    }

    // The Riemann flux of the configured solver; true when Roe fell back to HLLE.
    bool riemann(int d, const R UL[5], const R UR[5], R F[5]) const {
        if (solver == 1) {
            hllc(d, UL, UR, F);
            return false;
        }
        return roe(d, UL, UR, true, F);
    }
};

// cells of a padded box that the step reads (see READING on corner ghosts):
// at most one coordinate outside the box, or exactly two, both one cell out.
inline bool is_read_cell(int i, int j, int k, int nx, int ny, int nz) {
    const int oi = (i < 0 || i >= nx), oj = (j < 0 || j >= ny), ok = (k < 0 || k >= nz);
    const int o = oi + oj + ok;
    if (o <= 1) return true;
    if (o == 3) return false;
    const bool di = !oi || i == -1 || i == nx;
    const bool dj = !oj || j == -1 || j == ny;
    const bool dk = !ok || k == -1 || k == nz;
    return di && dj && dk;
}

template <class R>
int advance_box(const Scheme<R>& S, const R* in, int nx, int ny, int nz, R* out, R* ff, R dt,
                R dh, uint32_t* status_out, R* partials) {
    const int px = nx + 4, py = ny + 4, pz = nz + 4;
    const std::size_t pcells = (std::size_t)px * py * pz;
    uint32_t st = 0;
    if (!(std::isfinite(val(dt)) && std::isfinite(val(dh)) && val(dt) >= 0.0 && val(dh) > 0.0))
        st |= ORACLE_ST_BAD_INPUT;
    auto pidx = [&](int i, int j, int k) -> std::size_t {
        return ((std::size_t)(k + 2) * py + (j + 2)) * px + (i + 2);
    };
    auto U_in = [&](int i, int j, int k, R U[5]) {
        for (int v = 0; v < 5; ++v) U[v] = in[v * pcells + pidx(i, j, k)];
    };
    for (int k = -2; k < nz + 2; ++k)
        for (int j = -2; j < ny + 2; ++j)
            for (int i = -2; i < nx + 2; ++i) {
                if (!is_read_cell(i, j, k, nx, ny, nz)) continue;
                R U[5];
                U_in(i, j, k, U);
                for (int v = 0; v < 5; ++v)
                    if (!std::isfinite(val(U[v]))) st |= ORACLE_ST_BAD_INPUT;
            }
    const R lam = dt / dh;

    // Stage 1 (reconstruction input): primitive variables of every cell.
    std::vector<R> W(pcells * 5);
    for (int k = -2; k < nz + 2; ++k)
        for (int j = -2; j < ny + 2; ++j)
            for (int i = -2; i < nx + 2; ++i) {
                R U[5];
                U_in(i, j, k, U);
                S.prim(U, &W[pidx(i, j, k) * 5]);
            }

    // Stages 1-2: limited slopes and the Hancock half-step for every cell of
    // the predicted set (interior plus one-deep face slabs).
    const int qx = nx + 2, qy = ny + 2;
    auto qidx = [&](int i, int j, int k) -> std::size_t {
        return ((std::size_t)(k + 1) * qy + (j + 1)) * qx + (i + 1);
    };
    std::vector<R> Uh((std::size_t)qx * qy * (nz + 2) * 30);  // [cell][face][var]
    const R half_lam = R(0.5) * lam;
    for (int k = -1; k <= nz; ++k)
        for (int j = -1; j <= ny; ++j)
            for (int i = -1; i <= nx; ++i) {
                const int o = (i < 0 || i >= nx) + (j < 0 || j >= ny) + (k < 0 || k >= nz);
                if (o > 1) continue;
                const R* Wc = &W[pidx(i, j, k) * 5];
                R Uc[5];
                U_in(i, j, k, Uc);
                R Wf[6][5], Uf[6][5];
                for (int d = 0; d < 3; ++d) {
                    const int di = (d == 0), dj = (d == 1), dk = (d == 2);
                    const R* Wl = &W[pidx(i - di, j - dj, k - dk) * 5];
                    const R* Wr = &W[pidx(i + di, j + dj, k + dk) * 5];
                    R slope[5];
                    if (S.recon == 1) {
                        S.char_slopes(d, Wl, Wc, Wr, slope);
                    } else {
                        for (int q = 0; q < 5; ++q) slope[q] = S.limit(Wc[q] - Wl[q], Wr[q] - Wc[q]);
                    }
                    for (int q = 0; q < 5; ++q) {
                        Wf[2 * d][q] = Wc[q] - R(0.5) * slope[q];
                        Wf[2 * d + 1][q] = Wc[q] + R(0.5) * slope[q];
                    }
                    S.cons(Wf[2 * d], Uf[2 * d]);
                    S.cons(Wf[2 * d + 1], Uf[2 * d + 1]);
                }
                R acc[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
                for (int d = 0; d < 3; ++d) {
                    R Fm[5], Fp[5];
                    Scheme<R>::flux(d, Wf[2 * d], Uf[2 * d][4], Fm);
                    Scheme<R>::flux(d, Wf[2 * d + 1], Uf[2 * d + 1][4], Fp);
                    for (int q = 0; q < 5; ++q) acc[q] = acc[q] + (Fm[q] - Fp[q]);
                }
                R* Uo = &Uh[qidx(i, j, k) * 30];
                bool ok = true;
                for (int f = 0; f < 6; ++f) {
                    for (int q = 0; q < 5; ++q) Uo[f * 5 + q] = Uf[f][q] + half_lam * acc[q];
                    if (!S.positive(&Uo[f * 5])) ok = false;
                }
                if (!ok) {  // READING R4
                    st |= ORACLE_ST_PREDICTOR_FALLBACK;
                    for (int f = 0; f < 6; ++f)
                        for (int q = 0; q < 5; ++q)
                            Uo[f * 5 + q] = (S.pred_fallback == 0) ? Uc[q] : Uf[f][q];
                }
            }

    // Stage 3: Roe fluxes on every face touching the updated cells.
    // Face index f in direction d sits between cells f-1 and f.
    std::vector<R> Fx((std::size_t)nz * ny * (nx + 1) * 5);
    std::vector<R> Fy((std::size_t)nz * (ny + 1) * nx * 5);
    std::vector<R> Fz((std::size_t)(nz + 1) * ny * nx * 5);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int f = 0; f <= nx; ++f) {
                const R* L = &Uh[qidx(f - 1, j, k) * 30 + 1 * 5];  // x+ face of left cell
                const R* Rr = &Uh[qidx(f, j, k) * 30 + 0 * 5];     // x- face of right cell
                if (S.riemann(0, L, Rr, &Fx[(((std::size_t)k * ny + j) * (nx + 1) + f) * 5]))
                    st |= ORACLE_ST_HLLE_FALLBACK;
            }
    for (int k = 0; k < nz; ++k)
        for (int f = 0; f <= ny; ++f)
            for (int i = 0; i < nx; ++i) {
                const R* L = &Uh[qidx(i, f - 1, k) * 30 + 3 * 5];
                const R* Rr = &Uh[qidx(i, f, k) * 30 + 2 * 5];
                if (S.riemann(1, L, Rr, &Fy[(((std::size_t)k * (ny + 1) + f) * nx + i) * 5]))
                    st |= ORACLE_ST_HLLE_FALLBACK;
            }
    for (int f = 0; f <= nz; ++f)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const R* L = &Uh[qidx(i, j, f - 1) * 30 + 5 * 5];
                const R* Rr = &Uh[qidx(i, j, f) * 30 + 4 * 5];
                if (S.riemann(2, L, Rr, &Fz[(((std::size_t)f * ny + j) * nx + i) * 5]))
                    st |= ORACLE_ST_HLLE_FALLBACK;
            }
    auto FX = [&](int f, int j, int k) { return &Fx[(((std::size_t)k * ny + j) * (nx + 1) + f) * 5]; };
    auto FY = [&](int i, int f, int k) { return &Fy[(((std::size_t)k * (ny + 1) + f) * nx + i) * 5]; };
    auto FZ = [&](int i, int j, int f) { return &Fz[(((std::size_t)f * ny + j) * nx + i) * 5]; };

    // Stage 4: full-step conservative update, directions summed x, y, z.
    const std::size_t ocells = (std::size_t)nx * ny * nz;
    R maxs = R(0.0);
    R sums[5] = {R(0.0), R(0.0), R(0.0), R(0.0), R(0.0)};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                R U[5], Un[5];
                U_in(i, j, k, U);
                for (int q = 0; q < 5; ++q) {
                    R acc = FX(i + 1, j, k)[q] - FX(i, j, k)[q];
                    acc = acc + (FY(i, j + 1, k)[q] - FY(i, j, k)[q]);
                    acc = acc + (FZ(i, j, k + 1)[q] - FZ(i, j, k)[q]);
                    Un[q] = U[q] - lam * acc;
                }
                // Optional floors on the updated state: density first (momentum
                // kept), then pressure, by setting the total energy to the kinetic
                // energy plus max(p_floor / (gamma - 1), 4 eps ke) where rho > 0 and
                // p < p_floor (eps = 2^-52: the thermal part stays resolvable next
                // to the kinetic energy, so the stored state keeps p > 0).
                if (S.rho_floor > R(0.0) && Un[0] < S.rho_floor) {
                    Un[0] = S.rho_floor;
                    st |= ORACLE_ST_FLOOR;
                }
                if (S.p_floor > R(0.0) && Un[0] > R(0.0)) {
                    const R ke = R(0.5) * (Un[1] * Un[1] + Un[2] * Un[2] + Un[3] * Un[3]) / Un[0];
                    if (S.gm1 * (Un[4] - ke) < S.p_floor) {
                        const R eth = S.p_floor / S.gm1, res = R(4.0 * 2.220446049250313e-16) * ke;
                        Un[4] = ke + (eth > res ? eth : res);
                        st |= ORACLE_ST_FLOOR;
                    }
                }
                for (int q = 0; q < 5; ++q) out[q * ocells + ((std::size_t)k * ny + j) * nx + i] = Un[q];
                // epilogue: positivity flag and the time-step / conservation partials
                R Wn[5];
                S.prim(Un, Wn);
                if (!(Wn[0] > R(0.0)) || !(Wn[4] > R(0.0))) st |= ORACLE_ST_NONPOSITIVE_OUT;
                R c2 = S.gamma * Wn[4] / Wn[0];
                R c = (c2 > R(0.0)) ? r_sqrt(c2) : R(0.0);
                R s = r_max(r_max(r_abs(Wn[1]), r_abs(Wn[2])), r_abs(Wn[3])) + c;
                if (s > maxs) maxs = s;
                for (int q = 0; q < 5; ++q) sums[q] = sums[q] + Un[q];
            }

    // Coarse-fine face fluxes: raw flux on the six box faces, or on nine planes
    // (per direction at 0, n/2 and n cells: the faces and the patch boundary).
    if (ff && S.flux_layout == 1) {
        R* p = ff;
        for (int f : {0, nx / 2, nx})  // x planes : [v][k][j]
            for (int q = 0; q < 5; ++q)
                for (int k = 0; k < nz; ++k)
                    for (int j = 0; j < ny; ++j) *p++ = FX(f, j, k)[q];
        for (int f : {0, ny / 2, ny})  // y planes : [v][k][i]
            for (int q = 0; q < 5; ++q)
                for (int k = 0; k < nz; ++k)
                    for (int i = 0; i < nx; ++i) *p++ = FY(i, f, k)[q];
        for (int f : {0, nz / 2, nz})  // z planes : [v][j][i]
            for (int q = 0; q < 5; ++q)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) *p++ = FZ(i, j, f)[q];
    } else if (ff) {
        R* p = ff;
        for (int side = 0; side < 2; ++side) {  // -x, +x : [v][k][j]
            const int f = side ? nx : 0;
            for (int q = 0; q < 5; ++q)
                for (int k = 0; k < nz; ++k)
                    for (int j = 0; j < ny; ++j) *p++ = FX(f, j, k)[q];
        }
        for (int side = 0; side < 2; ++side) {  // -y, +y : [v][k][i]
            const int f = side ? ny : 0;
            for (int q = 0; q < 5; ++q)
                for (int k = 0; k < nz; ++k)
                    for (int i = 0; i < nx; ++i) *p++ = FY(i, f, k)[q];
        }
        for (int side = 0; side < 2; ++side) {  // -z, +z : [v][j][i]
            const int f = side ? nz : 0;
            for (int q = 0; q < 5; ++q)
                for (int j = 0; j < ny; ++j)
                    for (int i = 0; i < nx; ++i) *p++ = FZ(i, j, f)[q];
        }
    }
    if (partials) {
        partials[0] = maxs;
        for (int q = 0; q < 5; ++q) partials[1 + q] = sums[q];
    }
    if (status_out) *status_out = st;
    return 0;
}

template <class R>
Scheme<R> make_scheme(const oracle_params* p) {
    Scheme<R> S;
    S.gamma = R(p->gamma);
    S.gm1 = R(p->gamma - 1.0);
    S.limiter = p->limiter;
    S.pred_fallback = p->predictor_fallback;
    S.rho_floor = R(p->rho_floor);
    S.p_floor = R(p->p_floor);
    S.flux_layout = p->flux_layout;
    S.solver = p->riemann;
    S.recon = p->reconstruction;
    return S;
}

bool params_ok(const oracle_params* p) {
    return p && std::isfinite(p->gamma) && p->gamma > 1.0 && p->limiter >= 0 && p->limiter <= 2 &&
           (p->predictor_fallback == 0 || p->predictor_fallback == 1) &&
           std::isfinite(p->rho_floor) && p->rho_floor >= 0.0 && std::isfinite(p->p_floor) &&
           p->p_floor >= 0.0 && (p->flux_layout == 0 || p->flux_layout == 1) &&
           (p->riemann == 0 || p->riemann == 1) &&
           (p->reconstruction == 0 || p->reconstruction == 1);
}

// ---------------------------------------------------------------------------
// Exact Riemann solver for the Euler equations (Toro 2009, ch. 4): pressure
// function f(p) = f_L(p) + f_R(p) + (u_R - u_L), Newton iteration from the
// primitive-variable guess.
struct ExactSide {
    double r, u, p, c;
};
void pressure_fn(double p, const ExactSide& s, double g, double* f, double* df) {
    if (p > s.p) {  // shock
        const double A = 2.0 / ((g + 1.0) * s.r);
        const double B = (g - 1.0) / (g + 1.0) * s.p;
        const double q = std::sqrt(A / (B + p));
        *f = (p - s.p) * q;
        *df = q * (1.0 - 0.5 * (p - s.p) / (B + p));
    } else {  // rarefaction
        const double pr = p / s.p;
        *f = 2.0 * s.c / (g - 1.0) * (std::pow(pr, (g - 1.0) / (2.0 * g)) - 1.0);
        *df = 1.0 / (s.r * s.c) * std::pow(pr, -(g + 1.0) / (2.0 * g));
    }
}

}  // namespace

// ===========================================================================
extern "C" {

int oracle_advance_box(const double* in, int nx, int ny, int nz, double* out, double* face_flux,
                       double dt, double dh, const oracle_params* p, uint32_t* status,
                       double* partials) {
    if (!in || !out || !params_ok(p) || nx < 1 || ny < 1 || nz < 1) return -1;
    if (p->flux_layout == 1 && ((nx | ny | nz) & 1)) return -1;
    Scheme<double> S = make_scheme<double>(p);
    return advance_box<double>(S, in, nx, ny, nz, out, face_flux, dt, dh, status, partials);
}

int oracle_advance_groups(const double* in, double* out, double* face_flux, const double* dt,
                          const double* dh, int64_t N, const oracle_params* p, uint32_t* status,
                          double* partials, int nthreads) {
    if (N < 0 || !params_ok(p)) return -1;
    if (N == 0) return 0;
    if (!in || !out || !dt || !dh) return -1;
    Scheme<double> S = make_scheme<double>(p);
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (int64_t g = 0; g < N; ++g) {
        advance_box<double>(S, in + g * 40000, 16, 16, 16, out + g * 20480,
                            face_flux ? face_flux + g * (p->flux_layout ? 11520 : 7680) : nullptr,
                            dt[g], dh[g],
                            status ? status + g : nullptr, partials ? partials + g * 6 : nullptr);
    }
    return 0;
}

int oracle_fill_ghosts_uniform(const double* level, int gx, int gy, int gz, int bc, double* in) {
    if (!level || !in || gx < 1 || gy < 1 || gz < 1 || (bc != 0 && bc != 1)) return -1;
    const int nxg = 16 * gx, nyg = 16 * gy, nzg = 16 * gz;
    auto wrap = [&](int X, int n) {
        if (bc == 0) return ((X % n) + n) % n;
        return X < 0 ? 0 : (X >= n ? n - 1 : X);
    };
    for (int bz = 0; bz < gz; ++bz)
        for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) {
                const std::size_t g = ((std::size_t)bz * gy + by) * gx + bx;
                double* dst = in + g * 40000;
                for (int v = 0; v < 5; ++v)
                    for (int k = -2; k < 18; ++k)
                        for (int j = -2; j < 18; ++j)
                            for (int i = -2; i < 18; ++i) {
                                const int X = wrap(bx * 16 + i, nxg);
                                const int Y = wrap(by * 16 + j, nyg);
                                const int Z = wrap(bz * 16 + k, nzg);
                                const std::size_t src =
                                    ((std::size_t)(Z / 16) * gy + (Y / 16)) * gx + (X / 16);
                                dst[((v * 20 + (k + 2)) * 20 + (j + 2)) * 20 + (i + 2)] =
                                    level[src * 20480 + ((v * 16 + Z % 16) * 16 + Y % 16) * 16 +
                                          X % 16];
                            }
            }
    return 0;
}

int oracle_hydro_dt(const double* partials, int64_t N, const int32_t* level, int32_t n_levels,
                    const double* dh_level, double cfl, double* dt_out, double* totals) {
    if (N < 0 || n_levels < 1 || !dh_level || !dt_out || (N > 0 && !partials)) return -1;
    std::vector<double> mx(n_levels, 0.0);
    double tot[5] = {0, 0, 0, 0, 0};
    for (int64_t g = 0; g < N; ++g) {
        const int l = level ? level[g] : 0;
        if (l < 0 || l >= n_levels) return -1;
        if (partials[g * 6] > mx[l]) mx[l] = partials[g * 6];
        for (int q = 0; q < 5; ++q) tot[q] += partials[g * 6 + 1 + q];
    }
    for (int l = 0; l < n_levels; ++l) dt_out[l] = (mx[l] > 0.0) ? cfl * dh_level[l] / mx[l] : 0.0;
    if (totals)
        for (int q = 0; q < 5; ++q) totals[q] = tot[q];
    return 0;
}

void oracle_prim_from_cons(const double U[5], double gamma, double W[5]) {
    oracle_params p = {gamma, 0, 0};
    make_scheme<double>(&p).prim(U, W);
}
void oracle_cons_from_prim(const double W[5], double gamma, double U[5]) {
    oracle_params p = {gamma, 0, 0};
    make_scheme<double>(&p).cons(W, U);
}
void oracle_euler_flux(int dir, const double W[5], double E, double F[5]) {
    Scheme<double>::flux(dir, W, E, F);
}
double oracle_limiter(int id, double a, double b) {
    oracle_params p = {1.4, id, 0};
    return make_scheme<double>(&p).limit(a, b);
}
int oracle_roe_flux(int dir, const double UL[5], const double UR[5], double gamma, int entropy_fix,
                    double F[5]) {
    oracle_params p = {gamma, 0, 0};
    return make_scheme<double>(&p).roe(dir, UL, UR, entropy_fix != 0, F) ? 1 : 0;
}
void oracle_char_slopes(int dir, const double Wl[5], const double Wc[5], const double Wr[5],
                        double gamma, int limiter, double slope[5]) {
    oracle_params p = {gamma, limiter, 0};
    Scheme<double> S = make_scheme<double>(&p);
    S.char_slopes(dir, Wl, Wc, Wr, slope);
}

void oracle_hllc_flux(int dir, const double UL[5], const double UR[5], double gamma, double F[5]) {
    oracle_params p = {gamma, 0, 0};
    p.riemann = 1;
    Scheme<double> S = make_scheme<double>(&p);
    S.hllc(dir, UL, UR, F);
}

void oracle_hlle_flux(int dir, const double UL[5], const double UR[5], double gamma, double F[5]) {
    oracle_params p = {gamma, 0, 0};
    Scheme<double> S = make_scheme<double>(&p);
    double WL[5], WR[5], FL[5], FR[5];
    S.prim(UL, WL);
    S.prim(UR, WR);
    Scheme<double>::flux(dir, WL, UL[4], FL);
    Scheme<double>::flux(dir, WR, UR[4], FR);
    const int n = 1 + dir;
    const double cL = std::sqrt(gamma * WL[4] / WL[0]), cR = std::sqrt(gamma * WR[4] / WR[0]);
    const double rr = std::sqrt(WR[0] / WL[0]);
    double q2 = 0.0, uT = 0.0;
    double vel[3];
    for (int a = 0; a < 3; ++a) {
        vel[a] = (WL[1 + a] + rr * WR[1 + a]) / (1.0 + rr);
        q2 += vel[a] * vel[a];
    }
    uT = vel[dir];
    const double HT = ((UL[4] + WL[4]) / WL[0] + rr * (UR[4] + WR[4]) / WR[0]) / (1.0 + rr);
    const double cT2 = (gamma - 1.0) * (HT - 0.5 * q2);
    const bool have = cT2 > 0.0;
    S.hlle(UL, UR, FL, FR, WL[n], cL, WR[n], cR, have, uT, have ? std::sqrt(cT2) : 0.0, F);
}

int oracle_exact_riemann_star(double rl, double ul, double pl, double rr, double ur, double pr,
                              double g, double star[4]) {
    const ExactSide L = {rl, ul, pl, std::sqrt(g * pl / rl)};
    const ExactSide R = {rr, ur, pr, std::sqrt(g * pr / rr)};
    if (2.0 / (g - 1.0) * (L.c + R.c) <= R.u - L.u) return -1;  // vacuum is generated
    double p = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (L.c + R.c);
    if (p < 1e-12) p = 1e-12;
    int it = 0;
    for (; it < 200; ++it) {
        double fl, dfl, fr, dfr;
        pressure_fn(p, L, g, &fl, &dfl);
        pressure_fn(p, R, g, &fr, &dfr);
        double pn = p - (fl + fr + (ur - ul)) / (dfl + dfr);
        if (pn < 1e-14) pn = 1e-14;
        const double change = 2.0 * std::fabs((pn - p) / (pn + p));
        p = pn;
        if (change < 1e-15) break;
    }
    double fl, dfl, fr, dfr;
    pressure_fn(p, L, g, &fl, &dfl);
    pressure_fn(p, R, g, &fr, &dfr);
    const double u = 0.5 * (ul + ur) + 0.5 * (fr - fl);
    const double g6 = (g - 1.0) / (g + 1.0);
    auto rho_star = [&](const ExactSide& s) {
        const double ratio = p / s.p;
        if (p > s.p) return s.r * (ratio + g6) / (g6 * ratio + 1.0);
        return s.r * std::pow(ratio, 1.0 / g);
    };
    star[0] = p;
    star[1] = u;
    star[2] = rho_star(L);
    star[3] = rho_star(R);
    return it + 1;
}

void oracle_exact_riemann_sample(double rl, double ul, double pl, double rr, double ur, double pr,
                                 double g, double xi, double W[3]) {
    double star[4];
    if (oracle_exact_riemann_star(rl, ul, pl, rr, ur, pr, g, star) < 0) {
        W[0] = W[1] = W[2] = NAN;
        return;
    }
    const double ps = star[0], us = star[1];
    const double g1 = (g - 1.0) / (2.0 * g), g2 = (g + 1.0) / (2.0 * g);
    // Sample on the side of the contact that xi falls on; the right side is
    // the mirror image of the left side (x -> -x, u -> -u).
    const bool left = xi <= us;
    const double sgn = left ? 1.0 : -1.0;
    const double r = left ? rl : rr, u = sgn * (left ? ul : ur), p = left ? pl : pr;
    const double x = sgn * xi, uss = sgn * us, rs = left ? star[2] : star[3];
    const double c = std::sqrt(g * p / r);
    double o_r, o_u, o_p;
    if (ps > p) {  // shock
        const double S = u - c * std::sqrt(g2 * ps / p + g1);
        if (x <= S) { o_r = r; o_u = u; o_p = p; }
        else { o_r = rs; o_u = uss; o_p = ps; }
    } else {  // rarefaction fan
        const double head = u - c;
        const double cs = c * std::pow(ps / p, g1);
        const double tail = uss - cs;
        if (x <= head) { o_r = r; o_u = u; o_p = p; }
        else if (x >= tail) { o_r = rs; o_u = uss; o_p = ps; }
        else {
            const double cf = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * (u - x));
            o_u = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * u + x);
            o_r = r * std::pow(cf / c, 2.0 / (g - 1.0));
            o_p = p * std::pow(cf / c, 2.0 * g / (g - 1.0));
        }
    }
    W[0] = o_r;
    W[1] = sgn * o_u;
    W[2] = o_p;
}

int oracle_count_ops_piece(int piece, int dir, const double* a, const double* b, double gamma,
                           double counts[5]) {
    if (!a || !counts || piece < 0 || piece > 5 || dir < 0 || dir > 2 ||
        !(std::isfinite(gamma) && gamma > 1.0))
        return -1;
    if ((piece == 2 || piece == 3 || piece == 4) && !b) return -1;
    oracle_params p = {};
    p.gamma = gamma;
    Scheme<Cnt> S = make_scheme<Cnt>(&p);
    Cnt A[5], B[5], R[5];
    for (int q = 0; q < 5; ++q) {
        A[q] = Cnt(a[q]);
        B[q] = Cnt(b ? b[q] : 0.0);
    }
    g_tally = Tally();
    switch (piece) {
        case 0: S.prim(A, R); break;
        case 1: S.cons(A, R); break;
        case 2: Scheme<Cnt>::flux(dir, A, B[0], R); break;
        case 3: R[0] = S.limit(A[0], B[0]); break;
        case 4: S.roe(dir, A, B, true, R); break;
        default: (void)S.positive(A); break;
    }
    counts[0] = g_tally.add;
    counts[1] = g_tally.mul;
    counts[2] = g_tally.div;
    counts[3] = g_tally.sqrt;
    counts[4] = g_tally.cmp;
    return 0;
}

int oracle_count_ops_group(const double* in, double dt, double dh, const oracle_params* p,
                           double counts[6]) {
    if (!in || !counts || !params_ok(p)) return -1;
    std::vector<Cnt> cin(40000), cout_(20480), cff(7680);
    for (int i = 0; i < 40000; ++i) cin[i] = Cnt(in[i]);
    Scheme<Cnt> S = make_scheme<Cnt>(p);
    Cnt partials[6];
    uint32_t st = 0;
    g_tally = Tally();
    advance_box<Cnt>(S, cin.data(), 16, 16, 16, cout_.data(), cff.data(), Cnt(dt), Cnt(dh), &st,
                     partials);
    counts[0] = g_tally.add;
    counts[1] = g_tally.mul;
    counts[2] = g_tally.div;
    counts[3] = g_tally.sqrt;
    counts[4] = g_tally.cmp;
    counts[5] = 4096.0;
    return 0;
}

}  // extern "C"

// ===========================================================================
// AMR coarse-fine coupling (the step after the hydro path): flux fix-up and
// restriction, written as plain loops over the records.
extern "C" {

int64_t oracle_flux_fixup(double* coarse, const double* coarse_flux, const double* fine_flux,
                          int n_sub, const double* dt, const double* dh, int64_t Nc, int64_t Nf,
                          const oracle_cf_face* faces, int64_t n) {
    if (n < 0 || Nc < 0 || Nf < 0 || n_sub < 1) return -1;
    if (n == 0) return 0;
    if (!coarse || !coarse_flux || !fine_flux || !dt || !dh || !faces) return -1;
    int64_t bad = 0;
    for (int cls = 0; cls < 6; ++cls) {
        for (int64_t r = 0; r < n; ++r) {
            const oracle_cf_face& F = faces[r];
            const bool ok = F.coarse >= 0 && F.coarse < Nc && F.fine >= 0 && F.fine < Nf &&
                            F.dir >= 0 && F.dir <= 2 && F.plane >= 0 && F.plane <= 2 &&
                            (F.side == 0 || F.side == 1) && F.quadrant >= 0 && F.quadrant <= 3 &&
                            !(F.side == 1 && F.plane == 0) && !(F.side == 0 && F.plane == 2);
            if (!ok) {
                if (cls == 0) ++bad;
                continue;
            }
            if (2 * F.dir + F.side != cls) continue;
            const double lam = dt[F.coarse] / dh[F.coarse];
            const int layer = F.side ? 8 * F.plane - 1 : 8 * F.plane;
            const int fface = 2 * F.dir + (F.side ? 0 : 1);  // the fine group's face
            const int a0 = (F.quadrant & 1) ? 8 : 0, b0 = (F.quadrant & 2) ? 8 : 0;
            const double* Fc = coarse_flux + ((std::size_t)F.coarse * 9 + 3 * F.dir + F.plane) * 1280;
            double* U = coarse + (std::size_t)F.coarse * 20480;
            for (int q = 0; q < 5; ++q)
                for (int a = a0; a < a0 + 8; ++a)
                    for (int b = b0; b < b0 + 8; ++b) {
                        double sum = 0.0;
                        for (int s = 0; s < n_sub; ++s) {
                            const double* Ff =
                                fine_flux + (((std::size_t)s * Nf + F.fine) * 6 + fface) * 1280 +
                                (std::size_t)q * 256;
                            for (int A = 2 * (a - a0); A < 2 * (a - a0) + 2; ++A)
                                for (int B = 2 * (b - b0); B < 2 * (b - b0) + 2; ++B)
                                    sum = sum + Ff[A * 16 + B];
                        }
                        const double mean = sum / double(4 * n_sub);
                        const double corr = lam * (Fc[q * 256 + a * 16 + b] - mean);
                        int i, j, k;
                        if (F.dir == 0) { k = a; j = b; i = layer; }
                        else if (F.dir == 1) { k = a; i = b; j = layer; }
                        else { j = a; i = b; k = layer; }
                        double& u = U[((q * 16 + k) * 16 + j) * 16 + i];
                        u = F.side ? u + corr : u - corr;
                    }
        }
    }
    return bad;
}

int64_t oracle_restrict(const double* fine, double* coarse, int64_t Nc, int64_t Nf,
                        const oracle_cf_child* children, int64_t n) {
    if (n < 0 || Nc < 0 || Nf < 0) return -1;
    if (n == 0) return 0;
    if (!fine || !coarse || !children) return -1;
    int64_t bad = 0;
    for (int64_t r = 0; r < n; ++r) {
        const oracle_cf_child& C = children[r];
        if (!(C.coarse >= 0 && C.coarse < Nc && C.fine >= 0 && C.fine < Nf && C.octant >= 0 &&
              C.octant <= 7)) {
            ++bad;
            continue;
        }
        const int ox = (C.octant & 1) ? 8 : 0, oy = (C.octant & 2) ? 8 : 0,
                  oz = (C.octant & 4) ? 8 : 0;
        const double* f = fine + (std::size_t)C.fine * 20480;
        double* c = coarse + (std::size_t)C.coarse * 20480;
        for (int q = 0; q < 5; ++q)
            for (int k = 0; k < 8; ++k)
                for (int j = 0; j < 8; ++j)
                    for (int i = 0; i < 8; ++i) {
                        double sum = 0.0;
                        for (int dk = 0; dk < 2; ++dk)
                            for (int dj = 0; dj < 2; ++dj)
                                for (int di = 0; di < 2; ++di)
                                    sum = sum + f[((q * 16 + 2 * k + dk) * 16 + 2 * j + dj) * 16 +
                                                  2 * i + di];
                        c[((q * 16 + oz + k) * 16 + oy + j) * 16 + ox + i] = sum * 0.125;
                    }
    }
    return bad;
}

}  // extern "C"
