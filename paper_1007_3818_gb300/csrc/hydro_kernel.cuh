// hydro_kernel.cuh -- the MUSCL-Hancock + Roe patch-group step for sm_103a.
//
// Paper Sec. 2: spatial data reconstruction, half-step prediction, Riemann
// solver (Roe), full-step update; unsplit; five-point stencil per direction.
// Scheme details (the readings the C ABI documents): primitive reconstruction
// with a van Leer / minmod / MC limiter, conservative Hancock half-step with a
// cell-average fallback, Roe flux with Harten's smoothing of |lambda| on the
// acoustic waves using Harten-Hyman widths from the Roe intermediate states,
// HLLE with Einfeldt speeds as fallback.
//
// GB300 design (one CTA of 160 threads per patch group, persistent over the
// batch):
//  * z-marching: the 20^3 input arrives one z-plane (5 x 20 x 20 values) at a
//    time through the TMA engine (cp.async.bulk, 5 x 1600 B per plane in FP32)
//    into a 2-slot shared ring; the copy of plane k+2 is issued as soon as
//    plane k has been read (after phase A) and lands while phase B runs.  Each
//    plane is converted once per cell into a 3-plane ring of primitives.
//  * per plane k: phase A predicts the 320 cells of the plane (16^2 interior +
//    4 x 16 face-slab cells), two per thread; phase B solves the 800 Riemann
//    problems of the plane (272 x-faces and 272 y-faces from shared memory,
//    256 z-faces from registers), exactly five per thread; phase C finishes
//    plane k-1 and converts plane k+2.
//  * each interior column (i,j) has an owner thread that keeps its z-face
//    state, z-flux and partial update in registers, so nothing of the z
//    direction goes through shared memory.  The two half-warps of a warp own
//    rows j and j+4, 80 floats apart in a 20-wide plane, so every plane access
//    of a warp hits 32 distinct banks; the 16-wide face and flux arrays store
//    row j at j ^ ((j >> 2) & 1) for the same reason.
//  * epilogue sums are compensated (TwoSum) per thread and reduced in FP64
//    across threads; FP32 modes issue no FP64 instruction per cell.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "gamer_gb300.h"

namespace gamer {

constexpr int kThreads = 160;
constexpr int kPlane = 400;       // 20 x 20 cells per input plane
constexpr int kFaceStride = 288;  // 16^2 interior, 16 slab entries, 16 write-only entries

template <int MODE> struct Prec;
template <> struct Prec<GAMER_MODE_F32> { using T = float; using P = float; };
template <> struct Prec<GAMER_MODE_MIXED> { using T = float; using P = double; };
template <> struct Prec<GAMER_MODE_F64> { using T = double; using P = double; };
template <> struct Prec<GAMER_MODE_FF> { using T = float; using P = float; };

// Error-free transformations for the float-float mode: Knuth's TwoSum and the
// rounding error of a product from one FMA.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
    return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
    const float p = a * b;
    e = fmaf(a, b, -p);
    return p;
}

// |m|^2 as a float-float pair s + se (the squares exact, their sums with
// TwoSum); accurate to about 2^-47 relative.
__device__ __forceinline__ float sq3_ff(float m1, float m2, float m3, float& se) {
    float e1, e2, e3, t1, t2;
    float s = two_prod(m1, m1, e1);
    s = two_sum(s, two_prod(m2, m2, e2), t1);
    s = two_sum(s, two_prod(m3, m3, e3), t2);
    se = ((e1 + e2) + e3) + (t1 + t2);
    return s;
}

// The same three on paired FP32 instructions (two independent lanes, each the
// same IEEE operations in the same order as the scalar forms above).
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2& e) {
    const float2 s = __fadd2_rn(a, b);
    const float2 bp = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bp)))), __fadd2_rn(b, neg2(bp)));
    return s;
}
__device__ __forceinline__ float2 two_prod2(float2 a, float2 b, float2& e) {
    const float2 p = __fmul2_rn(a, b);
    e = __ffma2_rn(a, b, neg2(p));
    return p;
}
__device__ __forceinline__ float2 sq3_ff2(float2 m1, float2 m2, float2 m3, float2& se) {
    float2 e1, e2, e3, t1, t2;
    float2 s = two_prod2(m1, m1, e1);
    s = two_sum2(s, two_prod2(m2, m2, e2), t1);
    s = two_sum2(s, two_prod2(m3, m3, e3), t2);
    se = __fadd2_rn(__fadd2_rn(__fadd2_rn(e1, e2), e3), __fadd2_rn(t1, t2));
    return s;
}

template <class T, int RING = 2>
struct alignas(16) Smem {
    T raw[RING][5 * kPlane + 4];  // ring of conserved input planes (TMA / cp.async)
    T W[3][5 * kPlane];    // primitive planes
    // face states of the x/y faces; after a face's Riemann solve, its flux
    // in both state slots the solve consumed (each slot feeds one solve), so
    // the owner of a cell finds F(i -/+ 1/2) in its own xm / xp slots (y
    // alike).  The group epilogue's per-warp partials reuse xm.
    T xm[5 * kFaceStride], xp[5 * kFaceStride], ym[5 * kFaceStride], yp[5 * kFaceStride];
    uint64_t mbar[RING];
    uint32_t status;
    T lam;  // dt / dh of the group being advanced (rounded once from FP64 by thread 0)
};

template <class T, class P>
struct KConst {
    T gamma, gm1;
    P gm1p;
    int limiter, pfb;
    int flux9;          // face-flux layout: 0 six group faces, 1 nine planes
    int floors;         // bit 0: density floor on, bit 1: pressure floor on
    T rho_floor, p_floor;
    P eth_floor;        // p_floor / (gamma - 1)
    T gm1_lo;           // gamma - 1 - gm1: the float-float mode's low part
};

// row slot of a 16-wide face array (see the bank note above)
__device__ __forceinline__ int frow(int j) { return j ^ ((j >> 2) & 1); }

// Face-flux plane of the face at cell index b in [0, 16] along direction dir
// (the face between cells b-1 and b), or -1 when the layout does not store it:
// six group faces (-x, +x, -y, +y, -z, +z) or nine planes (b = 0, 8, 16 per
// direction).
__device__ __forceinline__ int flux_plane(int dir, int b, int flux9) {
    if (flux9) return (b & 7) ? -1 : 3 * dir + (b >> 3);
    return (b == 0) ? 2 * dir : (b == 16) ? 2 * dir + 1 : -1;
}
constexpr int kFluxPlane = 5 * 256;  // one plane: [5][16][16]

// ---------------------------------------------------------------------------
// Selective FP64 in the mixed mode.  The pressure p = (gamma - 1)(E - ke),
// ke = |m|^2 / (2 rho), is recovered in FP32 as gm1 E - gm1 ke + gm1_lo (E -
// ke), with gamma - 1 held as the float pair (gm1, gm1_lo): the product with
// E is exact inside the final FMA, so E - ke is never rounded before it is
// scaled and no rounding bias of gamma - 1 enters.  Its relative error is
// about u + 8 u r / (1 - r), r = ke / E, u = 2^-24 (ke and gm1 ke carry some
// eight roundings, rcp.approx included, each magnified by ke / (E - ke)):
// below one ulp for small r, 9 u at r = 1/2, unbounded as E - ke cancels.
// Where the kinetic energy is more than half the total (r > 1/2: the flow is
// supersonic to within a factor of order one) p is recovered in FP64
// instead: 1/rho from the FP32 seed plus one Newton step, E - ke in FP64, one
// rounding.  In the Riemann solves and the half-step admissibility tests the
// FP32 path runs for every state and one rarely taken branch per solve or
// per predicted cell redoes it exactly when any of its states needs FP64.
constexpr float kMixedKeFraction = 0.5f;

static __device__ __noinline__ float pressure_fp64(float r, float m1, float m2, float m3, float E,
                                            float ir, double gm1p) {
    const double rd = r;
    double ird = ir;
    ird = fma(ird, fma(-rd, ird, 1.0), ird);
    const double a = m1, b = m2, c = m3;
    const double ke = 0.5 * (a * a + b * b + c * c) * ird;
    return static_cast<float>(gm1p * (static_cast<double>(E) - ke));
}

// rho > 0 and rho E - |m|^2 / 2 > 0 of six conserved states, the difference
// in FP64 (a predicted cell whose FP32 tests were not all certain)
struct States6 {
    float v[6][5];
};
static __device__ __noinline__ bool admissible6_fp64(States6 f) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const double a = f.v[i][1], b = f.v[i][2], c = f.v[i][3];
        ok &= (f.v[i][0] > 0.0f) &
              ((double(f.v[i][0]) * double(f.v[i][4]) - 0.5 * (a * a + b * b + c * c)) > 0.0);
    }
    return ok;
}

// the same in float-float (the FF mode): |m|^2 and rho E as exact pairs,
// their difference by TwoSum
static __device__ __noinline__ bool admissible6_ff(States6 f) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        float se, ee, t;
        const float s = sq3_ff(f.v[i][1], f.v[i][2], f.v[i][3], se);
        const float re = two_prod(f.v[i][0], f.v[i][4], ee);
        const float d = two_sum(re, -0.5f * s, t);
        ok &= (f.v[i][0] > 0.0f) & ((d + ((ee - 0.5f * se) + t)) > 0.0f);
    }
    return ok;
}

// The mixed mode's FP32 recovery from E and ke (see above).
__device__ __forceinline__ float p_mixed32(float E, float ke, float gm1, float gm1_lo) {
    return fmaf(gm1, E, fmaf(gm1_lo, E - ke, -(gm1 * ke)));
}

// The mixed mode's FP32 recovery of one state; hi is set where the state
// needs the FP64 recovery instead (ke > E / 2).
template <class P>
__device__ __forceinline__ float pressure_mixed32(float m1, float m2, float m3, float E, float ir,
                                                  const KConst<float, P>& kc, bool& hi) {
    const float ke = 0.5f * (m1 * m1 + m2 * m2 + m3 * m3) * ir;
    hi = ke > kMixedKeFraction * E;
    return p_mixed32(E, ke, kc.gm1, kc.gm1_lo);
}

// Pressure from a conserved state, given 1/rho in T.  MIXED: the selective
// recovery above.
template <int MODE, class T, class P>
__device__ __forceinline__ T pressure(T r, T m1, T m2, T m3, T E, T ir, const KConst<T, P>& kc) {
    if constexpr (MODE == GAMER_MODE_MIXED) {
        const float ke = 0.5f * (m1 * m1 + m2 * m2 + m3 * m3) * ir;
        if (ke > kMixedKeFraction * E) return pressure_fp64(r, m1, m2, m3, E, ir, kc.gm1p);
        return p_mixed32(E, ke, kc.gm1, kc.gm1_lo);
    } else if constexpr (MODE == GAMER_MODE_FF) {
        // the same recovery in float-float: 1/rho = ir (1 + d), d = 1 - rho ir
        // from one FMA; |m|^2 ir exactly as p + pe; E - ke by TwoSum
        float se;
        const float s = sq3_ff(m1, m2, m3, se);
        const float il = ir * fmaf(-r, ir, 1.0f);
        float pe;
        const float p = two_prod(s, ir, pe);
        const float kh = 0.5f * p, kl = 0.5f * (pe + fmaf(s, il, se * ir));
        float de;
        const float d = two_sum(E, -kh, de);
        const float dl = de - kl;
        // (gm1 + gm1_lo) (d + dl), rounded once
        const float ph = kc.gm1 * d;
        const float pl = fmaf(kc.gm1, d, -ph) + fmaf(kc.gm1, dl, kc.gm1_lo * d);
        return ph + pl;
    } else {
        return kc.gm1 * (E - T(0.5) * (m1 * m1 + m2 * m2 + m3 * m3) * ir);
    }
}

// Optional floors on an updated state (kc.floors != 0): a density below
// rho_floor is raised to it, momentum kept; then, where rho > 0 and
// p < p_floor, the total energy becomes ke + max(p_floor / (gamma - 1),
// 4 eps ke), ke = |m|^2 / (2 rho) and eps the storage type's machine epsilon:
// the thermal part is never below what E can resolve next to ke, so the
// stored state keeps p > 0 (MIXED evaluates ke in FP64).  ir = 1/rho and p
// are updated to the final state.
template <int MODE, class T, class P>
__device__ __forceinline__ void apply_floors(T o[5], T& ir, T& p, const KConst<T, P>& kc,
                                             uint32_t& st) {
    if ((kc.floors & 1) && o[0] < kc.rho_floor) {
        o[0] = kc.rho_floor;
        ir = rcp_(o[0]);
        p = pressure<MODE>(o[0], o[1], o[2], o[3], o[4], ir, kc);
        st |= GAMER_ST_FLOOR;
    }
    if ((kc.floors & 2) && o[0] > T(0) && p < kc.p_floor) {
        constexpr T kRes = T(4) * (sizeof(T) == 4 ? T(1.1920928955078125e-7)    // 2^-23
                                                   : T(2.220446049250313e-16));  // 2^-52
        if constexpr (MODE == GAMER_MODE_MIXED) {
            const double rd = o[0];
            double ird = ir;
            ird = fma(ird, fma(-rd, ird, 1.0), ird);
            const double a = o[1], b = o[2], c = o[3];
            const double ke = 0.5 * (a * a + b * b + c * c) * ird;
            o[4] = static_cast<T>(ke + fmax(kc.eth_floor, double(kRes) * ke));
        } else {
            const T ke = T(0.5) * (o[1] * o[1] + o[2] * o[2] + o[3] * o[3]) * ir;
            o[4] = ke + max_(kc.eth_floor, kRes * ke);
        }
        p = pressure<MODE>(o[0], o[1], o[2], o[3], o[4], ir, kc);
        st |= GAMER_ST_FLOOR;
    }
}

// rho > 0 and p > 0, tested as rho > 0 and rho E - |m|^2 / 2 > 0 (no division).
// MIXED takes the decision of the FP64 difference: the FP32 difference d
// carries an error below 4 u (|rho E| + |m|^2 / 2), so where |d| exceeds
// 2^-20 (|rho E| + |m|^2 / 2) its sign is the FP64 sign; only the cases
// closer to zero are decided in FP64.
// MIXED and FF take the FP32 decision where its sign is certain and raise
// `und` elsewhere; the caller then decides those cells exactly
// (admissible6_exact: FP64, or float-float in FF).
template <int MODE, class T>
__device__ __forceinline__ bool admissible(T r, T m1, T m2, T m3, T E, bool& und) {
    if constexpr (MODE == GAMER_MODE_MIXED || MODE == GAMER_MODE_FF) {
        const float h = 0.5f * (m1 * m1 + m2 * m2 + m3 * m3);
        const float re = r * E;
        const float d = re - h;
        und |= !(fabsf(d) > 0x1p-20f * (fabsf(re) + h));
        return (r > 0.0f) & (d > 0.0f);
    } else {
        return (r > T(0)) & ((r * E - T(0.5) * (m1 * m1 + m2 * m2 + m3 * m3)) > T(0));
    }
}

// LIM >= 0 fixes the limiter at compile time (no branch per slope); LIM < 0
// reads it from kc.limiter.
template <int LIM = -1, class T, class P>
__device__ __forceinline__ T limit(T a, T b, const KConst<T, P>& kc) {
    const T ab = a * b;
    const int lim = (LIM >= 0) ? LIM : kc.limiter;
    T r;
    if (lim == 1) {
        r = (a > T(0)) ? min_(a, b) : max_(a, b);
    } else if (lim == 2) {
        T m = min_(T(2) * abs_(a), T(2) * abs_(b));
        m = min_(m, T(0.5) * abs_(a + b));
        r = (a > T(0)) ? m : -m;
    } else {
        r = (T(2) * ab) * rcp_(a + b);
    }
    return (ab > T(0)) ? r : T(0);
}

// ---------------------------------------------------------------------------
// HLLE flux (rotated frame) with Einfeldt speed bounds.
template <class T>
__device__ __forceinline__ void hlle_rot(const T L[5], const T R[5], const T FL[5],
                                         const T FR[5], T sl, T sr, T F[5]) {
    const T bm = min_(sl, T(0));
    const T bp = max_(sr, T(0));
    const T inv = rcp_(bp - bm);
#pragma unroll
    for (int i = 0; i < 5; ++i) F[i] = (bp * FL[i] - bm * FR[i] + bp * bm * (R[i] - L[i])) * inv;
}

// Roe flux through a face whose normal is the first velocity component of the
// rotated states L, R = (rho, m_n, m_t1, m_t2, E), with Harten's smoothing of
// the acoustic eigenvalues and Harten-Hyman widths from the states beside each
// acoustic wave.  Branch-free (in FP64 but for the entropy-fix smoothing,
// see below): returns true when the HLLE fallback must
// replace F (Roe sound speed squared not positive, or an intermediate state
// with rho <= 0 or p <= 0; F is then meaningless).  Having no branch, the
// whole solve is one block of instructions the scheduler can interleave.
template <int MODE, class T, class P>
__device__ __forceinline__ bool roe_main(const T L[5], const T R[5], const KConst<T, P>& kc,
                                         T F[5]) {
    const T irL = rcp_(L[0]), irR = rcp_(R[0]);
    const T uL = L[1] * irL, vL = L[2] * irL, wL = L[3] * irL;
    const T uR = R[1] * irR, vR = R[2] * irR, wR = R[3] * irR;
    const T pL = pressure<MODE>(L[0], L[1], L[2], L[3], L[4], irL, kc);
    const T pR = pressure<MODE>(R[0], R[1], R[2], R[3], R[4], irR, kc);
    const T mL = L[1], mR = R[1];
    const T cL = sqrt_(kc.gamma * pL * irL);
    const T cR = sqrt_(kc.gamma * pR * irR);
    const T HL = (L[4] + pL) * irL;
    const T HR = (R[4] + pR) * irR;
    const T rr = sqrt_(R[0] * irL);
    const T i1 = rcp_(T(1) + rr);
    const T uT = (uL + rr * uR) * i1;
    const T vT = (vL + rr * vR) * i1;
    const T wT = (wL + rr * wR) * i1;
    const T HT = (HL + rr * HR) * i1;
    const T q2 = uT * uT + vT * vT + wT * wT;
    const T cT2 = kc.gm1 * (HT - T(0.5) * q2);
    const T cT = sqrt_(cT2);
    const T rT = rr * L[0];
    const T dr = R[0] - L[0], du = uR - uL, dv = vR - vL, dw = wR - wL, dp = pR - pL;
    const T ic2 = rcp_(cT2);
    const T a1 = (dp - rT * cT * du) * (T(0.5) * ic2);
    const T a2 = dr - dp * ic2;
    const T a3 = rT * dv;
    const T a4 = rT * dw;
    const T a5 = (dp + rT * cT * du) * (T(0.5) * ic2);
    const T K1u = uT - cT, K5u = uT + cT;
    const T K1E = HT - uT * cT, K5E = HT + uT * cT;
    const T s1r = L[0] + a1, s1n = L[1] + a1 * K1u, s1a = L[2] + a1 * vT, s1b = L[3] + a1 * wT,
            s1E = L[4] + a1 * K1E;
    const T s4r = R[0] - a5, s4n = R[1] - a5 * K5u, s4a = R[2] - a5 * vT, s4b = R[3] - a5 * wT,
            s4E = R[4] - a5 * K5E;
    const T is1 = rcp_(s1r), is4 = rcp_(s4r);
    const T p1 = pressure<MODE>(s1r, s1n, s1a, s1b, s1E, is1, kc);
    const T p4 = pressure<MODE>(s4r, s4n, s4a, s4b, s4E, is4, kc);
    const bool fallback =
        !((cT2 > T(0)) & (s1r > T(0)) & (p1 > T(0)) & (s4r > T(0)) & (p4 > T(0)));
    const T l1s = s1n * is1 - sqrt_(kc.gamma * p1 * is1);
    const T l5s = s4n * is4 + sqrt_(kc.gamma * p4 * is4);
    const T d1 = max_(T(0), max_(K1u - (uL - cL), l1s - K1u));
    const T d5 = max_(T(0), max_(K5u - l5s, (uR + cR) - K5u));
    T e1 = abs_(K1u), e5 = abs_(K5u);
    if constexpr (sizeof(T) == 8) {
        // FP64: the smoothing is rarely selected and its IEEE divisions are
        // costly on the FP64 pipe, so it is evaluated only where selected
        // (the same values)
        if (e1 < d1) e1 = (K1u * K1u + d1 * d1) * rcp_(T(2) * d1);
        if (e5 < d5) e5 = (K5u * K5u + d5 * d5) * rcp_(T(2) * d5);
    } else {
        const T f1 = (K1u * K1u + d1 * d1) * rcp_(T(2) * d1);
        const T f5 = (K5u * K5u + d5 * d5) * rcp_(T(2) * d5);
        e1 = (e1 < d1) ? f1 : e1;
        e5 = (e5 < d5) ? f5 : e5;
    }
    const T e2 = abs_(uT);
    const T s1 = e1 * a1, s2 = e2 * a2, s3 = e2 * a3, s4 = e2 * a4, s5 = e5 * a5;
    const T D0 = s1 + s2 + s5;
    const T D1 = s1 * K1u + s2 * uT + s5 * K5u;
    const T D2 = D0 * vT + s3;
    const T D3 = D0 * wT + s4;
    const T D4 = s1 * K1E + s2 * (T(0.5) * q2) + s3 * vT + s4 * wT + s5 * K5E;
    F[0] = T(0.5) * (mL + mR) - T(0.5) * D0;
    F[1] = T(0.5) * ((mL * uL + pL) + (mR * uR + pR)) - T(0.5) * D1;
    F[2] = T(0.5) * (mL * vL + mR * vR) - T(0.5) * D2;
    F[3] = T(0.5) * (mL * wL + mR * wR) - T(0.5) * D3;
    F[4] = T(0.5) * ((L[4] + pL) * uL + (R[4] + pR) * uR) - T(0.5) * D4;
    return fallback;
}

// The HLLE fallback recomputed from the two states alone (rare path, one
// out-of-line copy): Einfeldt speeds with the Roe speeds when c~^2 > 0,
// Davis's bounds over both states otherwise.
template <class T>
struct RoeIO {
    T v[5];
    uint32_t st;
};
// Roe solve of the FP32-storage modes with the left/right-symmetric work on
// paired FP32 instructions (one instruction, both lanes of a float2: .x the
// left state, .y the right).  Same formulas as roe_main; the FP32 mode also
// pairs its pressure recoveries, the mixed and float-float modes recover each
// lane's pressure in their own precision.
__device__ __forceinline__ float2 pk(float a, float b) { return make_float2(a, b); }
template <int MODE, class P>
__device__ __forceinline__ float2 pressure_x2(float2 r, float2 m, float2 ma, float2 mb, float2 E,
                                              float2 ir, const KConst<float, P>& kc, bool& hi) {
    if constexpr (MODE == GAMER_MODE_F32) {
        float2 s = __fmul2_rn(m, m);
        s = __ffma2_rn(ma, ma, s);
        s = __ffma2_rn(mb, mb, s);
        return __fmul2_rn(pk(kc.gm1, kc.gm1), __ffma2_rn(__fmul2_rn(s, ir), pk(-0.5f, -0.5f), E));
    } else if constexpr (MODE == GAMER_MODE_MIXED) {
        // the FP32 recovery of both lanes; hi marks a lane that needs FP64
        float2 s = __fmul2_rn(m, m);
        s = __ffma2_rn(ma, ma, s);
        s = __ffma2_rn(mb, mb, s);
        const float2 k2 = __fmul2_rn(s, ir);  // 2 ke
        const float2 ke = __fmul2_rn(k2, pk(0.5f, 0.5f));
        // ke > E / 2 as 2 ke > E (both sides scaled by 2 exactly)
        static_assert(kMixedKeFraction == 0.5f, "the test below assumes 1/2");
        hi |= (k2.x > E.x) | (k2.y > E.y);
        const float2 gk = __fmul2_rn(pk(kc.gm1, kc.gm1), ke);
        const float2 t = __ffma2_rn(pk(kc.gm1_lo, kc.gm1_lo), __fadd2_rn(E, pk(-ke.x, -ke.y)),
                                    pk(-gk.x, -gk.y));
        return __ffma2_rn(pk(kc.gm1, kc.gm1), E, t);
    } else if constexpr (MODE == GAMER_MODE_FF) {
        // the float-float recovery of pressure<FF>, both lanes at once
        float2 se;
        const float2 s = sq3_ff2(m, ma, mb, se);
        const float2 il = __fmul2_rn(ir, __ffma2_rn(neg2(r), ir, pk(1.0f, 1.0f)));
        float2 pe;
        const float2 p = two_prod2(s, ir, pe);
        const float2 half = pk(0.5f, 0.5f);
        const float2 kh = __fmul2_rn(half, p);
        const float2 kl = __fmul2_rn(half, __fadd2_rn(pe, __ffma2_rn(s, il, __fmul2_rn(se, ir))));
        float2 de;
        const float2 d = two_sum2(E, neg2(kh), de);
        const float2 dl = __fadd2_rn(de, neg2(kl));
        const float2 g = pk(kc.gm1, kc.gm1);
        const float2 ph = __fmul2_rn(g, d);
        const float2 pl = __fadd2_rn(__ffma2_rn(g, d, neg2(ph)),
                                     __ffma2_rn(g, dl, __fmul2_rn(pk(kc.gm1_lo, kc.gm1_lo), d)));
        return __fadd2_rn(ph, pl);
    } else {
        return pk(pressure<MODE>(r.x, m.x, ma.x, mb.x, E.x, ir.x, kc),
                  pressure<MODE>(r.y, m.y, ma.y, mb.y, E.y, ir.y, kc));
    }
}
template <int MODE, class P>
__device__ __forceinline__ bool roe_main_x2(const float L[5], const float R[5],
                                            const KConst<float, P>& kc, float F[5]) {
    const float2 r = pk(L[0], R[0]), m = pk(L[1], R[1]), ma = pk(L[2], R[2]),
                 mb = pk(L[3], R[3]), E = pk(L[4], R[4]);
    const float2 ir = pk(rcp_(L[0]), rcp_(R[0]));
    const float2 u = __fmul2_rn(m, ir), v = __fmul2_rn(ma, ir), w = __fmul2_rn(mb, ir);
    const float2 ga2 = pk(kc.gamma, kc.gamma);
    bool hi = false;  // MIXED: a state needs the FP64 recovery
    const float2 p = pressure_x2<MODE>(r, m, ma, mb, E, ir, kc, hi);
    const float2 Ep = __fadd2_rn(E, p);
    const float2 H = __fmul2_rn(Ep, ir);
    const float2 c2 = __fmul2_rn(__fmul2_rn(ga2, p), ir);
    const float cL = sqrt_(c2.x), cR = sqrt_(c2.y);
    const float rr = sqrt_(R[0] * ir.x);
    const float i1 = rcp_(1.0f + rr);
    const float uT = (u.x + rr * u.y) * i1;
    const float vT = (v.x + rr * v.y) * i1;
    const float wT = (w.x + rr * w.y) * i1;
    const float HT = (H.x + rr * H.y) * i1;
    const float q2 = uT * uT + vT * vT + wT * wT;
    const float cT2 = kc.gm1 * (HT - 0.5f * q2);
    const float cT = sqrt_(cT2);
    const float rT = rr * L[0];
    const float dr = R[0] - L[0], du = u.y - u.x, dv = v.y - v.x, dw = w.y - w.x, dp = p.y - p.x;
    const float ic2 = rcp_(cT2);
    const float a1 = (dp - rT * cT * du) * (0.5f * ic2);
    const float a2 = dr - dp * ic2;
    const float a3 = rT * dv;
    const float a4 = rT * dw;
    const float a5 = (dp + rT * cT * du) * (0.5f * ic2);
    const float K1u = uT - cT, K5u = uT + cT;
    const float K1E = HT - uT * cT, K5E = HT + uT * cT;
    // intermediate states U*_L = U_L + a1 K1 (.x), U*_R = U_R - a5 K5 (.y)
    const float2 A = pk(a1, -a5);
    const float2 sr = __fadd2_rn(r, A);
    const float2 sn = __ffma2_rn(A, pk(K1u, K5u), m);
    const float2 sa = __ffma2_rn(A, pk(vT, vT), ma);
    const float2 sb = __ffma2_rn(A, pk(wT, wT), mb);
    const float2 sE = __ffma2_rn(A, pk(K1E, K5E), E);
    const float2 is = pk(rcp_(sr.x), rcp_(sr.y));
    const float2 ps = pressure_x2<MODE>(sr, sn, sa, sb, sE, is, kc, hi);
    const bool fallback =
        !((cT2 > 0.0f) & (sr.x > 0.0f) & (ps.x > 0.0f) & (sr.y > 0.0f) & (ps.y > 0.0f)) | hi;
    const float2 un = __fmul2_rn(sn, is);
    const float2 cs2 = __fmul2_rn(__fmul2_rn(ga2, ps), is);
    const float l1s = un.x - sqrt_(cs2.x);
    const float l5s = un.y + sqrt_(cs2.y);
    const float d1 = max_(0.0f, max_(K1u - (u.x - cL), l1s - K1u));
    const float d5 = max_(0.0f, max_(K5u - l5s, (u.y + cR) - K5u));
    float e1 = abs_(K1u), e5 = abs_(K5u);
    const float f1 = (K1u * K1u + d1 * d1) * rcp_(2.0f * d1);
    const float f5 = (K5u * K5u + d5 * d5) * rcp_(2.0f * d5);
    e1 = (e1 < d1) ? f1 : e1;
    e5 = (e5 < d5) ? f5 : e5;
    const float e2 = abs_(uT);
    const float s1 = e1 * a1, s2 = e2 * a2, s3 = e2 * a3, s4 = e2 * a4, s5 = e5 * a5;
    const float D0 = s1 + s2 + s5;
    const float D1 = s1 * K1u + s2 * uT + s5 * K5u;
    const float D2 = D0 * vT + s3;
    const float D3 = D0 * wT + s4;
    const float D4 = s1 * K1E + s2 * (0.5f * q2) + s3 * vT + s4 * wT + s5 * K5E;
    const float2 f1n = __ffma2_rn(m, u, p), f2n = __fmul2_rn(m, v), f3n = __fmul2_rn(m, w),
                 f4n = __fmul2_rn(Ep, u);
    F[0] = 0.5f * (m.x + m.y) - 0.5f * D0;
    F[1] = 0.5f * (f1n.x + f1n.y) - 0.5f * D1;
    F[2] = 0.5f * (f2n.x + f2n.y) - 0.5f * D2;
    F[3] = 0.5f * (f3n.x + f3n.y) - 0.5f * D3;
    F[4] = 0.5f * (f4n.x + f4n.y) - 0.5f * D4;
    return fallback;
}

template <int MODE, class T, class P>
__device__ __forceinline__ void hlle_core(const T L[5], const T R[5], const KConst<T, P>& kc,
                                          T F[5]) {
    const T irL = rcp_(L[0]), irR = rcp_(R[0]);
    const T uL = L[1] * irL, vL = L[2] * irL, wL = L[3] * irL;
    const T uR = R[1] * irR, vR = R[2] * irR, wR = R[3] * irR;
    const T pL = pressure<MODE>(L[0], L[1], L[2], L[3], L[4], irL, kc);
    const T pR = pressure<MODE>(R[0], R[1], R[2], R[3], R[4], irR, kc);
    T FL[5], FR[5];
    const T mL = L[1], mR = R[1];
    FL[0] = mL; FL[1] = mL * uL + pL; FL[2] = mL * vL; FL[3] = mL * wL; FL[4] = (L[4] + pL) * uL;
    FR[0] = mR; FR[1] = mR * uR + pR; FR[2] = mR * vR; FR[3] = mR * wR; FR[4] = (R[4] + pR) * uR;
    const T cL = sqrt_(kc.gamma * pL * irL);
    const T cR = sqrt_(kc.gamma * pR * irR);
    const T rr = sqrt_(R[0] * irL);
    const T i1 = rcp_(T(1) + rr);
    const T uT = (uL + rr * uR) * i1, vT = (vL + rr * vR) * i1, wT = (wL + rr * wR) * i1;
    const T HT = ((L[4] + pL) * irL + rr * ((R[4] + pR) * irR)) * i1;
    const T cT2 = kc.gm1 * (HT - T(0.5) * (uT * uT + vT * vT + wT * wT));
    T sl = uL - cL, sr = uR + cR;
    if (cT2 > T(0)) {
        const T cT = sqrt_(cT2);
        sl = min_(sl, uT - cT);
        sr = max_(sr, uT + cT);
    } else {  // Davis's bounds over both states (S_L < S_R)
        sl = min_(sl, uR - cR);
        sr = max_(sr, uL + cL);
    }
    hlle_rot(L, R, FL, FR, sl, sr, F);
}
template <int MODE, class T, class P>
__device__ __noinline__ RoeIO<T> hlle_full(RoeIO<T> Li, RoeIO<T> Ri, KConst<T, P> kc) {
    RoeIO<T> out;
    hlle_core<MODE>(Li.v, Ri.v, kc, out.v);
    out.st = GAMER_ST_HLLE_FALLBACK;
    return out;
}

template <int MODE, class T, class P>
__device__ __forceinline__ void hlle_apply(const T L[5], const T R[5], const KConst<T, P>& kc,
                                           T F[5], uint32_t& st) {
    RoeIO<T> a, b;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        a.v[q] = L[q];
        b.v[q] = R[q];
    }
    a.st = b.st = 0;
    const RoeIO<T> r = hlle_full<MODE>(a, b, kc);
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = r.v[q];
    st |= r.st;
}

// Roe flux with its HLLE fallback (sets GAMER_ST_HLLE_FALLBACK in st when
// used): the branch-free solve, then one rarely taken branch into the single
// out-of-line HLLE copy (measured faster than an inline fallback per call
// site, which adds spills).
// MIXED: the Roe flux of a face whose FP32 solve could not stand -- a state
// needs the FP64 pressure recovery, or the HLLE fallback applies -- redone
// with the selective scalar recovery (one out-of-line copy, rarely run).
template <int MODE, class T, class P>
__device__ __noinline__ RoeIO<T> roe_exact(RoeIO<T> Li, RoeIO<T> Ri, KConst<T, P> kc) {
    RoeIO<T> out;
    out.st = 0;
    if (roe_main<MODE>(Li.v, Ri.v, kc, out.v)) {
        hlle_core<MODE>(Li.v, Ri.v, kc, out.v);
        out.st = GAMER_ST_HLLE_FALLBACK;
    }
    return out;
}

template <int MODE, class T, class P>
__device__ __forceinline__ void roe_rot(const T L[5], const T R[5], const KConst<T, P>& kc,
                                        T F[5], uint32_t& st) {
    bool fb;
    if constexpr (sizeof(T) == 4) fb = roe_main_x2<MODE>(L, R, kc, F);  // FP32 storage
    else fb = roe_main<MODE>(L, R, kc, F);
    if (fb) {
        if constexpr (MODE == GAMER_MODE_MIXED) {
            RoeIO<T> a, b;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                a.v[q] = L[q];
                b.v[q] = R[q];
            }
            a.st = b.st = 0;
            const RoeIO<T> r = roe_exact<MODE>(a, b, kc);
#pragma unroll
            for (int q = 0; q < 5; ++q) F[q] = r.v[q];
            st |= r.st;
        } else {
            hlle_apply<MODE>(L, R, kc, F, st);
        }
    }
}

// Out-of-line form of roe_rot (one copy of the solver in the kernel's code):
// states and flux travel by value, the status bits come back in the result.
template <int MODE, class T, class P>
__device__ __noinline__ RoeIO<T> roe_call(RoeIO<T> L, RoeIO<T> R, KConst<T, P> kc) {
    RoeIO<T> out;
    out.st = 0;
    roe_rot<MODE>(L.v, R.v, kc, out.v, out.st);
    return out;
}

// HLLC flux (Toro 2009, Sec. 10.4) in the rotated frame, with the wave-speed
// bounds of the HLLE fallback: Einfeldt's (u_L - c_L, u~ - c~ / u_R + c_R,
// u~ + c~) when c~^2 > 0, Davis's over both states otherwise.  The contact
// speed S* from the two momentum balances; the star state of the side that
// holds the face.  Never falls back.
template <int MODE, class T, class P>
__device__ __forceinline__ void hllc_rot(const T L[5], const T R[5], const KConst<T, P>& kc,
                                         T F[5]) {
    const T irL = rcp_(L[0]), irR = rcp_(R[0]);
    const T uL = L[1] * irL, vL = L[2] * irL, wL = L[3] * irL;
    const T uR = R[1] * irR, vR = R[2] * irR, wR = R[3] * irR;
    const T pL = pressure<MODE>(L[0], L[1], L[2], L[3], L[4], irL, kc);
    const T pR = pressure<MODE>(R[0], R[1], R[2], R[3], R[4], irR, kc);
    const T cL = sqrt_(kc.gamma * pL * irL);
    const T cR = sqrt_(kc.gamma * pR * irR);
    const T rr = sqrt_(R[0] * irL);
    const T i1 = rcp_(T(1) + rr);
    const T uT = (uL + rr * uR) * i1, vT = (vL + rr * vR) * i1, wT = (wL + rr * wR) * i1;
    const T HT = ((L[4] + pL) * irL + rr * ((R[4] + pR) * irR)) * i1;
    const T cT2 = kc.gm1 * (HT - T(0.5) * (uT * uT + vT * vT + wT * wT));
    T sl = uL - cL, sr = uR + cR;
    if (cT2 > T(0)) {
        const T cT = sqrt_(cT2);
        sl = min_(sl, uT - cT);
        sr = max_(sr, uT + cT);
    } else {
        sl = min_(sl, uR - cR);
        sr = max_(sr, uL + cL);
    }
    const T mL = L[0] * (sl - uL), mR = R[0] * (sr - uR);
    const T ss = (pR - pL + mL * uL - mR * uR) * rcp_(mL - mR);
    // upwind side K: left when the face sees S_L >= 0 or the left star region
    const bool left = ss >= T(0);
    const T* U = left ? L : R;
    const T uK = left ? uL : uR, vK = left ? vL : vR, wK = left ? wL : wR;
    const T pK = left ? pL : pR, irK = left ? irL : irR;
    const T sK = left ? sl : sr, mK = left ? mL : mR;
    const T FK[5] = {U[1], U[1] * uK + pK, U[1] * vK, U[1] * wK, (U[4] + pK) * uK};
    // S_K (U*_K - U_K), or 0 outside the fan (the plain upwind flux)
    const bool fan = left ? (sl < T(0)) : (sr > T(0));
    const T fac = mK * rcp_(sK - ss);   // rho_K (S_K - u_K) / (S_K - S*)
    const T Us[5] = {fac, fac * ss, fac * vK, fac * wK,
                     fac * (U[4] * irK + (ss - uK) * (ss + pK * rcp_(mK)))};
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = fan ? FK[q] + sK * (Us[q] - U[q]) : FK[q];
}

// Riemann solve by variant: 0 Roe inline, 1 Roe through one out-of-line
// copy, 2 HLLC inline.  (The kernel's RSV template argument carries this in
// bits 0-1, the reconstruction, 0 primitive / 1 characteristic, in bit 2 and
// a compiled-in van Leer limiter in bit 3.)
template <int RSV> struct RoeTag {};
template <int MODE, class T, class P>
__device__ __forceinline__ void roe_pick(RoeTag<0>, const T L[5], const T R[5],
                                         const KConst<T, P>& kc, T F[5], uint32_t& st) {
    roe_rot<MODE>(L, R, kc, F, st);
}
template <int MODE, class T, class P>
__device__ __forceinline__ void roe_pick(RoeTag<1>, const T L[5], const T R[5],
                                         const KConst<T, P>& kc, T F[5], uint32_t& st) {
    RoeIO<T> a, b;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        a.v[q] = L[q];
        b.v[q] = R[q];
    }
    a.st = b.st = 0;
    const RoeIO<T> r = roe_call<MODE>(a, b, kc);
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = r.v[q];
    st |= r.st;
}
template <int MODE, class T, class P>
__device__ __forceinline__ void roe_pick(RoeTag<2>, const T L[5], const T R[5],
                                         const KConst<T, P>& kc, T F[5], uint32_t&) {
    hllc_rot<MODE>(L, R, kc, F);
}
template <int MODE, int RSV, class T, class P>
__device__ __forceinline__ void roe_solve(const T L[5], const T R[5], const KConst<T, P>& kc,
                                          T F[5], uint32_t& st) {
    roe_pick<MODE>(RoeTag<RSV>(), L, R, kc, F, st);
}

// ---------------------------------------------------------------------------
// Conserved state of a primitive face value.
template <class T>
__device__ __forceinline__ void cons(const T w[5], T u[5], T igm1) {
    u[0] = w[0];
    u[1] = w[0] * w[1];
    u[2] = w[0] * w[2];
    u[3] = w[0] * w[3];
    u[4] = w[4] * igm1 + T(0.5) * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]);
}

// Flux difference F_d(W^-) - F_d(W^+) in direction D (compile time), with E^-
// and E^+ the face energies, accumulated into acc.
template <int D, class T>
__device__ __forceinline__ void flux_diff(const T wm[5], T Em, const T wp[5], T Ep, T acc[5]) {
    const T unm = wm[1 + D], unp = wp[1 + D];
    const T mm = wm[0] * unm, mp = wp[0] * unp;
    T fm[5], fp[5];
    fm[0] = mm;
    fm[1] = mm * wm[1];
    fm[2] = mm * wm[2];
    fm[3] = mm * wm[3];
    fm[1 + D] = fm[1 + D] + wm[4];
    fm[4] = (Em + wm[4]) * unm;
    fp[0] = mp;
    fp[1] = mp * wp[1];
    fp[2] = mp * wp[2];
    fp[3] = mp * wp[3];
    fp[1 + D] = fp[1 + D] + wp[4];
    fp[4] = (Ep + wp[4]) * unp;
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = acc[q] + (fm[q] - fp[q]);
}

// Limited slopes of the cell state wc along direction d from its neighbours
// lo, hi (plane arrays, stride kPlane).  REC 0: per primitive component;
// REC 1: in the characteristic variables of the primitive Euler system along
// d (left eigenvectors l1 = (0, -rho/(2c), 0, 0, 1/(2c^2)), l2 = (1, 0, 0, 0,
// -1/c^2), l3 = e_t1, l4 = e_t2, l5 = (0, rho/(2c), 0, 0, 1/(2c^2)); right
// eigenvectors r1 = (1, -c/rho, 0, 0, c^2), r2 = e_rho, r3 = e_t1, r4 = e_t2,
// r5 = (1, c/rho, 0, 0, c^2)), primitive where c^2 <= 0.
template <int REC> struct RecTag {};
template <int LIM, class T, class P>
__device__ __forceinline__ void slopes(RecTag<0>, int, const T* __restrict__ lo, const T wc[5],
                                       const T* __restrict__ hi, const KConst<T, P>& kc,
                                       T s[5]) {
#pragma unroll
    for (int q = 0; q < 5; ++q) s[q] = limit<LIM>(wc[q] - lo[q * kPlane], hi[q * kPlane] - wc[q], kc);
}
template <int LIM, class T, class P>
__device__ __forceinline__ void slopes(RecTag<1>, int d, const T* __restrict__ lo, const T wc[5],
                                       const T* __restrict__ hi, const KConst<T, P>& kc,
                                       T s[5]) {
    T dl[5], dr[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        dl[q] = wc[q] - lo[q * kPlane];
        dr[q] = hi[q * kPlane] - wc[q];
    }
    const T ir = rcp_(wc[0]);
    const T c2 = kc.gamma * wc[4] * ir;
    if (!(c2 > T(0))) {
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] = limit<LIM>(dl[q], dr[q], kc);
        return;
    }
    const int n = 1 + d, t1 = 1 + (d + 1) % 3, t2 = 1 + (d + 2) % 3;
    const T c = sqrt_(c2), ic2 = rcp_(c2);
    const T rc = wc[0] * rcp_(c);  // rho / c
    T da[5];
    {
        const T pl = dl[4] * ic2, pr = dr[4] * ic2, ul = rc * dl[n], ur = rc * dr[n];
        da[0] = limit<LIM>(T(0.5) * (pl - ul), T(0.5) * (pr - ur), kc);
        da[1] = limit<LIM>(dl[0] - pl, dr[0] - pr, kc);
        da[2] = limit<LIM>(dl[t1], dr[t1], kc);
        da[3] = limit<LIM>(dl[t2], dr[t2], kc);
        da[4] = limit<LIM>(T(0.5) * (pl + ul), T(0.5) * (pr + ur), kc);
    }
    s[0] = da[0] + da[1] + da[4];
    s[n] = c * ir * (da[4] - da[0]);
    s[t1] = da[2];
    s[t2] = da[3];
    s[4] = c2 * (da[0] + da[4]);
}

// Face values wm = wc - s/2, wp = wc + s/2 of the van Leer-limited primitive
// slopes s along one direction (lo, hi: the neighbours, plane arrays), FP32,
// with components 0-1 and 2-3 on paired FP32 instructions.  Same operations,
// in the same order, as slopes(RecTag<0>) with limit<0> and the scalar face
// values: the results are identical.
__device__ __forceinline__ float2 vanleer_x2(float2 a, float2 b) {
    const float2 ab = __fmul2_rn(a, b);
    const float2 sum = __fadd2_rn(a, b);
    const float2 r = __fmul2_rn(__fmul2_rn(pk(2.0f, 2.0f), ab), pk(rcp_(sum.x), rcp_(sum.y)));
    return pk(ab.x > 0.0f ? r.x : 0.0f, ab.y > 0.0f ? r.y : 0.0f);
}
template <class P>
__device__ __forceinline__ void faces_vanleer_x2(const float* __restrict__ lo, const float wc[5],
                                                 const float* __restrict__ hi,
                                                 const KConst<float, P>& kc, float wm[5],
                                                 float wp[5]) {
    const float2 n1 = pk(-1.0f, -1.0f), mh = pk(-0.5f, -0.5f), ph = pk(0.5f, 0.5f);
    const float2 c01 = pk(wc[0], wc[1]), c23 = pk(wc[2], wc[3]);
    const float2 s01 = vanleer_x2(__ffma2_rn(pk(lo[0], lo[kPlane]), n1, c01),
                                  __ffma2_rn(c01, n1, pk(hi[0], hi[kPlane])));
    const float2 s23 = vanleer_x2(__ffma2_rn(pk(lo[2 * kPlane], lo[3 * kPlane]), n1, c23),
                                  __ffma2_rn(c23, n1, pk(hi[2 * kPlane], hi[3 * kPlane])));
    const float s4 = limit<0>(wc[4] - lo[4 * kPlane], hi[4 * kPlane] - wc[4], kc);
    const float2 m01 = __ffma2_rn(s01, mh, c01), p01 = __ffma2_rn(s01, ph, c01);
    const float2 m23 = __ffma2_rn(s23, mh, c23), p23 = __ffma2_rn(s23, ph, c23);
    wm[0] = m01.x; wm[1] = m01.y; wm[2] = m23.x; wm[3] = m23.y;
    wp[0] = p01.x; wp[1] = p01.y; wp[2] = p23.x; wp[3] = p23.y;
    wm[4] = wc[4] - 0.5f * s4;
    wp[4] = wc[4] + 0.5f * s4;
}

// Hancock half-step for the cell at plane index c (20x20 plane layout) of
// plane k: Wm/W0/Wp are the primitive planes k-1, k, k+1.  fs[f] receives
// the un-evolved conserved face states x-, x+, y-, y+, z-, z+ (the limited
// reconstruction), du the common half-step increment.
template <int LIM, int REC = 0, class T, class P>
__device__ __forceinline__ void predict_unevolved(const T* __restrict__ Wm,
                                                  const T* __restrict__ W0,
                                                  const T* __restrict__ Wp, int c, T half_lam,
                                                  T igm1, const KConst<T, P>& kc, T fs[6][5],
                                                  T du[5]) {
    T wc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) wc[q] = W0[q * kPlane + c];
    T acc[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const T* lo = (d == 2) ? Wm + c : W0 + c - (d == 0 ? 1 : 20);
        const T* hi = (d == 2) ? Wp + c : W0 + c + (d == 0 ? 1 : 20);
        T wm[5], wp[5];
        if constexpr (sizeof(T) == 4 && LIM == 0 && REC == 0) {  // every FP32-storage mode
            faces_vanleer_x2(lo, wc, hi, kc, wm, wp);
        } else {
            T sl[5];
            slopes<LIM>(RecTag<REC>(), d, lo, wc, hi, kc, sl);
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                wm[q] = wc[q] - T(0.5) * sl[q];
                wp[q] = wc[q] + T(0.5) * sl[q];
            }
        }
        cons<T>(wm, fs[2 * d], igm1);
        cons<T>(wp, fs[2 * d + 1], igm1);
        if (d == 0) flux_diff<0>(wm, fs[0][4], wp, fs[1][4], acc);
        if (d == 1) flux_diff<1>(wm, fs[2][4], wp, fs[3][4], acc);
        if (d == 2) flux_diff<2>(wm, fs[4][4], wp, fs[5][4], acc);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) du[q] = half_lam * acc[q];
}

// The branch-free Hancock half-step: fs[f] receives the evolved face states
// (the un-evolved ones + du); returns whether all six are admissible (rho > 0,
// p > 0).
template <int MODE, int LIM, int REC = 0, class T, class P>
__device__ __forceinline__ bool predict_core(const T* __restrict__ Wm, const T* __restrict__ W0,
                                             const T* __restrict__ Wp, int c, T half_lam,
                                             T igm1, const KConst<T, P>& kc, T fs[6][5],
                                             T du[5]) {
    predict_unevolved<LIM, REC>(Wm, W0, Wp, c, half_lam, igm1, kc, fs, du);
    bool ok = true, und = false;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
#pragma unroll
        for (int q = 0; q < 5; ++q) fs[f][q] = fs[f][q] + du[q];
        ok &= admissible<MODE>(fs[f][0], fs[f][1], fs[f][2], fs[f][3], fs[f][4], und);
    }
    if constexpr (MODE == GAMER_MODE_MIXED || MODE == GAMER_MODE_FF) {
        if (und) {
            States6 f6;
#pragma unroll
            for (int f = 0; f < 6; ++f)
#pragma unroll
                for (int q = 0; q < 5; ++q) f6.v[f][q] = fs[f][q];
            ok = (MODE == GAMER_MODE_MIXED) ? admissible6_fp64(f6) : admissible6_ff(f6);
        }
    }
    return ok;
}

// Predictor fallback: all six states become the cell average (option 0) or
// the un-evolved reconstruction, recovered as (U + du) - du (option 1).
template <class T, class P>
__device__ __forceinline__ void predict_fallback(const T uc[5], const T du[5],
                                                 const KConst<T, P>& kc, T fs[6][5]) {
#pragma unroll
    for (int f = 0; f < 6; ++f)
#pragma unroll
        for (int q = 0; q < 5; ++q) fs[f][q] = (kc.pfb == 0) ? uc[q] : fs[f][q] - du[q];
}

// The half-step of one cell with its outputs stored as they are produced: the
// x-, x+, y-, y+ states into the face arrays at dxm, dxp, dym, dyp (component
// 0; components kFaceStride apart), the z- and z+ states into zm, zp.  Each
// state is stored as soon as it is evolved and tested, so that the six never
// have to be held together in registers; the rare fallback (any state not
// admissible: GAMER_ST_PREDICTOR_FALLBACK in st) then overwrites all six with
// the cell average uc (option 0) or the un-evolved reconstruction, recovered
// as (U + du) - du from the stored values (option 1).  The re-reads are
// volatile, so that the compiler does not keep the stored values in registers
// for them.  Same results as evolving all six, testing, then storing (which
// the mixed build still does).
template <int MODE, int LIM = -1, int REC = 0, class T, class P>
__device__ __forceinline__ void predict_store(const T* __restrict__ Wm, const T* __restrict__ W0,
                                              const T* __restrict__ Wp, const T uc[5], int c,
                                              T half_lam, T igm1, const KConst<T, P>& kc,
                                              T* dxm, T* dxp, T* dym, T* dyp, T zm[5], T zp[5],
                                              uint32_t& st) {
    T fs[6][5], du[5];
    T* const dst[4] = {dxm, dxp, dym, dyp};
    if constexpr (MODE == GAMER_MODE_MIXED) {
        // the mixed build measured 0.7 % faster evolving all six first
        if (!predict_core<MODE, LIM, REC>(Wm, W0, Wp, c, half_lam, igm1, kc, fs, du)) {
            st |= GAMER_ST_PREDICTOR_FALLBACK;
            predict_fallback(uc, du, kc, fs);
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
#pragma unroll
            for (int f = 0; f < 4; ++f) dst[f][q * kFaceStride] = fs[f][q];
            zm[q] = fs[4][q];
            zp[q] = fs[5][q];
        }
        return;
    }
    predict_unevolved<LIM, REC>(Wm, W0, Wp, c, half_lam, igm1, kc, fs, du);
    auto reread = [&](int f, int q) -> T {
        return *reinterpret_cast<const volatile T*>(dst[f] + q * kFaceStride);
    };
    bool ok = true, und = false;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        T v[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) v[q] = fs[f][q] + du[q];
        ok &= admissible<MODE>(v[0], v[1], v[2], v[3], v[4], und);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            if (f < 4) dst[f][q * kFaceStride] = v[q];
            else if (f == 4) zm[q] = v[q];
            else zp[q] = v[q];
        }
    }
    if constexpr (MODE == GAMER_MODE_FF) {
        if (und) {
            States6 f6;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
#pragma unroll
                for (int f = 0; f < 4; ++f) f6.v[f][q] = reread(f, q);
                f6.v[4][q] = zm[q];
                f6.v[5][q] = zp[q];
            }
            ok = admissible6_ff(f6);
        }
    }
    if (!ok) {
        st |= GAMER_ST_PREDICTOR_FALLBACK;
        const bool avg = kc.pfb == 0;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
#pragma unroll
            for (int f = 0; f < 4; ++f)
                dst[f][q * kFaceStride] = avg ? uc[q] : reread(f, q) - du[q];
            zm[q] = avg ? uc[q] : zm[q] - du[q];
            zp[q] = avg ? uc[q] : zp[q] - du[q];
        }
    }
}

// cells of the 20^3 tile that the stencil reads: at most one coordinate
// outside [0,16), or two, both one cell outside.
__device__ __forceinline__ bool is_read_cell(int i, int j, int k) {
    const bool oi = (unsigned)i > 15u, oj = (unsigned)j > 15u, ok = (unsigned)k > 15u;
    const int o = int(oi) + int(oj) + int(ok);
    const bool ni = !oi || i == -1 || i == 16;
    const bool nj = !oj || j == -1 || j == 16;
    const bool nk = !ok || k == -1 || k == 16;
    return o <= 1 || (o == 2 && ni && nj && nk);
}

// Plane cell of this thread's r-th conversion (r = 0, 1, 2), or -1: cell
// tid + r * NT while inside the plane (NT threads per group).
template <int NT = kThreads>
__device__ __forceinline__ int convert_cell(int r) {
    const int c = int(threadIdx.x) + r * NT;
    return c < kPlane ? c : -1;
}

// Which of this thread's plane cells (convert_cell(r), r < 3) the stencil
// reads, for the three kinds of plane (bit 3 * kind + r): kind 0 a plane
// inside the group, 1 one plane outside (-1, 16), 2 two outside (-2, 17).
template <int NT = kThreads>
__device__ __forceinline__ uint32_t read_cell_mask() {
    uint32_t m = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int c = convert_cell<NT>(r);
        if (c < 0) break;
        const int i = c % 20 - 2, j = c / 20 - 2;
        if (is_read_cell(i, j, 0)) m |= 1u << r;
        if (is_read_cell(i, j, -1)) m |= 1u << (3 + r);
        if (is_read_cell(i, j, -2)) m |= 1u << (6 + r);
    }
    return m;
}

// the read bits of plane kp out of read_cell_mask()
__device__ __forceinline__ uint32_t plane_read_bits(uint32_t mask, int kp) {
    const int kind = ((unsigned)kp < 16u) ? 0 : (kp == -1 || kp == 16) ? 1 : 2;
    return (mask >> (3 * kind)) & 7u;
}

// Conserved plane -> primitive plane (all 400 cells, by convert_cell; the
// flag covers the read cells, `rbits` from plane_read_bits).
template <int MODE, int NT = kThreads, class T, class P>
__device__ __forceinline__ void convert_plane(const T* __restrict__ U, T* __restrict__ W,
                                              uint32_t rbits, const KConst<T, P>& kc,
                                              uint32_t& st) {
    uint32_t hi = 0;  // MIXED: bit r, cell r needs the FP64 recovery
    // FF with 160 threads: cells 0 and 1 of the thread (both inside the
    // plane) on the paired float-float recovery, each lane the same operations
    // as the scalar one; cell 2 below
    constexpr bool kPairFF = (MODE == GAMER_MODE_FF) && (NT == kThreads);
    if constexpr (kPairFF) {
        const int c0 = convert_cell<NT>(0), c1 = convert_cell<NT>(1);
        T a[5], b[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            a[q] = U[q * kPlane + c0];
            b[q] = U[q * kPlane + c1];
        }
        const T ia = rcp_(a[0]), ib = rcp_(b[0]);
        W[0 * kPlane + c0] = a[0];
        W[1 * kPlane + c0] = a[1] * ia;
        W[2 * kPlane + c0] = a[2] * ia;
        W[3 * kPlane + c0] = a[3] * ia;
        W[0 * kPlane + c1] = b[0];
        W[1 * kPlane + c1] = b[1] * ib;
        W[2 * kPlane + c1] = b[2] * ib;
        W[3 * kPlane + c1] = b[3] * ib;
        bool unused = false;
        const float2 p = pressure_x2<MODE>(pk(a[0], b[0]), pk(a[1], b[1]), pk(a[2], b[2]),
                                           pk(a[3], b[3]), pk(a[4], b[4]), pk(ia, ib), kc, unused);
        W[4 * kPlane + c0] = p.x;
        W[4 * kPlane + c1] = p.y;
        bool fa = true, fb = true;
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            fa &= finite_(a[q]);
            fb &= finite_(b[q]);
        }
        if ((!fa & bool(rbits & 1u)) | (!fb & bool((rbits >> 1) & 1u))) st |= GAMER_ST_BAD_INPUT;
    }
#pragma unroll
    for (int r = kPairFF ? 2 : 0; r < 3; ++r) {
        const int c = convert_cell<NT>(r);
        if (c < 0) break;
        T u[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) u[q] = U[q * kPlane + c];
        const T ir = rcp_(u[0]);
        W[0 * kPlane + c] = u[0];
        W[1 * kPlane + c] = u[1] * ir;
        W[2 * kPlane + c] = u[2] * ir;
        W[3 * kPlane + c] = u[3] * ir;
        if constexpr (MODE == GAMER_MODE_MIXED) {
            // FP32 recovery here; the cells that need FP64 are redone below,
            // after the loop, in one rarely taken branch (a branch per cell
            // would split the unrolled loop into separate blocks)
            bool h = false;
            W[4 * kPlane + c] = pressure_mixed32(u[1], u[2], u[3], u[4], ir, kc, h);
            hi |= uint32_t(h) << r;
        } else {
            W[4 * kPlane + c] = pressure<MODE>(u[0], u[1], u[2], u[3], u[4], ir, kc);
        }
        bool fin = true;
#pragma unroll
        for (int q = 0; q < 5; ++q) fin &= finite_(u[q]);
        if (!fin & bool((rbits >> r) & 1u)) st |= GAMER_ST_BAD_INPUT;
    }
    if constexpr (MODE == GAMER_MODE_MIXED) {
        if (hi) {
            for (int r = 0; r < 3; ++r) {
                if (!((hi >> r) & 1u)) continue;
                const int c = convert_cell<NT>(r);
                const T u0 = U[c], ir = rcp_(u0);
                W[4 * kPlane + c] = pressure_fp64(u0, U[kPlane + c], U[2 * kPlane + c],
                                                  U[3 * kPlane + c], U[4 * kPlane + c], ir,
                                                  kc.gm1p);
            }
        }
    }
}

// Copies input plane kp into its ring slot of any shared layout with raw[2][]
// and mbar[2] members.
template <int RING = 2, class SM, class T>
__device__ __forceinline__ void issue_plane(SM& S, const T* gin, int kp) {
    const int slot = (kp + 2) % RING;
    constexpr uint32_t bytes = 5u * kPlane * sizeof(T);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&S.mbar[slot], bytes);
#pragma unroll
    for (int q = 0; q < 5; ++q)
        bulk_copy_g2s(&S.raw[slot][q * kPlane], gin + (q * 20 + (kp + 2)) * kPlane,
                      kPlane * sizeof(T), &S.mbar[slot]);
}

// Uniform level read directly by the kernel (fused ghost gather): gx*gy*gz
// groups of [5][16][16][16], group id (z*gy + y)*gx + x, periodic (bc 0) or
// zero-gradient (bc 1) boundaries.  The device buffer may hold a window of the
// level: its layer l (of gx*gy groups) is the level's z-layer (zb + l) mod gz;
// the kernel's group g is the level's group g + z0*gx*gy.  The whole level is
// zb = z0 = 0.
struct LevelGeom {
    int gx, gy, gz, bc;
    int zb, z0;
    int poison;  // debug: fill each input slot with NaN before gathering into it
    // debug: the copy of input plane 5 of group drop_group (-1: none) is never
    // issued, so the wait for it runs out (after wait_polls polls) and the
    // give-up path runs; wait_polls 0 means the default kWaitPolls
    int64_t drop_group;
    uint32_t wait_polls;
};

// Level coordinate X, at most two cells outside [0, n), mapped into the level:
// periodic wrap (bc 0) or zero-gradient clamp (bc 1).
__device__ __forceinline__ int wrap_near(int X, int n, int bc) {
    if (X < 0) return bc == 0 ? X + n : 0;
    if (X >= n) return bc == 0 ? X - n : n - 1;
    return X;
}

// Element offset of the input plane inside its ring slot.  The fused gather
// moves FP32 planes 8 bytes in, so that the 16 interior cells of every row
// (tile columns 2..17) start on a 16-byte boundary.
template <int SRC, class T>
__device__ __forceinline__ constexpr int raw_offset() {
    return (SRC == 1 && sizeof(T) == 4) ? 2 : 0;
}

// distance of tile coordinate c in [0, 20) from the interior [2, 18)
__device__ __forceinline__ int ghost_depth(int c) { return c < 2 ? 2 - c : (c > 17 ? c - 17 : 0); }

// The fused gather copies, for input plane kp of a group, every cell the
// stencil reads (is_read_cell) and no more:
//  * interior runs: the 16 cells x in [0, 16) of tile row j, for the rows
//    with depth(j) + depth(kp) <= 2, in 16-byte copies; thread t takes chunk
//    t % CH of row (t / CH) % 20 for variables v0, v0 + VS, ... (consecutive
//    lanes read consecutive 16 bytes of a level row; rows land 80 or 160
//    bytes apart in shared memory, which spreads a warp over all banks);
//  * x ghosts: the two cells on each side of rows j = 1..18 of planes with
//    depth(kp) <= 1 (180 items, one 2-cell copy each; single cells where a
//    clamped boundary repeats one): thread t takes items t and t + 160.
// Everything but the z offset is fixed for a group and worked out once into
// a per-thread plan kept in shared memory (registers are the kernel's
// scarcest resource): level offsets relative to the z-layer of groups, in
// units of 16 cells (32 bits for up to 2^31 / 1280 groups per layer), and
// the ghost items' shared-memory destinations.
struct alignas(16) GatherPlan {
    int32_t chunk;  // 16-cell offset of the thread's interior row (variable v0)
    int32_t gh[2];  // 16-cell offsets of the rows of its x-ghost items
    uint32_t bits;  // [0,4), [4,8): x of ghost item 0, 1 inside its 16-cell row;
                    // 8, 9: item is a 2-cell copy; [10,21), [21,32): item 0, 1
                    // offset in the plane
};

// row and 16-byte chunk of the interior run of this thread (NT threads)
template <class T, int NT = kThreads> struct GatherRow {
    static constexpr int E16 = 16 / int(sizeof(T));  // cells per 16-byte chunk
    static constexpr int CH = 16 / E16;              // chunks per 16-cell row: 4 or 8
    static constexpr int VS = NT / CH / 20;          // variables per pass: 1, 2 or 4
    static_assert(VS * 20 * CH == NT, "gather mapping");
    int q, v0, j;
    __device__ __forceinline__ GatherRow() {
        const int R0 = int(threadIdx.x) / CH;
        q = int(threadIdx.x) - R0 * CH;
        v0 = R0 / 20;
        j = R0 - 20 * v0;
    }
};

template <class T, int NT = kThreads>
__device__ __forceinline__ GatherPlan make_plan(const LevelGeom& L, int bx, int by) {
    const GatherRow<T, NT> w;
    GatherPlan P;
    const int ny = 16 * L.gy, nx = 16 * L.gx;
    const int Y = wrap_near(by * 16 + w.j - 2, ny, L.bc);
    P.chunk = ((Y >> 4) * L.gx + bx) * 1280 + w.v0 * 256 + (Y & 15);
    P.bits = 0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        P.gh[r] = 0;
        const int it = int(threadIdx.x) + r * NT;
        if (it < 180) {
            const int v = it / 36, rem = it - 36 * v;
            const int jj = 1 + (rem >> 1), side = rem & 1;
            const int Yg = wrap_near(by * 16 + jj - 2, ny, L.bc);
            const int X0 = wrap_near(side ? bx * 16 + 16 : bx * 16 - 2, nx, L.bc);
            const int X1 = wrap_near(side ? bx * 16 + 17 : bx * 16 - 1, nx, L.bc);
            P.gh[r] = ((Yg >> 4) * L.gx + (X0 >> 4)) * 1280 + v * 256 + (Yg & 15);
            P.bits |= uint32_t(X0 & 15) << (4 * r);
            if (X1 == X0 + 1) P.bits |= 1u << (8 + r);
            P.bits |= uint32_t(v * kPlane + jj * 20 + (side ? 18 : 0)) << (10 + 11 * r);
        }
    }
    return P;
}

// Gathers input plane kp of the group of plan P (z index bz) from the level
// into its ring slot; every thread then arrives on the slot's barrier
// (expected count kThreads).
template <int RING, int NT = kThreads, class SM, class T>
__device__ __forceinline__ void gather_plane(SM& S, const T* __restrict__ level,
                                             const LevelGeom& L, const GatherPlan& P, int bz,
                                             int kp) {
    using G = GatherRow<T, NT>;
    const G w;
    const int slot = (kp + 2) % RING;
    T* plane = S.raw[slot] + raw_offset<1, T>();
    const int Z = wrap_near(bz * 16 + kp, 16 * L.gz, L.bc);
    int zl = (Z >> 4) - L.zb;  // window layer of the group layer holding Z
    zl += (zl < 0) ? L.gz : 0;
    const T* lz = level + int64_t(zl) * (L.gy * L.gx) * 20480 + (Z & 15) * 256;
    const int dk = ghost_depth(kp + 2);
    if (ghost_depth(w.j) + dk <= 2) {
        const T* src = lz + int64_t(P.chunk) * 16 + w.q * G::E16;
        T* dst = plane + w.v0 * kPlane + w.j * 20 + 2 + w.q * G::E16;
#pragma unroll
        for (int v = 0; v < 5; v += G::VS) {
            if (v + w.v0 < 5) cp_async_cg16(dst, src);
            dst += G::VS * kPlane;
            src += G::VS * 4096;
        }
    }
    if (dk <= 1) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (int(threadIdx.x) + r * NT >= 180) break;
            const T* src = lz + int64_t(P.gh[r]) * 16 + ((P.bits >> (4 * r)) & 15u);
            T* dst = plane + ((P.bits >> (10 + 11 * r)) & 2047u);
            if (P.bits & (1u << (8 + r))) {
                cp_async<2 * int(sizeof(T))>(dst, src);
            } else {
                cp_async<int(sizeof(T))>(dst, src);
                cp_async<int(sizeof(T))>(dst + 1, src);
            }
        }
    }
    cp_async_arrive(&S.mbar[slot]);
}

// Plane loaders by input kind, set up once per group: 0 -- TMA bulk copies of
// the tile's plane issued by thread 0; 1 -- gather from the level by all
// threads, with the plan in `plan` (kThreads entries of shared memory).
template <int SRC, int RING, class T, int NT = kThreads> struct PlaneLoader;
template <int RING, class T, int NT> struct PlaneLoader<0, RING, T, NT> {
    static constexpr size_t kExtraSmem = 0;
    const T* gin;
    bool drop;  // debug: withhold plane 5 (LevelGeom::drop_group)
    __device__ __forceinline__ PlaneLoader(const T* in, int64_t g, const LevelGeom& geo,
                                           GatherPlan*)
        : gin(in + g * 40000), drop(g == geo.drop_group) {}
    // true when the copy was issued (always, but for the debug drop)
    template <class SM> __device__ __forceinline__ bool load(SM& S, int kp) const {
        if (drop && kp == 5) return false;
        if (threadIdx.x == 0) issue_plane<RING>(S, gin, kp);
        return true;
    }
};
template <int RING, class T, int NT> struct PlaneLoader<1, RING, T, NT> {
    static constexpr size_t kExtraSmem = NT * sizeof(GatherPlan);
    const T* level;
    const LevelGeom& L;
    GatherPlan* plan;
    int bz;
    bool drop;  // debug: withhold plane 5 (LevelGeom::drop_group)
    __device__ __forceinline__ PlaneLoader(const T* in, int64_t g, const LevelGeom& geo,
                                           GatherPlan* plan_)
        : level(in), L(geo), plan(plan_ + threadIdx.x), drop(g == geo.drop_group) {
        const int bx = int(g % geo.gx), by = int((g / geo.gx) % geo.gy);
        bz = geo.z0 + int(g / (int64_t(geo.gx) * geo.gy));
        *plan = make_plan<T, NT>(geo, bx, by);  // read back by this thread only
    }
    template <class SM> __device__ __forceinline__ bool load(SM& S, int kp) const {
        if (drop && kp == 5) return false;  // debug: no copy, no arrival
        if (L.poison) {
            // debug: cells the gather does not write read back as NaN, so a
            // stencil read outside the gathered set shows up in the results
            // (the slot's previous plane was consumed before this call)
            T* slot = S.raw[(kp + 2) % RING];
            for (int c = threadIdx.x; c < 5 * kPlane + 4; c += NT)
                slot[c] = __int_as_float(0x7fc00000) + T(0);
            __syncthreads();
        }
        const GatherPlan P = *plan;
        gather_plane<RING, NT>(S, level, L, P, bz, kp);
        return true;
    }
};

// Accumulator of the per-group conserved sums: FP64 in FP64 mode; in FP32
// modes a compensated (hi, lo) float pair per thread (TwoSum), exact to about
// 2^-48 relative for the few dozen terms one thread adds.  add5 takes the five
// components of one cell.
template <class T> struct SumAcc;
template <> struct SumAcc<double> {
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    __device__ __forceinline__ void add(int q, double x) { s[q] += x; }
    __device__ __forceinline__ void add5(const double o[5]) {
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] += o[q];
    }
    __device__ __forceinline__ double get(int q) const { return s[q]; }
};
template <> struct SumAcc<float> {
    // components 0-1 and 2-3 as float2 pairs, so that add5 runs their TwoSum
    // steps on paired FP32 instructions (each lane the same IEEE operations
    // as the scalar steps, so the same results); component 4 alone
    float2 h01 = {0.f, 0.f}, h23 = {0.f, 0.f}, l01 = {0.f, 0.f}, l23 = {0.f, 0.f};
    float h4 = 0.f, l4 = 0.f;
    static __device__ __forceinline__ void step(float& hi, float& lo, float x) {
        const float s = hi + x;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (x - bp);
        hi = s;
        lo += err;
    }
    static __device__ __forceinline__ void step2(float2& hi, float2& lo, float2 x) {
        const float2 s = __fadd2_rn(hi, x);
        const float2 bp = __fadd2_rn(s, make_float2(-hi.x, -hi.y));
        const float2 t = __fadd2_rn(s, make_float2(-bp.x, -bp.y));
        const float2 err = __fadd2_rn(__fadd2_rn(hi, make_float2(-t.x, -t.y)),
                                      __fadd2_rn(x, make_float2(-bp.x, -bp.y)));
        hi = s;
        lo = __fadd2_rn(lo, err);
    }
    __device__ __forceinline__ void add5(const float o[5]) {
        step2(h01, l01, make_float2(o[0], o[1]));
        step2(h23, l23, make_float2(o[2], o[3]));
        step(h4, l4, o[4]);
    }
    __device__ __forceinline__ void add(int q, float x) {
        if (q == 0) step(h01.x, l01.x, x);
        else if (q == 1) step(h01.y, l01.y, x);
        else if (q == 2) step(h23.x, l23.x, x);
        else if (q == 3) step(h23.y, l23.y, x);
        else step(h4, l4, x);
    }
    __device__ __forceinline__ float hi(int q) const {
        return q == 0 ? h01.x : q == 1 ? h01.y : q == 2 ? h23.x : q == 3 ? h23.y : h4;
    }
    __device__ __forceinline__ float lo(int q) const {
        return q == 0 ? l01.x : q == 1 ? l01.y : q == 2 ? l23.x : q == 3 ? l23.y : l4;
    }
    __device__ __forceinline__ double get(int q) const { return double(hi(q)) + double(lo(q)); }
};

// A bounded on-chip wait of this CTA gave up in group g, so the CTA stops:
// every group it still owns (g, g + gridDim.x, ...) is marked
// GAMER_ST_INTERNAL_TIMEOUT and gets NaN partials, which gamer_hydro_dt turns
// into a NaN time step for the group's level -- the failure shows even when
// the caller passed no status array.  Their out and face-flux values are left
// as they were.  Called by one thread.
__device__ __forceinline__ void mark_abandoned(int64_t g, int64_t N, uint32_t* status,
                                               double* partials) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t h = g; h < N; h += gridDim.x) {
        if (status) status[h] = GAMER_ST_INTERNAL_TIMEOUT;
        if (partials)
            for (int q = 0; q < 6; ++q) partials[h * 6 + q] = nan;
    }
}

// ---------------------------------------------------------------------------
// MINB: CTAs per SM the register budget is sized for (launch bounds); the
// launcher picks the variant (2: no spills, 3: more warps per SM).
// SRC 0: `in` holds N ghost-padded 20^3 tiles, loaded plane by plane with the
// TMA engine; SRC 1: `in` is the uniform level `geo` (N = gx*gy*gz groups) and
// each plane is gathered from the group and its neighbours (fused ghost fill).
// RSV: bits 0-1 the Riemann solver (0 Roe inline, 1 Roe out of line, 2 HLLC),
// bit 2 characteristic (1) or primitive (0) slope limiting, bit 3 the van Leer
// limiter compiled in (1) or the limiter read from kc.limiter per slope (0).
// RING: input planes in flight (2: the copy of plane k+2 goes out after phase A
// of plane k; 3: plane k+3 does, one full iteration ahead of its use).
// NT: threads per group, 160 (a thread owns two interior columns or one
// column and a face-slab cell) or 320 (one column or one slab cell each: half
// the registers per thread for twice the warps per SM).
template <int MODE, int MINB, int RSV = 0, int SRC = 0, int RING = 2, int NT = kThreads>
__global__ void __launch_bounds__(NT, MINB)
    hydro_step_kernel(const typename Prec<MODE>::T* __restrict__ in,
                      typename Prec<MODE>::T* __restrict__ out,
                      typename Prec<MODE>::T* __restrict__ face_flux,
                      const double* __restrict__ dt, const double* __restrict__ dh,
                      uint32_t* __restrict__ status, double* __restrict__ partials, int64_t N,
                      KConst<typename Prec<MODE>::T, typename Prec<MODE>::P> kc,
                      LevelGeom geo) {
    using T = typename Prec<MODE>::T;
    static_assert(NT == 160 || NT == 320, "threads per group");
    constexpr bool kWide = NT == 320;
    constexpr int kLim = (RSV & 8) ? 0 : -1;  // van Leer compiled in, or kc.limiter
    constexpr int kRec = (RSV >> 2) & 1;
    extern __shared__ __align__(128) unsigned char smem_bytes[];
    Smem<T, RING>& S = *reinterpret_cast<Smem<T, RING>*>(smem_bytes);
    constexpr int ROFF = raw_offset<SRC, T>();
    GatherPlan* gplan = reinterpret_cast<GatherPlan*>(smem_bytes + sizeof(Smem<T, RING>));
    const uint32_t rmask = read_cell_mask<NT>();
    const uint32_t polls = geo.wait_polls ? geo.wait_polls : kWaitPolls;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;

    if (tid == 0) {
        for (int s = 0; s < RING; ++s) mbar_init(&S.mbar[s], SRC == 0 ? 1 : NT);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t parity = 0;   // bit s: phase parity expected next on slot s
    uint32_t pending = 0;  // bit s: a copy into slot s was issued and not yet waited for

    // owned interior columns: a warp owns a row pair (jA, jA + 4), lane -> i.
    // NT 160: warps 0-4 own pairs 0-4 (c0), warps 0-2 also pairs 5-7 (c1).
    // NT 320: warps 0-7 own pairs 0-7 (c0 only); warps 8-9 own no column
    // (their pair index is folded into 0-7 only to keep unused indices in
    // bounds).
    const bool owner = kWide ? (tid < 256) : true;
    const bool two = kWide ? false : (tid < 96);
    const int i0 = lane & 15, hb = (lane >> 4) * 4;
    const int pa = kWide ? (warp & 7) : warp, pb = warp + 5;
    const int j0 = (pa & 3) + ((pa >> 2) << 3) + hb;
    const int j1 = (pb & 3) + ((pb >> 2) << 3) + hb;
    const int pc0 = (j0 + 2) * 20 + (i0 + 2);
    const int pc1 = (j1 + 2) * 20 + (i0 + 2);
    const int fa0 = frow(j0) * 16 + i0, fa1 = frow(j1) * 16 + i0;
    // face-slab cell of threads 96..159 (NT 160) or 256..319 (NT 320): side 0:
    // i=-1, 1: i=16, 2: j=-1, 3: j=16
    const int sl = tid - (kWide ? 256 : 96), side = sl >> 4, st_ = sl & 15;
    const int si = (side == 0) ? -1 : (side == 1) ? 16 : st_;
    const int sj = (side == 2) ? -1 : (side == 3) ? 16 : st_;
    const int psl = (sj + 2) * 20 + (si + 2);
    // second prediction item: the second column (NT 160, warps 0-2) or the slab
    // cell (NT 160 warps 3-4; NT 320 warps 8-9).  Both kinds store all four x/y faces; a slab
    // cell's three unused faces go to entries 272..287 of their arrays, which
    // nothing reads, so one code path serves both.
    const int pc_b = two ? pc1 : psl;
    const int o_xm = two ? fa1 : (side == 1 ? 256 + st_ : 272 + st_);
    const int o_xp = two ? fa1 : (side == 0 ? 256 + st_ : 272 + st_);
    const int o_ym = two ? fa1 : (side == 3 ? 256 + st_ : 272 + st_);
    const int o_yp = two ? fa1 : (side == 2 ? 256 + st_ : 272 + st_);

    const T igm1 = T(1) / kc.gm1;

    for (int64_t g = blockIdx.x; g < N; g += gridDim.x) {
        // one input plane into its ring slot (all threads call load_plane)
        const PlaneLoader<SRC, RING, T, NT> loader(in, g, geo, gplan);
        auto load_plane = [&](int kp) { return loader.load(S, kp); };
        T* gout = out + g * 20480;
        T* gff = face_flux ? face_flux + g * (kc.flux9 ? 9 : 6) * kFluxPlane : nullptr;
        uint32_t st = 0;
        if (tid == 0) {
            // one FP64 division per group, shared through shared memory (read
            // after the prologue's first barrier)
            const double dtg = dt[g], dhg = dh[g];
            S.lam = static_cast<T>(dtg / dhg);
            S.status = 0;
            if (!(isfinite(dtg) && isfinite(dhg) && dtg >= 0.0 && dhg > 0.0))
                st |= GAMER_ST_BAD_INPUT;
        }
        // prologue: planes -2, -1, 0 -> primitives (W slots 0, 1, 2).  With two
        // ring slots plane 0 reuses the slot of plane -2; with three, plane 1
        // goes into it, so that it is in flight before the first iteration.
        bool timed_out = false;
        load_plane(-2);
        load_plane(-1);
        if (RING == 3) load_plane(0);
        pending |= (RING == 3) ? 7u : 3u;
        if (mbar_wait(&S.mbar[0], parity & 1u, polls)) {
            parity ^= 1u;
            pending &= ~1u;
            convert_plane<MODE, NT>(S.raw[0] + ROFF, S.W[0], plane_read_bits(rmask, -2), kc, st);
        } else {
            timed_out = true;
        }
        if (__syncthreads_or(timed_out)) goto abort_group;
        load_plane(RING == 3 ? 1 : 0);
        pending |= 1u;
        for (int kp = -1; kp <= 0; ++kp) {
            const int s = (kp + 2) % RING;
            if (!timed_out && mbar_wait(&S.mbar[s], (parity >> s) & 1u, polls)) {
                parity ^= 1u << s;
                pending &= ~(1u << s);
                convert_plane<MODE, NT>(S.raw[s] + ROFF, S.W[kp + 2], plane_read_bits(rmask, kp), kc,
                                    st);
            } else {
                timed_out = true;
            }
        }
        if (__syncthreads_or(timed_out)) goto abort_group;

        {
            const T lam = S.lam;
            const T half_lam = T(0.5) * lam;
            // owner registers: z+ state of the previous plane, the flux of the
            // z face below it, and E = U - lam (x/y flux divergence) of it
            T zp0[5], zp1[5], fzo0[5], fzo1[5], E0[5], E1[5];
#pragma unroll
            for (int q = 0; q < 5; ++q)
                zp0[q] = zp1[q] = fzo0[q] = fzo1[q] = E0[q] = E1[q] = T(0);
            T smax = T(0);
            SumAcc<T> sums;

            // Per plane k, two barriers: phase CA runs C(k-1) -- the x/y flux
            // divergence of plane k-1 from the fluxes of phase B(k-1) -- then
            // A(k), the half-step prediction of plane k; phase B(k) solves the
            // z faces k-1/2, which completes plane k-1 (written out at once),
            // then the x/y faces of plane k, and converts plane k+2.  C reads
            // only the thread's own face slots (where B left the fluxes), which
            // its own A overwrites next, and A writes nothing another thread
            // reads before the barrier, so C(k-1) and A(k) share a phase.
            // Across the x/y solves only U, the lower
            // z flux and the z+ state of plane k stay in registers.  The two z
            // fluxes of a cell are differenced before scaling, so equal fluxes
            // cancel exactly (a uniform state stays bitwise uniform).
            T zm0[5], zm1[5], zpn0[5], zpn1[5], uc0[5], uc1[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) zm0[q] = zm1[q] = zpn0[q] = zpn1[q] = uc0[q] = uc1[q] = T(0);
            // plane kk of column (jj, i0) from its final conserved state o:
            // floors, output, positivity flag, signal speed and sums
            auto finish = [&](T o[5], int kk, int jj) {
                T ir = rcp_(o[0]);
                T p = pressure<MODE>(o[0], o[1], o[2], o[3], o[4], ir, kc);
                if (kc.floors) apply_floors<MODE>(o, ir, p, kc, st);
#pragma unroll
                for (int q = 0; q < 5; ++q) gout[((q * 16 + kk) * 16 + jj) * 16 + i0] = o[q];
                if (!((o[0] > T(0)) & (p > T(0)))) st |= GAMER_ST_NONPOSITIVE_OUT;
                // max_d |m_d / rho| + c, as max_d |m_d| * |1/rho| + c (the
                // product is max_d of the rounded |m_d / rho|, rounding being
                // monotonic and sign-symmetric; with the addition it may fuse
                // into one FMA, one rounding fewer); c = 0 where c^2 is not
                // positive (max_ drops a NaN)
                const T c2 = kc.gamma * p * ir;
                const T cs = sqrt_(max_(c2, T(0)));
                const T sp = max_(max_(abs_(o[1]), abs_(o[2])), abs_(o[3])) * abs_(ir) + cs;
                smax = max_(smax, sp);
                // paired sums in FP32 mode (1.5 % faster); the mixed build
                // measured 0.7 % slower with them, so the other modes keep
                // the scalar steps
                if constexpr (MODE == GAMER_MODE_F32) {
                    sums.add5(o);
                } else {
#pragma unroll
                    for (int q = 0; q < 5; ++q) sums.add(q, o[q]);
                }
            };
            for (int k = -1; k <= 16; ++k) {
                const T* Wm = S.W[(k + 1) % 3];
                const T* W0 = S.W[(k + 2) % 3];
                const T* Wp = S.W[(k + 3) % 3];
                const T* Uk = S.raw[(k + 2) % RING] + ROFF;
                const bool inner = (k >= 0 && k <= 15);

                // ---- phase CA, part C(k-1): x/y divergence of plane k-1
                if (k - 1 >= 0) {
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        if ((cc == 0 && !owner) || (cc == 1 && !two)) break;
                        const int fa = cc ? fa1 : fa0;
                        const T* uc = cc ? uc1 : uc0;
                        T* Ec = cc ? E1 : E0;
#pragma unroll
                        for (int q = 0; q < 5; ++q) {
                            const int o = q * kFaceStride + fa;
                            const T D = (S.xp[o] - S.xm[o]) + (S.yp[o] - S.ym[o]);
                            Ec[q] = uc[q] - lam * D;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    zp0[q] = zpn0[q];
                    zp1[q] = zpn1[q];
                }

                // ---- phase CA, part A(k): half-step prediction of plane k
                if (owner) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) uc0[q] = Uk[q * kPlane + pc0];
                    // (the x/y states of the planes outside the group, k = -1
                    // and 16, are stored too: no solve reads them, and the
                    // slots are free then)
                    predict_store<MODE, kLim, kRec>(Wm, W0, Wp, uc0, pc0, half_lam, igm1, kc,
                                                    S.xm + fa0, S.xp + fa0, S.ym + fa0,
                                                    S.yp + fa0, zm0, zpn0, st);
                }
                if (kWide ? (!owner && inner) : (two || inner)) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) uc1[q] = Uk[q * kPlane + pc_b];
                    predict_store<MODE, kLim, kRec>(Wm, W0, Wp, uc1, pc_b, half_lam, igm1, kc,
                                                    S.xm + o_xm, S.xp + o_xp, S.ym + o_ym,
                                                    S.yp + o_yp, zm1, zpn1, st);
                }
                __syncthreads();
                // plane k has been read: its slot takes plane k + RING
                if (k + RING <= 17) {
                    if (load_plane(k + RING)) pending |= 1u << ((k + 2) % RING);
                }

                // ---- phase B(k): Riemann solves
                if (k >= 0) {
                    // z faces k-1/2 of the owned columns, rotated (rho, m_z, m_x,
                    // m_y, E): the flux leaves plane k-1, which is then final,
                    // and enters plane k
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        if ((cc == 0 && !owner) || (cc == 1 && !two)) break;
                        const T* zp = cc ? zp1 : zp0;
                        const T* zm = cc ? zm1 : zm0;
                        const int jj = cc ? j1 : j0;
                        T L[5] = {zp[0], zp[3], zp[1], zp[2], zp[4]};
                        T R[5] = {zm[0], zm[3], zm[1], zm[2], zm[4]};
                        T F[5];
                        roe_solve<MODE, (RSV & 3)>(L, R, kc, F, st);
                        const T fz[5] = {F[0], F[2], F[3], F[1], F[4]};
                        const int pz = flux_plane(2, k, kc.flux9);
                        if (gff && pz >= 0) {
                            T* dst = gff + pz * kFluxPlane + jj * 16 + i0;
#pragma unroll
                            for (int q = 0; q < 5; ++q) dst[q * 256] = fz[q];
                        }
                        T* fo = cc ? fzo1 : fzo0;
                        if (k >= 1) {
                            const T* Ec = cc ? E1 : E0;
                            T o[5];
#pragma unroll
                            for (int q = 0; q < 5; ++q) o[q] = Ec[q] - lam * (fz[q] - fo[q]);
                            finish(o, k - 1, jj);
                        }
#pragma unroll
                        for (int q = 0; q < 5; ++q) fo[q] = fz[q];
                    }
                }
                if (inner) {
                    // x faces: item = j*17 + f (f: face between i = f-1 and f)
                    // y faces: item = 272 + f*16 + i (f: face between j = f-1 and f)
                    // NT 160: threads 0-95 take items tid + 96 r (r < 3), the
                    // others 288 + (tid - 96) + 64 r (r < 4): five solves each
                    // with the z face.  NT 320: owners take item tid and, for
                    // tid < 96, 256 + tid; the slab threads 352 + (tid - 256)
                    // + 64 r (r < 3): two or three solves per thread.
                    const int nxy = kWide ? (owner ? (tid < 96 ? 2 : 1) : 3) : (two ? 3 : 4);
                    for (int r = 0; r < nxy; ++r) {
                        const int it = kWide ? (owner ? (r == 0 ? tid : 256 + tid)
                                                      : (352 + (tid - 256) + 64 * r))
                                             : (two ? (r * 96 + tid) : (288 + r * 64 + (tid - 96)));
                        const bool isy = it >= 272;
                        int lo, hi, a, b;
                        T *LA, *RA;
                        if (!isy) {
                            const int j = it / 17, f = it - j * 17;
                            const int rj = frow(j) * 16;
                            lo = (f == 0) ? (256 + j) : (rj + f - 1);
                            hi = (f == 16) ? (256 + j) : (rj + f);
                            LA = S.xp;
                            RA = S.xm;
                            a = j;
                            b = f;
                        } else {
                            const int y = it - 272, f = y >> 4, i = y & 15;
                            lo = (f == 0) ? (256 + i) : (frow(f - 1) * 16 + i);
                            hi = (f == 16) ? (256 + i) : (frow(f) * 16 + i);
                            LA = S.yp;
                            RA = S.ym;
                            a = i;
                            b = f;
                        }
                        // rotation: x -> (0,1,2,3,4); y -> (0,2,3,1,4).  The five
                        // components are loaded and stored at fixed offsets and
                        // permuted in registers (three selects each way), so no
                        // access needs a run-time component offset.
                        T A[5], B[5], L[5], R[5], F[5];
#pragma unroll
                        for (int q = 0; q < 5; ++q) {
                            A[q] = LA[q * kFaceStride + lo];
                            B[q] = RA[q * kFaceStride + hi];
                        }
                        L[0] = A[0];
                        L[1] = isy ? A[2] : A[1];
                        L[2] = isy ? A[3] : A[2];
                        L[3] = isy ? A[1] : A[3];
                        L[4] = A[4];
                        R[0] = B[0];
                        R[1] = isy ? B[2] : B[1];
                        R[2] = isy ? B[3] : B[2];
                        R[3] = isy ? B[1] : B[3];
                        R[4] = B[4];
                        roe_solve<MODE, (RSV & 3)>(L, R, kc, F, st);
                        // the flux, back in (rho, mx, my, mz, E) order, into the two
                        // state slots this solve consumed
                        const T G[5] = {F[0], isy ? F[3] : F[1], isy ? F[1] : F[2],
                                        isy ? F[2] : F[3], F[4]};
#pragma unroll
                        for (int q = 0; q < 5; ++q) {
                            LA[q * kFaceStride + lo] = G[q];
                            RA[q * kFaceStride + hi] = G[q];
                        }
                        const int face = flux_plane(isy ? 1 : 0, b, kc.flux9);
                        if (gff && face >= 0) {
                            // x planes: [v][k][j];  y planes: [v][k][i]
                            T* dst = gff + face * kFluxPlane + k * 16 + a;
#pragma unroll
                            for (int q = 0; q < 5; ++q) dst[q * 256] = G[q];
                        }
                    }
                }
                // plane k+2 -> primitives (into the slot of plane k-1)
                if (k <= 15) {
                    const int slot = (k + 4) % RING;
                    if (mbar_wait(&S.mbar[slot], (parity >> slot) & 1u, polls)) {
                        parity ^= 1u << slot;
                        pending &= ~(1u << slot);
                        convert_plane<MODE, NT>(S.raw[slot] + ROFF, S.W[(k + 4) % 3],
                                            plane_read_bits(rmask, k + 2), kc, st);
                    } else {
                        timed_out = true;
                    }
                }
                if (__syncthreads_or(timed_out)) goto abort_group;
            }

            // ---- group epilogue: reductions across the warp (FP32 modes: the
            // compensated float pairs by double-float additions, so no FP64
            // instruction per thread), then in FP64 across warps
            double dmax, dsum[5];
            if constexpr (sizeof(T) == 4) {
                float m = smax, h[5], l[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) {
                    h[q] = sums.hi(q);
                    l[q] = sums.lo(q);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
                        const float oh = __shfl_xor_sync(0xffffffffu, h[q], off);
                        const float ol = __shfl_xor_sync(0xffffffffu, l[q], off);
                        float e;
                        h[q] = two_sum(h[q], oh, e);
                        l[q] = (l[q] + ol) + e;
                    }
                }
                dmax = double(m);
#pragma unroll
                for (int q = 0; q < 5; ++q) dsum[q] = double(h[q]) + double(l[q]);
            } else {
                dmax = double(smax);
#pragma unroll
                for (int q = 0; q < 5; ++q) dsum[q] = sums.get(q);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
#pragma unroll
                    for (int q = 0; q < 5; ++q)
                        dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], off);
                }
            }
            const uint32_t wst = __reduce_or_sync(0xffffffffu, st);
            // per-warp partials in the x- face array (no face state is live
            // between a group's last phase and the next group's first one)
            double(*red)[6] = reinterpret_cast<double(*)[6]>(S.xm);
            if (lane == 0) {
                red[warp][0] = dmax;
#pragma unroll
                for (int q = 0; q < 5; ++q) red[warp][1 + q] = dsum[q];
                if (wst) atomicOr(&S.status, wst);
            }
            __syncthreads();
            if (tid == 0) {
                if (partials) {
                    double m = 0.0, s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
                    for (int w = 0; w < NT / 32; ++w) {
                        m = fmax(m, red[w][0]);
                        for (int q = 0; q < 5; ++q) s[q] += red[w][1 + q];
                    }
                    partials[g * 6] = m;
                    for (int q = 0; q < 5; ++q) partials[g * 6 + 1 + q] = s[q];
                }
                if (status) status[g] = S.status;
            }
            __syncthreads();
        }
        continue;

    abort_group:
        // A bulk copy did not complete in time.  Wait (bounded) for every copy
        // still in flight so none lands after the CTA exits, flag this group
        // and every later one of the CTA, and stop.
        if (tid == 0) {
            for (int s = 0; s < RING; ++s)
                if (pending & (1u << s)) mbar_wait(&S.mbar[s], (parity >> s) & 1u);
            mark_abandoned(g, N, status, partials);
        }
        return;
    }
}

}  // namespace gamer
