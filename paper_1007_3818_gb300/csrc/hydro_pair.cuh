// hydro_pair.cuh -- the patch-group step with two independent problems in
// flight per thread (instruction-level parallelism for a latency-bound step).
//
// Same scheme, data path and z-marching schedule as hydro_step_kernel (see
// hydro_kernel.cuh).  The difference is how the work of a plane is spread:
//  * every thread predicts its two cells together: the branch-free Hancock
//    core of both runs as one block of independent instructions, the rare
//    fallback after it;
//  * the 800 Riemann problems of a plane are uniform items -- 256 z faces
//    (states kept in shared memory instead of owner registers), 272 x faces,
//    272 y faces -- of which thread t takes items r*160 + t, r = 0..4, solved
//    as two interleaved pairs and one single through the branch-free Roe path;
//    HLLE recomputes out of line when a fallback is needed;
//  * the limiter is a compile-time choice on this path.
// The extra shared memory (z states, z fluxes) and registers size it for two
// CTAs per SM (FP32) or one (FP64).
#pragma once

#include "hydro_kernel.cuh"

namespace gamer {

constexpr int kOutStride = 800;  // flux slots: x [0,272), y [272,544), z [544,800)

template <class T>
struct alignas(16) SmemPair {
    T raw[2][5 * kPlane];  // TMA ring of conserved input planes
    T W[3][5 * kPlane];    // primitive planes
    // face states, each [5][kFaceStride]: 0 x-, 1 x+, 2 y-, 3 y+,
    // 4/5 z+ of alternate planes, 6 z-
    T fs[7][5 * kFaceStride];
    T flux[5 * kOutStride];
    double red[kThreads / 32][6];
    uint64_t mbar[2];
    uint32_t status;
};

// Where Riemann item `it` of plane k reads its left / right states (offsets in
// SmemPair::fs, component 0), writes its flux (offset in SmemPair::flux), how
// its components rotate, and which group face (or none) it belongs to.
struct ItemDesc {
    int lo, hi, wr, c1, c2, c3, face, foff;
};

__device__ __forceinline__ ItemDesc item_desc(int it, int k, int flux9) {
    constexpr int A = 5 * kFaceStride;  // one face-state array
    ItemDesc d;
    if (it < 256) {
        // z face k-1/2 of the column stored at slot it
        d.lo = (4 + ((k - 1) & 1)) * A + it;
        d.hi = 6 * A + it;
        d.wr = 544 + it;
        d.c1 = 3;
        d.c2 = 1;
        d.c3 = 2;
        d.face = flux_plane(2, k, flux9);
        d.foff = frow(it >> 4) * 16 + (it & 15);  // [j][i]
    } else if (it < 256 + 272) {
        // x face f of row j (between i = f-1 and f)
        const int x = it - 256, j = x / 17, f = x - j * 17;
        const int rj = frow(j) * 16;
        d.lo = 1 * A + ((f == 0) ? (256 + j) : (rj + f - 1));
        d.hi = 0 * A + ((f == 16) ? (256 + j) : (rj + f));
        d.wr = (f == 16) ? (256 + j) : (rj + f);
        d.c1 = 1;
        d.c2 = 2;
        d.c3 = 3;
        d.face = flux_plane(0, f, flux9);
        d.foff = k * 16 + j;  // [k][j]
    } else {
        // y face f of column i (between j = f-1 and f)
        const int y = it - 528, f = y >> 4, i = y & 15;
        d.lo = 3 * A + ((f == 0) ? (256 + i) : (frow(f - 1) * 16 + i));
        d.hi = 2 * A + ((f == 16) ? (256 + i) : (frow(f) * 16 + i));
        d.wr = 272 + ((f == 16) ? (256 + i) : (frow(f) * 16 + i));
        d.c1 = 2;
        d.c2 = 3;
        d.c3 = 1;
        d.face = flux_plane(1, f, flux9);
        d.foff = k * 16 + i;  // [k][i]
    }
    return d;
}

template <class T>
__device__ __forceinline__ void item_load(const T* fs, const ItemDesc& d, T L[5], T R[5]) {
    L[0] = fs[d.lo];
    L[1] = fs[d.lo + d.c1 * kFaceStride];
    L[2] = fs[d.lo + d.c2 * kFaceStride];
    L[3] = fs[d.lo + d.c3 * kFaceStride];
    L[4] = fs[d.lo + 4 * kFaceStride];
    R[0] = fs[d.hi];
    R[1] = fs[d.hi + d.c1 * kFaceStride];
    R[2] = fs[d.hi + d.c2 * kFaceStride];
    R[3] = fs[d.hi + d.c3 * kFaceStride];
    R[4] = fs[d.hi + 4 * kFaceStride];
}

template <class T>
__device__ __forceinline__ void item_store(T* flux, T* gff, const ItemDesc& d, const T F[5]) {
    flux[d.wr] = F[0];
    flux[d.wr + d.c1 * kOutStride] = F[1];
    flux[d.wr + d.c2 * kOutStride] = F[2];
    flux[d.wr + d.c3 * kOutStride] = F[3];
    flux[d.wr + 4 * kOutStride] = F[4];
    if (gff && d.face >= 0) {
        T* dst = gff + d.face * kFluxPlane + d.foff;
        dst[0] = F[0];
        dst[d.c1 * 256] = F[1];
        dst[d.c2 * 256] = F[2];
        dst[d.c3 * 256] = F[3];
        dst[4 * 256] = F[4];
    }
}

template <int MODE, int MINB, int LIM>
__global__ void __launch_bounds__(kThreads, MINB)
    hydro_pair_kernel(const typename Prec<MODE>::T* __restrict__ in,
                      typename Prec<MODE>::T* __restrict__ out,
                      typename Prec<MODE>::T* __restrict__ face_flux,
                      const double* __restrict__ dt, const double* __restrict__ dh,
                      uint32_t* __restrict__ status, double* __restrict__ partials, int64_t N,
                      KConst<typename Prec<MODE>::T, typename Prec<MODE>::P> kc) {
    using T = typename Prec<MODE>::T;
    extern __shared__ __align__(128) unsigned char smem_bytes[];
    SmemPair<T>& S = *reinterpret_cast<SmemPair<T>*>(smem_bytes);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const uint32_t rmask = read_cell_mask();

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) mbar_init(&S.mbar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t parity = 0, pending = 0;

    // owned columns as in hydro_step_kernel: warp w owns row pair w (c0) and,
    // for w < 3, row pair w + 5 (c1); warps 3-4 predict a face-slab cell as
    // their second item
    const bool two = tid < 96;
    const int i0 = lane & 15, hb = (lane >> 4) * 4;
    const int j0 = (warp & 3) + ((warp >> 2) << 3) + hb;
    const int j1 = ((warp + 5) & 3) + (((warp + 5) >> 2) << 3) + hb;
    const int pc0 = (j0 + 2) * 20 + (i0 + 2);
    const int fa0 = frow(j0) * 16 + i0, fa1 = frow(j1) * 16 + i0;
    const int sl = tid - 96, side = sl >> 4, st_ = sl & 15;
    const int si = (side == 0) ? -1 : (side == 1) ? 16 : st_;
    const int sj = (side == 2) ? -1 : (side == 3) ? 16 : st_;
    const int pc_b = two ? (j1 + 2) * 20 + (i0 + 2) : (sj + 2) * 20 + (si + 2);
    // store offsets of the second item (slab cells' unused faces -> 272..287)
    const int o_xm = two ? fa1 : (side == 1 ? 256 + st_ : 272 + st_);
    const int o_xp = two ? fa1 : (side == 0 ? 256 + st_ : 272 + st_);
    const int o_ym = two ? fa1 : (side == 3 ? 256 + st_ : 272 + st_);
    const int o_yp = two ? fa1 : (side == 2 ? 256 + st_ : 272 + st_);
    const int o_z = two ? fa1 : 272 + st_;
    const T igm1 = T(1) / kc.gm1;

    for (int64_t g = blockIdx.x; g < N; g += gridDim.x) {
        const T* gin = in + g * 40000;
        T* gout = out + g * 20480;
        T* gff = face_flux ? face_flux + g * (kc.flux9 ? 9 : 6) * kFluxPlane : nullptr;
        const double dtg = dt[g], dhg = dh[g];
        const T lam = static_cast<T>(dtg / dhg);
        const T half_lam = T(0.5) * lam;
        uint32_t st = 0;
        if (tid == 0) {
            S.status = 0;
            if (!(isfinite(dtg) && isfinite(dhg) && dtg >= 0.0 && dhg > 0.0))
                st |= GAMER_ST_BAD_INPUT;
            issue_plane(S, gin, -2);
            issue_plane(S, gin, -1);
        }
        pending |= 3u;
        bool timed_out = false;
        if (mbar_wait(&S.mbar[0], parity & 1u)) {
            parity ^= 1u;
            pending &= ~1u;
            convert_plane<MODE>(S.raw[0], S.W[0], plane_read_bits(rmask, -2), kc, st);
        } else {
            timed_out = true;
        }
        if (__syncthreads_or(timed_out)) goto abort_group;
        if (tid == 0) issue_plane(S, gin, 0);
        pending |= 1u;
        for (int s = 1; s >= 0; --s) {
            if (!timed_out && mbar_wait(&S.mbar[s], (parity >> s) & 1u)) {
                parity ^= 1u << s;
                pending &= ~(1u << s);
                convert_plane<MODE>(S.raw[s], S.W[(s == 1) ? 1 : 2],
                                    plane_read_bits(rmask, (s == 1) ? -1 : 0), kc, st);
            } else {
                timed_out = true;
            }
        }
        if (__syncthreads_or(timed_out)) goto abort_group;

        {
            T fzo0[5], fzo1[5], E0[5], E1[5], uc0[5], uc1[5];
#pragma unroll
            for (int q = 0; q < 5; ++q)
                fzo0[q] = fzo1[q] = E0[q] = E1[q] = uc0[q] = uc1[q] = T(0);
            T smax = T(0);
            SumAcc<T> sums;

            for (int k = -1; k <= 17; ++k) {
                const T* Wm = S.W[(k + 1) % 3];
                const T* W0 = S.W[(k + 2) % 3];
                const T* Wp = S.W[(k + 3) % 3];
                const T* Uk = S.raw[(k + 2) & 1];
                const bool inner = (k >= 0 && k <= 15);

                // ---- phase CA, part C(k-1): finish plane k-2, set up plane k-1
                const bool fin = (k - 1 >= 1), setup = (k - 1 >= 0 && k - 1 <= 15);
                if (fin || setup) {
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        if (cc == 1 && !two) break;
                        const int jj = cc ? j1 : j0;
                        const int fa = cc ? fa1 : fa0;
                        T* Ec = cc ? E1 : E0;
                        T* fo = cc ? fzo1 : fzo0;
                        const T* uc = cc ? uc1 : uc0;
                        T fn[5];
#pragma unroll
                        for (int q = 0; q < 5; ++q) fn[q] = S.flux[q * kOutStride + 544 + fa];
                        if (fin) {
                            const int kk = k - 2;
                            T o[5];
#pragma unroll
                            for (int q = 0; q < 5; ++q) o[q] = Ec[q] - lam * (fn[q] - fo[q]);
                            T ir = rcp_(o[0]);
                            T p = pressure<MODE>(o[0], o[1], o[2], o[3], o[4], ir, kc);
                            if (kc.floors) apply_floors<MODE>(o, ir, p, kc, st);
#pragma unroll
                            for (int q = 0; q < 5; ++q)
                                gout[((q * 16 + kk) * 16 + jj) * 16 + i0] = o[q];
                            if (!(o[0] > T(0)) || !(p > T(0))) st |= GAMER_ST_NONPOSITIVE_OUT;
                            const T c2 = kc.gamma * p * ir;
                            const T cs = (c2 > T(0)) ? sqrt_(c2) : T(0);
                            const T sp =
                                max_(max_(abs_(o[1] * ir), abs_(o[2] * ir)), abs_(o[3] * ir)) +
                                cs;
                            if (sp > smax) smax = sp;
#pragma unroll
                            for (int q = 0; q < 5; ++q) sums.add(q, o[q]);
                        }
                        if (setup) {
                            const int rxp = (i0 == 15) ? (256 + jj) : (fa + 1);
                            const int ryp =
                                272 + ((jj == 15) ? (256 + i0) : (frow(jj + 1) * 16 + i0));
#pragma unroll
                            for (int q = 0; q < 5; ++q) {
                                const T* fq = S.flux + q * kOutStride;
                                const T D = (fq[rxp] - fq[fa]) + (fq[ryp] - fq[272 + fa]);
                                Ec[q] = uc[q] - lam * D;
                                fo[q] = fn[q];
                            }
                        }
                    }
                }
                if (k == 17) break;

                // ---- phase CA, part A(k): both cells of the thread together
                {
                    T fa_[6][5], fb_[6][5], dua[5], dub[5];
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
                        uc0[q] = Uk[q * kPlane + pc0];
                        uc1[q] = Uk[q * kPlane + pc_b];
                    }
                    const bool oka =
                        predict_core<MODE, LIM>(Wm, W0, Wp, pc0, half_lam, igm1, kc, fa_, dua);
                    // a slab cell outside planes 0..15 is computed (one code
                    // path) but not part of the method: no status from it
                    const bool okb =
                        predict_core<MODE, LIM>(Wm, W0, Wp, pc_b, half_lam, igm1, kc, fb_, dub) ||
                        !(two || inner);
                    if (!(oka && okb)) {
                        st |= GAMER_ST_PREDICTOR_FALLBACK;
                        if (!oka) predict_fallback(uc0, dua, kc, fa_);
                        if (!okb) predict_fallback(uc1, dub, kc, fb_);
                    }
                    T* F0 = S.fs[0];
                    T* F1 = S.fs[1];
                    T* F2 = S.fs[2];
                    T* F3 = S.fs[3];
                    T* Fzp = S.fs[4 + (k & 1)];
                    T* Fzm = S.fs[6];
#pragma unroll
                    for (int q = 0; q < 5; ++q) {
                        if (inner) {
                            F0[q * kFaceStride + fa0] = fa_[0][q];
                            F1[q * kFaceStride + fa0] = fa_[1][q];
                            F2[q * kFaceStride + fa0] = fa_[2][q];
                            F3[q * kFaceStride + fa0] = fa_[3][q];
                            F0[q * kFaceStride + o_xm] = fb_[0][q];
                            F1[q * kFaceStride + o_xp] = fb_[1][q];
                            F2[q * kFaceStride + o_ym] = fb_[2][q];
                            F3[q * kFaceStride + o_yp] = fb_[3][q];
                        }
                        Fzm[q * kFaceStride + fa0] = fa_[4][q];
                        Fzp[q * kFaceStride + fa0] = fa_[5][q];
                        Fzm[q * kFaceStride + o_z] = fb_[4][q];
                        Fzp[q * kFaceStride + o_z] = fb_[5][q];
                    }
                }
                __syncthreads();
                if (k <= 15) {
                    if (tid == 0) issue_plane(S, gin, k + 2);
                    pending |= 1u << ((k + 2) & 1);
                }

                // ---- phase B(k): items r*160 + tid, r = 0..4, in pairs
                {
                    const T* FS = S.fs[0];
#pragma unroll 1
                    for (int r = 0; r < 5; r += 2) {
                        const int ia = r * kThreads + tid, ib = (r + 1) * kThreads + tid;
                        const bool va = (ia < 256) ? (k >= 0) : inner;
                        const bool vb = (r + 1 < 5) && ((ib < 256) ? (k >= 0) : inner);
                        if (va && vb) {
                            const ItemDesc da = item_desc(ia, k, kc.flux9),
                                           db = item_desc(ib, k, kc.flux9);
                            T La[5], Ra[5], Lb[5], Rb[5], Fa[5], Fb[5];
                            item_load(FS, da, La, Ra);
                            item_load(FS, db, Lb, Rb);
                            const bool fba = roe_main<MODE>(La, Ra, kc, Fa);
                            const bool fbb = roe_main<MODE>(Lb, Rb, kc, Fb);
                            if (fba || fbb) {
                                if (fba) hlle_apply<MODE>(La, Ra, kc, Fa, st);
                                if (fbb) hlle_apply<MODE>(Lb, Rb, kc, Fb, st);
                            }
                            item_store(S.flux, gff, da, Fa);
                            item_store(S.flux, gff, db, Fb);
                        } else if (va) {
                            const ItemDesc da = item_desc(ia, k, kc.flux9);
                            T La[5], Ra[5], Fa[5];
                            item_load(FS, da, La, Ra);
                            if (roe_main<MODE>(La, Ra, kc, Fa)) hlle_apply<MODE>(La, Ra, kc, Fa, st);
                            item_store(S.flux, gff, da, Fa);
                        }
                    }
                }
                if (k <= 15) {
                    const int slot = (k + 2) & 1;
                    if (mbar_wait(&S.mbar[slot], (parity >> slot) & 1u)) {
                        parity ^= 1u << slot;
                        pending &= ~(1u << slot);
                        convert_plane<MODE>(S.raw[slot], S.W[(k + 4) % 3],
                                            plane_read_bits(rmask, k + 2), kc, st);
                    } else {
                        timed_out = true;
                    }
                }
                if (__syncthreads_or(timed_out)) goto abort_group;
            }

            double dmax = double(smax);
            double dsum[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) dsum[q] = sums.get(q);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
#pragma unroll
                for (int q = 0; q < 5; ++q) dsum[q] += __shfl_xor_sync(0xffffffffu, dsum[q], off);
            }
            const uint32_t wst = __reduce_or_sync(0xffffffffu, st);
            if (lane == 0) {
                S.red[warp][0] = dmax;
#pragma unroll
                for (int q = 0; q < 5; ++q) S.red[warp][1 + q] = dsum[q];
                if (wst) atomicOr(&S.status, wst);
            }
            __syncthreads();
            if (tid == 0) {
                if (partials) {
                    double m = 0.0, s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
                    for (int w = 0; w < kThreads / 32; ++w) {
                        m = fmax(m, S.red[w][0]);
                        for (int q = 0; q < 5; ++q) s[q] += S.red[w][1 + q];
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
        // as hydro_step_kernel: drain the copies in flight, flag this group and
        // every later one of the CTA, stop
        if (tid == 0) {
            for (int s = 0; s < 2; ++s)
                if (pending & (1u << s)) mbar_wait(&S.mbar[s], (parity >> s) & 1u);
            mark_abandoned(g, N, status, partials);
        }
        return;
    }
}

}  // namespace gamer
