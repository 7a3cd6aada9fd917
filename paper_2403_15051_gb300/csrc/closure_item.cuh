// The closure of the FDLB stage as device code shared by the closure kernel and the
// persistent step kernel.  Results per cell do not depend on how cells are grouped into items,
// nor on the number of warps above four, so both kernels produce identical records.
#pragma once

#include "device_common.cuh"
#include "kernels.cuh"
#include "kernels_decl.h"

namespace fdlb {

constexpr int kClosureThreads = 128;  // the closure kernel's block; the order of the wall sums
constexpr int kClosureWarps = kClosureThreads / 32;

// ------------------------------------------------------------------------------ closure
// Per cell, once per stage.  A cell item covers up to kClosureCells own cells and the two
// stencil cells on each side ("reach", at most 32 cells); one lane per reach cell for the
// macroscopic fields, so that no arithmetic is spread thinly over lanes:
//  * n, u, T (Eq. macro_def) of every reach cell from the FP64 raw sums, in the wide type
//    (FP64, or double-float for FP32 populations); q and P_12 of the own cells;
//  * warps 1..3 meanwhile sum the FM bands (Eq. fm, n = 0 outside the domain) from the slice
//    densities staged in shared memory; chi = chi_SET(pi sigma^3 nbar / 6) (Eqs. chi, chi_ret),
//    or chi at the local density;
//  * the J1 gradients (Eq. j1) as stencils of logarithms of ratios to the own cell, exact
//    because the stencil weights sum to zero:  sum_q w_q ln(n_q^2 chi_q T_q) = sum_q w_q
//    [2 log1p(dn_q / n) + log1p(dchi_q / chi) + log1p(dT_q / T)], the differences taken in the
//    wide type; velocity gradients from wide differences;
//  * mu, Pr, tau (Eqs. viscosity, prandtl, tau), the covariant strain and the Shakhov
//    coefficient; the recurrences of the expansion coefficients of the equilibria (Sec. III.C;
//    warp = axis, lane = cell) and the per-axis vectors g_2, g_R, g_3 (whole block).
// chi and nbar of the own cells also go to a small side buffer, from which ca_kernel forms the
// FP64 closure record of the moments and closure queries.
// Wall items (kind 1 + side, part): the block sums the outgoing flux of one part of the momenta
// at one wall; the stage kernel forms n_w from the parts (diffuse walls, zero net mass flux).
// Output: the per-cell collision record in the populations' precision, [20 scalars | g_2 | g_R
// | g_3].
__host__ __device__ inline int closure_tab_elems(int nR, int n2, int n3) {
    return 4 * kMaxE + 2 + (nR + n2 + n3) * kMaxE + 2 * nR + n2 + n3;
}
// dynamic shared memory: [staged band rows | tables | band-union densities]
__host__ __device__ inline size_t closure_smem_bytes(int nR, int n2, int n3, int max_union, int wst_elems, int tsize) {
    return (size_t)wst_elems * tsize + ((size_t)closure_tab_elems(nR, n2, n3) + (size_t)max_union) * tsize + 16;
}

// Position q of the five-point derivative stencil of cell c (the stencils of stencil5).
template <typename R>
__device__ __forceinline__ void stencil5_at(int c, int N, int q, int& cell, R& w) {
    const R k = R(1) / R(12);
    if (c >= 2 && c <= N - 3) {
        cell = c - 2 + q;
        w = q == 0 ? k : q == 1 ? R(-8) * k : q == 2 ? R(0) : q == 3 ? R(8) * k : -k;
    } else if (c == 0) {
        cell = q;
        w = q == 0 ? R(-25) * k : q == 1 ? R(48) * k : q == 2 ? R(-36) * k : q == 3 ? R(16) * k : R(-3) * k;
    } else if (c == 1) {
        cell = q;
        w = q == 0 ? R(-3) * k : q == 1 ? R(-10) * k : q == 2 ? R(18) * k : q == 3 ? R(-6) * k : k;
    } else if (c == N - 2) {
        cell = N - 1 - q;
        w = q == 0 ? R(3) * k : q == 1 ? R(10) * k : q == 2 ? R(-18) * k : q == 3 ? R(6) * k : -k;
    } else {
        cell = N - 1 - q;
        w = q == 0 ? R(25) * k : q == 1 ? R(-48) * k : q == 2 ? R(36) * k : q == 3 ? R(-16) * k : R(3) * k;
    }
}

template <typename T>
__device__ __forceinline__ T inst_param(double d, float f) {
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}


template <typename T>
struct ClosureTabs {
    T *ha, *hb, *ihb, *h0t, *GR, *G2, *G3, *pRt, *wRt, *w2t, *w3t;
};

// The closure's tables in shared memory (closure_tab_elems elements from `base`), filled by the
// block's threads; the caller synchronises.
template <typename T>
__device__ ClosureTabs<T> closure_tables(T* base, const void* tabTv, const MomSet& M, int tid, int NT) {
    const int nR = M.nR, n2 = M.n2, n3 = M.n3;
    ClosureTabs<T> t;
    t.ha = base;
    t.hb = t.ha + kMaxE;
    t.ihb = t.hb + kMaxE + 1;  // 1 / hb
    t.h0t = t.ihb + kMaxE + 1;
    t.GR = t.h0t + kMaxE;
    t.G2 = t.GR + nR * kMaxE;
    t.G3 = t.G2 + n2 * kMaxE;
    t.pRt = t.G3 + n3 * kMaxE;
    t.wRt = t.pRt + nR;
    t.w2t = t.wRt + nR;
    t.w3t = t.w2t + n2;
    const T* tabT = reinterpret_cast<const T*>(tabTv);
    for (int e = tid; e < kMaxE; e += NT) {
        t.ha[e] = tabT[M.o_ha + e];
        t.h0t[e] = tabT[M.o_h0 + e];
    }
    for (int e = tid; e <= kMaxE; e += NT) {
        t.hb[e] = tabT[M.o_hb + e];
        t.ihb[e] = t.hb[e] != T(0) ? T(1) / t.hb[e] : T(0);
    }
    for (int e = tid; e < nR * kMaxE; e += NT) t.GR[e] = tabT[M.o_GR + e];
    for (int e = tid; e < n2 * kMaxE; e += NT) t.G2[e] = tabT[M.o_G2 + e];
    for (int e = tid; e < n3 * kMaxE; e += NT) t.G3[e] = tabT[M.o_G3 + e];
    for (int e = tid; e < nR; e += NT) {
        t.pRt[e] = tabT[M.o_pR + e];
        t.wRt[e] = tabT[M.o_wR + e];
    }
    for (int e = tid; e < n2; e += NT) t.w2t[e] = tabT[M.o_w2 + e];
    for (int e = tid; e < n3; e += NT) t.w3t[e] = tabT[M.o_w3 + e];
    return t;
}

// One thread's share of part `part` (of P) of the outgoing flux through a wall (side 0: inner,
// 1: outer): the sum over the outgoing momenta of |p_R| w vhat, vhat the WENO5 value at the
// wall face from the wall cell, its neighbour and the cubic extrapolation outside.  `wall` points
// at the populations of the wall cell (cell 0 or N-1), `st` is the step to the next cell inward
// (the rows may be in global or shared memory).  `tl` is the thread's index in a block of
// kClosureThreads threads, whose order of the sums this follows.
template <typename T>
__device__ T wall_flux_partial(const T* wall, long long st, const MomSet& M, const ClosureTabs<T>& tb, int side, int part,
                               int P, int tl) {
    const int Np = M.Np, nR = M.nR, n2 = M.n2, NT = kClosureThreads;
    const int mlo = (int)((long long)Np * part / P), mhi = (int)((long long)Np * (part + 1) / P);
    const long long base = 0;
    T acc = T(0);
    for (int m0 = mlo + tl; m0 < mhi; m0 += 4 * NT) {
        // four momenta per pass so that their sixteen loads are in flight together
        T fv[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = min(m0 + u * NT, mhi - 1);
#pragma unroll
            for (int r = 0; r < 4; ++r) fv[u][r] = wall[base + m + r * st];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = m0 + u * NT;
            if (m >= mhi) continue;
            const int k = m / (nR * n2), rem = m % (nR * n2), i = rem / n2, j = rem % n2;
            const T pr = tb.pRt[i];
            if (side == 0 ? !(pr < T(0)) : !(pr > T(0))) continue;
            if (M.reduced && k > 0) continue;  // the mass flux is phi's (chi = int p_z^2 f)
            const T wm = tb.wRt[i] * tb.w2t[j] * tb.w3t[k];
            const T iw = wm > (sizeof(T) == 4 ? T(1e-30) : T(0)) ? T(1) / wm : T(0);  // as the stage kernel
            const T f0 = fv[u][0], f1 = fv[u][1], f2 = fv[u][2], f3 = fv[u][3];
            const T g1 = T(4) * f0 - T(6) * f1 + T(4) * f2 - f3;
            const T g2 = T(10) * f0 - T(20) * f1 + T(15) * f2 - T(4) * f3;
            const T vh = weno5(f2 * iw, f1 * iw, f0 * iw, g1 * iw, g2 * iw);
            acc += fabs(pr) * wm * vh;
        }
    }
    return acc;
}

// A part of the wall flux from its four warp sums, in the closure kernel's order.
template <typename T>
__device__ __forceinline__ T wall_part_sum(const T* r) {
    return (r[0] + r[1]) + (r[2] + r[3]);
}

struct NoExtra {
    __device__ void operator()(int, int) const {}
};
struct NoAfterLoads {
    __device__ void operator()() const {}
};

// ---- the per-cell steps of the closure.  The item chain below (closure_cells) and the two
// kernels of the batch form (closure_band_kernel, closure_records_kernel) are made of these
// functions, so a cell's record is the same whichever form computes it.

// Raw sums of global cell `gc` over its slices, in the wide type: FP64, or for FP32 populations
// the double-float pairs the stage kernel stores beside the FP64 sums (no FP64 arithmetic).
template <typename T>
__device__ __forceinline__ void clo_load_sums(const ClosureArgs& A, long long gc, Wide<T> (&sv)[kSums]) {
    const int slices = A.slices;
    if constexpr (sizeof(T) == 4) {
        const float2* src = reinterpret_cast<const float2*>(A.sumsw) + gc * slices * kSums;
#pragma unroll
        for (int q = 0; q < kSums; ++q) {
            const float2 p = src[q];
            sv[q] = Wide<T>{p.x, p.y};
        }
        for (int sl = 1; sl < slices; ++sl)
#pragma unroll
            for (int q = 0; q < kSums; ++q) {
                const float2 p = src[sl * kSums + q];
                sv[q] = w_add(sv[q], Wide<T>{p.x, p.y});
            }
    } else {
        const double* src = A.sums + gc * slices * kSums;
#pragma unroll
        for (int q = 0; q < kSums; ++q) sv[q] = w_from(src[q], (T*)nullptr);
        for (int sl = 1; sl < slices; ++sl)
#pragma unroll
            for (int q = 0; q < kSums; ++q) sv[q] = w_add(sv[q], w_from(src[sl * kSums + q], (T*)nullptr));
    }
}

// n, u, T of a cell (Eq. macro_def) in the wide type, and the heat flux q in the populations'
// precision (it enters only the Shakhov factor and the diagnostics).
template <typename T>
__device__ __forceinline__ void clo_fields(const Wide<T> (&sv)[kSums], Wide<T>& n, Wide<T> (&u)[3], Wide<T>& Tc,
                                           T (&q)[3]) {
    using W = Wide<T>;
    n = sv[0];
    u[0] = w_div(sv[1], n);
    u[1] = w_div(sv[2], n);
    u[2] = w_div(sv[3], n);
    const W tr = w_add(w_add(sv[4], sv[5]), sv[6]);
    const W uu = w_add(w_add(w_mul(u[0], u[0]), w_mul(u[1], u[1])), w_mul(u[2], u[2]));
    Tc = w_div(w_sub(tr, w_mul(n, uu)), w_scale(n, T(3)));
    const T tn = w_hi(n), t0 = w_hi(u[0]), t1 = w_hi(u[1]), t2 = w_hi(u[2]), ttr = w_hi(tr), tuu = w_hi(uu);
    const T s4 = w_hi(sv[4]), s5 = w_hi(sv[5]), s6 = w_hi(sv[6]), s7 = w_hi(sv[7]), s8 = w_hi(sv[8]), s9 = w_hi(sv[9]);
    const T m0 = s4 * t0 + s7 * t1 + s8 * t2;
    const T m1 = s7 * t0 + s5 * t1 + s9 * t2;
    const T m2 = s8 * t0 + s9 * t1 + s6 * t2;
    q[0] = T(0.5) * (w_hi(sv[10]) - T(2) * m0 - t0 * ttr + T(2) * tn * tuu * t0);
    q[1] = T(0.5) * (w_hi(sv[11]) - T(2) * m1 - t1 * ttr + T(2) * tn * tuu * t1);
    q[2] = T(0.5) * (w_hi(sv[12]) - T(2) * m2 - t2 * ttr + T(2) * tn * tuu * t2);
}

// The FM band sum of one row (Eq. fm; a whole warp, every lane returns the sum): weights Wr[k]
// times densities dn(k), k < kmax, lane-strided into four accumulators (accumulator a takes
// k = lane + 32 a + 128 j in increasing j), then a butterfly.  The first loop takes two strides at
// a time so that sixteen loads per lane are in flight; the order of every accumulator is the same.
// Every term is an explicit fused multiply-add, so the sum does not depend on how the compiler
// contracts the expression in a given caller (clo_band_row2 must reproduce it bit for bit).
template <typename T, typename Dens>
__device__ __forceinline__ T clo_band_row(const T* Wr, const Dens& dn, int kmax, int lane) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    int k = lane;
    for (; k + 224 < kmax; k += 256) {
        T w[8], d[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            w[u] = Wr[k + 32 * u];
            d[u] = dn(k + 32 * u);
        }
        a0 = fma(w[0], d[0], a0);
        a1 = fma(w[1], d[1], a1);
        a2 = fma(w[2], d[2], a2);
        a3 = fma(w[3], d[3], a3);
        a0 = fma(w[4], d[4], a0);
        a1 = fma(w[5], d[5], a1);
        a2 = fma(w[6], d[6], a2);
        a3 = fma(w[7], d[7], a3);
    }
    for (; k + 96 < kmax; k += 128) {
        a0 = fma(Wr[k], dn(k), a0);
        a1 = fma(Wr[k + 32], dn(k + 32), a1);
        a2 = fma(Wr[k + 64], dn(k + 64), a2);
        a3 = fma(Wr[k + 96], dn(k + 96), a3);
    }
    for (; k < kmax; k += 32) a0 = fma(Wr[k], dn(k), a0);
    return warp_sum((a0 + a1) + (a2 + a3));
}

// Two band rows at once by one warp, each summed exactly as clo_band_row sums it, with the loads
// of both rows in flight together.  clo_band_row's eight-wide pass is two of its four-wide passes
// in the same order, so strides of 128 alone reproduce it; a row that has left a pass adds zeros
// there, which leaves its accumulators unchanged.
template <typename T, typename DensA, typename DensB>
__device__ __forceinline__ void clo_band_row2(const T* WrA, const DensA& dnA, int kmaxA, const T* WrB, const DensB& dnB,
                                              int kmaxB, int lane, T& totA, T& totB) {
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0), b0 = T(0), b1 = T(0), b2 = T(0), b3 = T(0);
    int ka = lane, kb = lane;
    for (;;) {
        const bool pa = ka + 96 < kmaxA, pb = kb + 96 < kmaxB;
        if (!pa && !pb) break;
        T wa[4], da[4], wb[4], db[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            wa[u] = pa ? WrA[ka + 32 * u] : T(0);
            da[u] = pa ? dnA(ka + 32 * u) : T(0);
            wb[u] = pb ? WrB[kb + 32 * u] : T(0);
            db[u] = pb ? dnB(kb + 32 * u) : T(0);
        }
        a0 = fma(wa[0], da[0], a0);
        a1 = fma(wa[1], da[1], a1);
        a2 = fma(wa[2], da[2], a2);
        a3 = fma(wa[3], da[3], a3);
        b0 = fma(wb[0], db[0], b0);
        b1 = fma(wb[1], db[1], b1);
        b2 = fma(wb[2], db[2], b2);
        b3 = fma(wb[3], db[3], b3);
        ka += pa ? 128 : 0;
        kb += pb ? 128 : 0;
    }
    for (;;) {
        const bool pa = ka < kmaxA, pb = kb < kmaxB;
        if (!pa && !pb) break;
        const T wa = pa ? WrA[ka] : T(0), da = pa ? dnA(ka) : T(0);
        const T wb = pb ? WrB[kb] : T(0), db = pb ? dnB(kb) : T(0);
        a0 = fma(wa, da, a0);
        b0 = fma(wb, db, b0);
        ka += pa ? 32 : 0;
        kb += pb ? 32 : 0;
    }
    totA = warp_sum((a0 + a1) + (a2 + a3));
    totB = warp_sum((b0 + b1) + (b2 + b3));
}

// chi = chi_SET(eta), eta = etafac x (Eqs. chi, chi_ret), in the wide type, rounded once: J1
// scales with b rho chi, and near finely resolved walls J1 is large enough that a few roundings of
// chi show in the right-hand side.
template <typename T>
__device__ __forceinline__ T clo_chi(T etafac, T x) {
    using W = Wide<T>;
    const W eta = w_scale(w_from_t(x), etafac);
    const W om = w_sub(w_from_t(T(1)), eta);
    const W om3 = w_mul(w_mul(om, om), om);
    return w_hi(w_div(w_sub(w_from_t(T(2)), eta), w_scale(om3, T(2))));
}

// The reach cells' fields as a block holds them (shared memory, reach-local index).
template <typename T>
struct ReachView {
    const Wide<T>* n;
    const Wide<T>* Tc;
    const Wide<T>* u[3];
    const T* chi;
    const T* nb;
};

// Position q of the J1 gradient stencils of own cell c (reach index lt; the stencil cell has
// reach index k, weight wq): the five gradient terms, logarithms of ratios to the own cell, exact
// because the stencil weights sum to zero:
//   sum_q w_q ln(n_q^2 chi_q T_q) = sum_q w_q [2 log1p(dn_q / n) + log1p(dchi_q / chi) + log1p(dT_q / T)],
// the differences taken in the wide type; ln chi_q - ln chi_c from the packing-fraction
// difference alone, since ln chi(eta) = ln(2 - eta) - ln 2 - 3 ln(1 - eta) (no rounding noise of
// chi itself); velocity differences in the wide type.
template <typename T>
__device__ __forceinline__ void clo_grad_terms(const ReachView<T>& R, int k, int lt, T wq, T etaf, bool chi_local,
                                               T (&g)[5]) {
    const Wide<T> nw = R.n[lt], Tw = R.Tc[lt];
    const T lT = log1p(ratio_fast(w_hi(w_sub(R.Tc[k], Tw)), w_hi(Tw)));
    const T ln = log1p(ratio_fast(w_hi(w_sub(R.n[k], nw)), w_hi(nw)));
    const T dnb = chi_local ? w_hi(w_sub(R.n[k], nw)) : R.nb[k] - R.nb[lt];
    const T etac = etaf * (chi_local ? w_hi(nw) : R.nb[lt]), deta = etaf * dnb;
    const T lchi = log1p(ratio_fast(-deta, T(2) - etac)) - T(3) * log1p(ratio_fast(-deta, T(1) - etac));
    g[0] = wq * (T(2) * ln + lchi + lT);
    g[1] = wq * lT;
    g[2] = wq * w_hi(w_sub(R.u[0][k], R.u[0][lt]));
    g[3] = wq * w_hi(w_sub(R.u[1][k], R.u[1][lt]));
    g[4] = wq * w_hi(w_sub(R.u[2][k], R.u[2][lt]));
}

// The 20 scalars of an own cell's collision record: n, u, 1/T, 1/tau (Eq. tau), the Shakhov
// coefficient (Eq. prandtl), q, -b rho chi, the J1 gradients X = d ln(n^2 chi T), Y = d ln T, the
// velocity derivative, the covariant strain (cylinder / sphere) and its divergence (Eq. j1);
// mu from Eq. viscosity.  Products the stage kernel would otherwise form per cell and thread are
// stored in place of their factors that it uses nowhere else: 0.4 S_11 / T in place of S_11,
// 2 S_01 / T in place of S_01, 1 / (2T) in the spare slot 18.  gp[v][q]: the gradient terms of the cell's five stencil positions.
template <typename T>
__device__ __forceinline__ void clo_record_scalars(T* ct, const ReachView<T>& R, int lt, const T (&gp)[5][5], T geo0,
                                                   T geo1, const T (&q)[3], const InstDev& I) {
    using C = T;
    const C cn = w_hi(R.n[lt]), cT = w_hi(R.Tc[lt]), cchi = R.chi[lt];
    const C in = ratio_fast(C(1), cn), iT = ratio_fast(C(1), cT), ichi = ratio_fast(C(1), cchi);
    C gsum[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) gsum[v] = (gp[v][0] + gp[v][1]) + (gp[v][2] + gp[v][3]) + gp[v][4];
    const C sc = geo1 * inst_param<C>(1.0 / I.ds, I.f_ids);
    const C X = gsum[0] * sc, Y = gsum[1] * sc;
    const C cd0 = gsum[2] * sc, cd1 = gsum[3] * sc, cd2 = gsum[4] * sc;
    const C iR = ratio_fast(C(1), geo0);
    const C cu0 = w_hi(R.u[0][lt]), cu1 = w_hi(R.u[1][lt]), cu2 = w_hi(R.u[2][lt]);
    const C sg = inst_param<C>(I.sigma, I.f_sigma);
    const C br = inst_param<C>(I.bfac, I.f_bfac) * cn, x = br * cchi;
    const C pi = C(3.14159265358979323846);
    const C mu = ratio_fast(C(5), C(16) * sg * sg) * sqrt(cT * C(0.31830988618379067154)) *
                 (ichi + C(0.8) * br + C(4.0 / 25.0) * (C(1) + C(12) / pi) * br * br * cchi);
    const C Pr = ratio_fast(C(2.0 / 3.0) * (C(1) + C(0.8) * x + C(4.0 / 25.0) * (C(1) + C(12) / pi) * x * x),
                            C(1) + C(1.2) * x + C(9.0 / 25.0) * (C(1) + C(32) / (C(9) * pi)) * x * x);
    C S11, S22, S01, S02, div;
    if (I.geometry == 0) {
        S11 = cu0 * iR;
        S22 = C(0);
        S01 = C(0.5) * (cd1 - cu1 * iR);
        S02 = C(0.5) * cd2;
        div = cd0 + cu0 * iR;
    } else {
        S11 = S22 = cu0 * iR;
        S01 = C(0.5) * (cd1 - cu1 * iR);
        S02 = C(0.5) * (cd2 - cu2 * iR);
        div = cd0 + C(2) * cu0 * iR;
    }
    ct[0] = cn;
    ct[1] = cu0;
    ct[2] = cu1;
    ct[3] = cu2;
    ct[4] = iT;
    ct[5] = ratio_fast(cn * cT, mu);
    ct[6] = (C(1) - Pr) * iT * iT * in;
    ct[7] = q[0];
    ct[8] = q[1];
    ct[9] = q[2];
    ct[10] = -x;
    ct[11] = X;
    ct[12] = Y;
    ct[13] = cd0;
    ct[14] = T(0.4) * iT * S11;
    ct[15] = S22;
    ct[16] = T(2) * iT * S01;
    ct[17] = S02;
    ct[18] = T(0.5) * iT;
    ct[19] = div;
}

// Expansion coefficients of one equilibrium factor of an own cell (Sec. III.C); job 0 / 1: the
// half-range axis on the half line of sign + / -, job 2 / 3: the full-range axes 2 / 3.  cT, tm1
// = T - 1 (without cancellation), ur = u_R, ua = u_2 (job 2) or u_3 (job 3).
template <typename T>
__device__ __forceinline__ void clo_eq_coeffs(int job, T cT, T tm1, T ur, T ua, const ClosureTabs<T>& tb,
                                              const MomSet& M, T (&ev)[kMaxE + 1]) {
    using C = T;
    const T *ha = tb.ha, *hb = tb.hb, *ihb = tb.ihb, *h0t = tb.h0t;
#pragma unroll
    for (int l = 0; l <= kMaxE; ++l) ev[l] = C(0);
    if (job < 2) {
        // half range, half line of sign s (job 0: +, 1: -), v = s u_R.  The recurrence of the
        // coefficients,
        //   e_0 = h_0 (1 + erf(v / sqrt(2T))) / 2,
        //   b_{l+1} e_{l+1} = (v - a_l) e_l + (T - 1) b_l e_{l-1}
        //                     + T h_l(0) [G_v(0) - sum_{k<l} h_k(0) e_k / sqrt(2 pi)],
        // is run for the deviation d_l = e_l - r_l from the rest state (v = 0, T = 1: r_0 = h_0 / 2,
        // r_l = 0 for l >= 1), where every term is small and nothing cancels: with
        // D = sqrt(2 pi) G_v(0) - 1 = (expm1(-z^2) - (T - 1)/(1 + sqrt T)) / sqrt T, z = v / sqrt(2T),
        // and h_0(0) r_0 = 1,
        //   d_0 = h_0 erf(z) / 2,
        //   b_1 d_1 = v r_0 + (v - a_0) d_0 + h_0 [(T - 1) + T D] / sqrt(2 pi),
        //   b_{l+1} d_{l+1} = (v - a_l) d_l + (T - 1) b_l e_{l-1}
        //                     + T h_l(0) [D - sum_{k<l} h_k(0) d_k] / sqrt(2 pi).
        const C v = job == 0 ? ur : -ur;
        const C sT = sqrt(cT), z = v * rsqrt(C(2) * cT);
        const C D = (expm1(-z * z) - tm1 / (C(1) + sT)) / sT;
        const C is2pi = C(0.39894228040143267794);
        const C r0 = h0t[0] * C(0.5);
        C d[kMaxE + 1];
#pragma unroll
        for (int l = 0; l <= kMaxE; ++l) d[l] = C(0);
        d[0] = r0 * erf(z);
        C run = C(0);  // sum_{k<l} h_k(0) d_k
#pragma unroll
        for (int l = 0; l < kMaxE; ++l) {
            if (l < M.NR) {
                C val;
                if (l == 0) {
                    val = v * r0 + (v - ha[0]) * d[0] + h0t[0] * (tm1 + cT * D) * is2pi;
                } else {
                    const C em1 = (l == 1 ? r0 : C(0)) + d[l > 0 ? l - 1 : 0];
                    val = (v - ha[l]) * d[l] + tm1 * hb[l] * em1 + cT * h0t[l] * (D - run) * is2pi;
                }
                run += h0t[l] * d[l];
                d[l + 1] = val * ihb[l + 1];
            }
        }
#pragma unroll
        for (int l = 0; l <= kMaxE; ++l) ev[l] = d[l];
        ev[0] += r0;
    } else {
        // full range: e_l = E[He_l(X)], X ~ N(u, T): e_{l+1} = u e_l + l (T - 1) e_{l-1}
        const int Nax = job == 2 ? M.N2 : M.N3;
        ev[0] = C(1);
        ev[1] = Nax >= 1 ? ua : C(0);
#pragma unroll
        for (int l = 1; l < kMaxE; ++l)
            if (l < Nax) ev[l + 1] = ua * ev[l] + C(l) * tm1 * ev[l - 1];
    }
}

// Entry k (of nR + n2 + n3) of an own cell's per-axis equilibrium vectors g_R, g_2, g_3 in the
// populations' precision; ecs: the cell's coefficients [job][l]; cT its temperature (the reduced
// pair's chi factor).  Returns the value, *dst its offset in the record.
template <typename T>
__device__ __forceinline__ T clo_g_entry(int k, const T (*ecs)[kMaxE], T cT, const ClosureTabs<T>& tb, const MomSet& M,
                                         int& dst) {
    const int nR = M.nR, n2 = M.n2, QR = nR / 2;
    T acc = T(0);
    // (the expansion orders are at most kMaxE - 1: every loop runs unrolled, predicated)
    if (k < nR) {
        const T* eh = ecs[k >= QR ? 1 : 0];
#pragma unroll
        for (int l = 0; l < kMaxE; ++l)
            if (l <= M.NR) acc += tb.GR[k * kMaxE + l] * eh[l];
        dst = rec_off_gR(n2) + k;
    } else if (k < nR + n2) {
        const int j = k - nR;
#pragma unroll
        for (int l = 0; l < kMaxE; ++l)
            if (l <= M.N2) acc += tb.G2[j * kMaxE + l] * ecs[2][l];
        dst = rec_off_g2() + j;
    } else {
        const int j = k - nR - n2;
        if (M.reduced) {
            // the pair's Gaussian factors: int g_z = 1 (phi), int p_z^2 g_z = T (chi)
            acc = j == 0 ? T(1) : cT;
        } else {
#pragma unroll
            for (int l = 0; l < kMaxE; ++l)
                if (l <= M.N3) acc += tb.G3[j * kMaxE + l] * ecs[3][l];
        }
        dst = rec_off_g3(nR, n2) + j;
    }
    return acc;
}

// Discrete mass of the stored equilibrium (one thread per own cell): the rounded vectors need not
// sum to exactly one per axis, and for FP32 populations that bias, times dt / tau every step, would
// make the total mass drift.  The density stored for f^MB = n g_R g_2 g_3 is the wide n divided by
// the wide product of the sums of the stored vectors (wide sums in the order of the entries).
template <typename T>
__device__ __forceinline__ void clo_mass_normalise(T* ct, Wide<T> n, const MomSet& M) {
    using W = Wide<T>;
    const int nR = M.nR, n2 = M.n2, n3 = M.n3;
    W sR = w_from_t(T(0)), s2 = w_from_t(T(0)), s3 = w_from_t(T(0));
    const T* gR = ct + rec_off_gR(n2);
    const T* g2 = ct + rec_off_g2();
    const T* g3 = ct + rec_off_g3(nR, n2);
    for (int k = 0; k < nR; ++k) sR = w_add(sR, w_from_t(gR[k]));
    for (int k = 0; k < n2; ++k) s2 = w_add(s2, w_from_t(g2[k]));
    if (M.reduced) {
        s3 = w_from_t(T(1));  // the mass is phi's: its p_z factor is exactly 1
    } else {
        for (int k = 0; k < n3; ++k) s3 = w_add(s3, w_from_t(g3[k]));
    }
    ct[0] = w_hi(w_div(n, w_mul(w_mul(sR, s2), s3)));
}

// Reach of an item of own cells [c0, c0 + cnt) of an instance of N cells: the own cells, two on
// each side (the gradient stencils), and the five cells next to a wall.
__device__ __forceinline__ void clo_reach(int c0, int cnt, int N, int& h0, int& h1) {
    h0 = max(0, min(c0 - 2, N - 5));
    h1 = min(N, max(c0 + cnt + 2, 5));
}

// Closure of the own cells [c0, c0 + cnt) of one instance (cnt <= kClosureCells): the collision
// records go to `recb` (the record of cell c0, stride A.rec_stride), chi and nbar to A.cw.
// Every thread of the block calls it (it holds block barriers); the block has at least
// kClosureWarps warps, and warps beyond them run extra(w, nw) (the w-th of nw such warps)
// while warps 0..2 run the chains of step 3; every thread runs after_loads() once the item's
// global loads are issued.  `wst` holds A.wst_elems staged band elements, `nbuf`
// A.max_union densities.  Returns false on every thread when the band-row copy never
// completed (A.err is set).
template <typename T, typename Extra, typename AfterLoads>
__device__ bool closure_cells(const ClosureArgs& A, const MomSet& M, const ClosureTabs<T>& tb, const InstDev& I, int c0,
                              int cnt, T* recb, T* wst, T* nbuf, uint64_t* cbar, uint32_t& phase, const Extra& extra,
                              const AfterLoads& after_loads) {
    using W = Wide<T>;
    __shared__ W sw_n[32], sw_T[32], sw_u[3][32];  // reach cells, wide
    __shared__ T s_chi[32], snb[32];               // reach cells: chi, band density
    __shared__ int sblo[32], scnt[32];             // reach cells: first band column, stored extent
    __shared__ T sq[3][32];                        // own cells: q
    __shared__ T ecs[kClosureCells][4][kMaxE];     // own cells: expansion coefficients
    __shared__ T sgp[kClosureCells][5][5];         // gradient terms per own cell and stencil position
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    const T* band = reinterpret_cast<const T*>(A.band);
    const T* dens = reinterpret_cast<const T*>(A.dens);
    const T* geoT = reinterpret_cast<const T*>(A.geoT);
    const int slices = A.slices;
    const int N = I.n_cells;
    int h0, h1;
    clo_reach(c0, cnt, N, h0, h1);
    const int nh = h1 - h0;
    const int rs = A.rec_stride;
    const ReachView<T> RV{sw_n, sw_T, {sw_u[0], sw_u[1], sw_u[2]}, s_chi, snb};
    // ---- 1. every global load of the item at once: the raw sums of the reach cells and the
    // geometry of the own cells (warp 0, lane per cell), the band rows of the reach cells
    // (bulk copies of their stored extents, issued by warp 0) and the densities of the union
    // of the bands (all threads)
    W sv[kSums];
    T geo0 = T(1), geo1 = T(0);
    if (warp == 0 && lane < nh) clo_load_sums<T>(A, (long long)I.cell_off + h0 + lane, sv);
    if (warp == 0 && lane < cnt) {
        const T* gc = geoT + (long long)(I.cell_off + c0 + lane) * kGeo;
        geo0 = gc[0];
        geo1 = gc[1];
    }
    int jlo = 0, nu = 0;
    const bool staged = !I.chi_local && nh * I.band_w <= A.wst_elems;
    if (!I.chi_local) {
        const int2* bl = reinterpret_cast<const int2*>(A.band_lo) + I.cell_off;
        const int2 first = bl[h0], last = bl[h1 - 1];
        jlo = first.x;
        // columns grow with the row, and extents are rounded up by at most 3
        const int jhi = min(N - 1, last.x + last.y - 1 + 3);
        nu = min(jhi - jlo + 1, A.max_union);
        if (warp == 0) {
            int2 mine = make_int2(0, 0);
            if (lane < nh) mine = bl[h0 + lane];
            if (lane < nh) {
                sblo[lane] = mine.x;
                scnt[lane] = mine.y;
            }
            if (staged) {
                // one bulk copy per row, of its stored extent (a multiple of 16 bytes)
                int bytes = lane < nh ? mine.y * (int)sizeof(T) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
                if (lane == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(cbar, (uint32_t)bytes);
                }
                __syncwarp();
                if (lane < nh && mine.y > 0)
                    bulk_g2s(wst + (long long)lane * I.band_w, band + I.band_off + (long long)(h0 + lane) * I.band_w,
                             (uint32_t)(mine.y * sizeof(T)), cbar);
            }
        }
        const T* nd = dens + ((long long)I.cell_off + jlo) * slices;
        for (int j0 = tid; j0 < nu; j0 += 4 * NT) {
            // four loads in flight per thread
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = min(j0 + u * NT, nu - 1);
                v[u] = nd[(long long)j * slices];
                for (int sl = 1; sl < slices; ++sl) v[u] += nd[(long long)j * slices + sl];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u * NT < nu) nbuf[j0 + u * NT] = v[u];
        }
    }
    after_loads();
    if (staged) {
        const bool ok = mbar_wait_bounded(cbar, phase);
        // every thread takes the same exit: a block-wide vote on the outcome
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(A.err, 2);
            mbar_wait_bounded(cbar, phase);  // bounded wait for the copy still in flight
            return false;
        }
        phase ^= 1u;
    } else {
        __syncthreads();  // staged: the vote above is the barrier
    }
    // ---- 2. warp 0: n, u, T of the reach cells (wide), q of the own cells; the other warps: FM
    // band sums of the reach cells from shared memory
    if (warp == 0) {
        if (lane < nh) {
            const int c = h0 + lane;
            W n, u[3], Tc;
            T q[3];
            clo_fields<T>(sv, n, u, Tc, q);
            sw_n[lane] = n;
            sw_u[0][lane] = u[0];
            sw_u[1][lane] = u[1];
            sw_u[2][lane] = u[2];
            sw_T[lane] = Tc;
            if (c >= c0 && c < c0 + cnt) {
                sq[0][c - c0] = q[0];
                sq[1][c - c0] = q[1];
                sq[2][c - c0] = q[2];
            }
        }
    } else if (!I.chi_local) {
        // one warp per row, every warp but the first (the row's sum does not depend on which)
        for (int t = warp - 1; t < nh; t += NT / 32 - 1) {
            const int c = h0 + t;
            const int lo = sblo[t];
            const int kmax = min(min(scnt[t], N - lo), nu - (lo - jlo));
            const T* Wr = staged ? wst + (long long)t * I.band_w : band + I.band_off + (long long)c * I.band_w;
            const T* nb = nbuf + (lo - jlo);
            const T tot = clo_band_row<T>(Wr, [&](int k) { return nb[k]; }, kmax, lane);
            if (lane == 0) snb[t] = tot;
        }
    }
    __syncthreads();
    // ---- 3. two concurrent chains.  Warp 0: chi of the reach cells, the gradient terms (one
    // lane per own cell and stencil position), then transport, strain and Shakhov coefficient
    // (lane per own cell).  Warps 1 and 2: the expansion coefficients of the equilibria (Sec.
    // III.C), lane per (own cell, axis half): warp 1 the half-range axis (+ and -), warp 2 the
    // axes 2 and 3.
    if (warp == 0) {
        const T etaf = inst_param<T>(I.etafac, I.f_etafac);
        if (lane < nh) s_chi[lane] = clo_chi<T>(etaf, I.chi_local ? w_hi(sw_n[lane]) : snb[lane]);
        __syncwarp();
        for (int e = lane; e < cnt * 5; e += 32) {
            const int t = e / 5, q = e % 5, c = c0 + t;
            int cq;
            T wq;
            stencil5_at<T>(c, N, q, cq, wq);
            T g[5];
            clo_grad_terms<T>(RV, cq - h0, c - h0, wq, etaf, I.chi_local != 0, g);
#pragma unroll
            for (int v = 0; v < 5; ++v) sgp[t][v][q] = g[v];
        }
        __syncwarp();
        if (lane < cnt) {
            const int t = lane, lt = c0 + t - h0;
            const T q[3] = {sq[0][t], sq[1][t], sq[2][t]};
            clo_record_scalars<T>(recb + (long long)t * rs, RV, lt, sgp[t], geo0, geo1, q, I);
            T* cw = reinterpret_cast<T*>(A.cw) + (long long)(I.cell_off + c0 + t) * 2;
            cw[0] = s_chi[lt];
            cw[1] = I.chi_local ? w_hi(sw_n[lt]) : snb[lt];
        }
    } else if (warp <= 2) {
        for (int e = lane; e < 2 * cnt; e += 32) {
            const int t = e % cnt, job = 2 * (warp - 1) + e / cnt, lt = c0 + t - h0;
            const T cT = w_hi(sw_T[lt]);
            const T tm1 = w_hi(w_sub(sw_T[lt], w_from_t(T(1))));  // T - 1 without cancellation
            T ev[kMaxE + 1];
            clo_eq_coeffs<T>(job, cT, tm1, w_hi(sw_u[0][lt]), w_hi(sw_u[job == 2 ? 1 : 2][lt]), tb, M, ev);
#pragma unroll
            for (int l = 0; l < kMaxE; ++l) ecs[t][job][l] = ev[l];
        }
    } else if (warp >= kClosureWarps) {
        extra(warp - kClosureWarps, NT / 32 - kClosureWarps);
    }
    __syncthreads();
    // ---- 5. per-axis equilibrium vectors of the own cells, in the populations' precision
    const int ng = M.nR + M.n2 + M.n3;
    for (int e = tid; e < cnt * ng; e += NT) {
        const int t = e / ng, k = e % ng;
        int dst;
        const T g = clo_g_entry<T>(k, ecs[t], w_hi(sw_T[c0 + t - h0]), tb, M, dst);
        recb[(long long)t * rs + dst] = g;
    }
    __syncthreads();
    // ---- 6. discrete mass of the stored equilibrium (a thread per own cell)
    for (int t = tid; t < cnt; t += NT) clo_mass_normalise<T>(recb + (long long)t * rs, sw_n[c0 + t - h0], M);
    __syncthreads();  // shared arrays are reused by the next call
    return true;
}

}  // namespace fdlb
