// Auxiliary kernels of the FDLB step (raw sums, closure, residual); the fused stage kernel is
// in stream_kernel.cuh.  See kernels.cuh for the data layout and the launch plan.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"
#include "kernels_decl.h"

namespace fdlb {

// ------------------------------------------------------------------------------ moments
// Raw quadrature sums (Eq. mom_quad) of the populations of whole cells; written into slice 0
// of the partial-sum array, the other slices are cleared.
template <typename T>
__global__ void moments_kernel(const T* __restrict__ f, double* __restrict__ sums, const int4* __restrict__ items,
                               const int* __restrict__ n_items, const InstDev* __restrict__ inst,
                               const double* __restrict__ tab, MomSet M) {
    __shared__ double red[kMaxRed][kSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nit = *n_items;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = items[it];
        const InstDev I = inst[w.x];
        for (int cl = 0; cl < w.z; ++cl) {
            const int c = w.y + cl;
            const T* fc = f + I.f_off + (long long)c * M.Np;
            T acc[kSums];
#pragma unroll
            for (int q = 0; q < kSums; ++q) acc[q] = T(0);
            for (int m = threadIdx.x; m < M.Np; m += blockDim.x) {
                const int k = m / (M.nR * M.n2), rem = m % (M.nR * M.n2), i = rem / M.n2, j = rem % M.n2;
                const T p0 = (T)tab[M.o_pR + i], p1 = (T)tab[M.o_p2 + j], p2 = (T)tab[M.o_p3 + k];
                const T v = fc[m], ps = p0 * p0 + p1 * p1 + p2 * p2;
                acc[0] += v;
                acc[1] += v * p0;
                acc[2] += v * p1;
                acc[3] += v * p2;
                acc[4] += v * p0 * p0;
                acc[5] += v * p1 * p1;
                acc[6] += v * p2 * p2;
                acc[7] += v * p0 * p1;
                acc[8] += v * p0 * p2;
                acc[9] += v * p1 * p2;
                acc[10] += v * ps * p0;
                acc[11] += v * ps * p1;
                acc[12] += v * ps * p2;
            }
            // per-thread partials and warp tree in the populations' precision, FP64 across warps
#pragma unroll
            for (int q = 0; q < kSums; ++q) {
                const T s = warp_sum(acc[q]);
                if (lane == 0) red[warp][q] = (double)s;
            }
            __syncthreads();
            if (threadIdx.x < kSums) {
                double s = 0.0;
                for (int ww = 0; ww < nw; ++ww) s += red[ww][threadIdx.x];
                double* dst = sums + ((long long)(I.cell_off + c) * M.slices) * kSums;
                dst[threadIdx.x] = s;
                for (int sl = 1; sl < M.slices; ++sl) dst[sl * kSums + threadIdx.x] = 0.0;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------------ closure
// Per cell, once per stage (one thread per cell in FP64, warps for the band sums):
//  * n, u, T, q, P_12 from the raw sums (Eq. macro_def);
//  * nbar over the stored FM band (Eq. fm, n = 0 outside the domain), chi = chi_SET(pi sigma^3
//    nbar / 6) (Eqs. chi, chi_ret), or chi at the local density;
//  * the J1 gradients by the five-point stencils (two halo cells each side are recomputed),
//    mu, Pr, tau (Eqs. viscosity, prandtl, tau), the covariant strain, the Shakhov coefficient;
//  * the per-axis equilibrium vectors g_R, g_2, g_3 (Sec. III.C) by their recurrences;
//  * at the two wall items, the wall density n_w from zero net mass flux (diffuse walls).
// Output: the FP64 closure record and the per-cell collision record in the populations'
// precision, [20 scalars | g_R | g_2 | g_3].
__host__ __device__ inline size_t closure_smem_bytes(int max_cells, int max_union, int tsize) {
    const size_t CH = (size_t)max_cells + 4;
    return (CH * kSums + 9 * CH + 32) * sizeof(double) + ((size_t)max_cells * 4 * kMaxE + max_union) * tsize + 16;
}

template <typename T>
__global__ void __launch_bounds__(256) closure_kernel(ClosureArgs A, MomSet M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5, NT = blockDim.x;
    const int CH = A.max_cells + 4;
    double* ssum = reinterpret_cast<double*>(smem_raw);  // [CH][13] raw sums of the cells in reach
    double* cb = ssum + CH * kSums;                       // [9][CH]: n u0 u1 u2 T chi phi1 phi2 nbar
    double* red = cb + 9 * CH;                            // [32]
    T* ec = reinterpret_cast<T*>(red + 32);               // [max_cells][4][kMaxE]
    T* nbuf = ec + (size_t)A.max_cells * 4 * kMaxE;
    const T* tabT = reinterpret_cast<const T*>(A.tabT);   // the tables in the populations' precision
    const T* band = reinterpret_cast<const T*>(A.band);
    const T* fin_all = reinterpret_cast<const T*>(A.f_in);
    T* rec_all = reinterpret_cast<T*>(A.rec);
    const double* tab = A.tab;
    const int nR = M.nR, n2 = M.n2, n3 = M.n3, Np = M.Np, QR = nR / 2;
    const int nit = *A.n_items;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = A.items[it];
        const InstDev I = A.inst[w.x];
        const int c0 = w.y, cnt = w.z, N = I.n_cells;
        // cells whose closure the gradients need: two on each side, and the five cells next to a
        // wall for the one-sided stencils (nh <= max(cnt + 4, 5) <= max_cells + 4)
        const int h0 = max(0, min(c0 - 2, N - 5)), h1 = min(N, max(c0 + cnt + 2, 5)), nh = h1 - h0;
        const double* S = A.sums + (long long)I.cell_off * A.slices * kSums;
        double* ca = A.ca + (long long)I.cell_off * kCA;
        // ---- 1. raw sums of the cells in reach (summed over the momentum slices in a fixed
        // order) and the densities of the union of their FM bands
        for (int e = tid; e < nh * kSums; e += NT) {
            const int t = e / kSums, q = e % kSums;
            const double* src = S + (long long)(h0 + t) * A.slices * kSums + q;
            double v = 0.0;
            for (int sl = 0; sl < A.slices; ++sl) v += src[sl * kSums];
            ssum[t * kSums + q] = v;
        }
        int jlo = 0, jhi = -1;
        if (!I.chi_local) {
            jlo = A.band_lo[I.cell_off + h0];
            jhi = min(N - 1, A.band_lo[I.cell_off + h1 - 1] + I.band_w - 1);
            const int nu = min(jhi - jlo + 1, A.max_union);
            for (int j = tid; j < nu; j += NT) {
                const double* src = S + (long long)(jlo + j) * A.slices * kSums;
                double nj = 0.0;
                for (int sl = 0; sl < A.slices; ++sl) nj += src[sl * kSums];
                nbuf[j] = (T)nj;
            }
        }
        __syncthreads();
        // ---- 2. n, u, T (Eq. macro_def) per cell in reach; q and P_12 of the own cells
        for (int t = tid; t < nh; t += NT) {
            const int c = h0 + t;
            const double* s = ssum + t * kSums;
            const double n = s[0], in = 1.0 / n;
            const double u0 = s[1] * in, u1 = s[2] * in, u2 = s[3] * in;
            const double tr = s[4] + s[5] + s[6];
            const double uu = u0 * u0 + u1 * u1 + u2 * u2;
            const double Tc = (tr - n * uu) * in * (1.0 / 3.0);
            cb[0 * CH + t] = n;
            cb[1 * CH + t] = u0;
            cb[2 * CH + t] = u1;
            cb[3 * CH + t] = u2;
            cb[4 * CH + t] = Tc;
            if (I.chi_local) {
                cb[5 * CH + t] = chi_cs(I.etafac * n);
                cb[8 * CH + t] = n;
            }
            if (c >= c0 && c < c0 + cnt) {
                const double m0 = s[4] * u0 + s[7] * u1 + s[8] * u2;
                const double m1 = s[7] * u0 + s[5] * u1 + s[9] * u2;
                const double m2 = s[8] * u0 + s[9] * u1 + s[6] * u2;
                double* r = ca + (long long)c * kCA;
                r[0] = n;
                r[1] = u0;
                r[2] = u1;
                r[3] = u2;
                r[4] = Tc;
                r[5] = 0.5 * (s[10] - 2.0 * m0 - u0 * tr + 2.0 * n * uu * u0);
                r[6] = 0.5 * (s[11] - 2.0 * m1 - u1 * tr + 2.0 * n * uu * u1);
                r[7] = 0.5 * (s[12] - 2.0 * m2 - u2 * tr + 2.0 * n * uu * u2);
                r[8] = s[7] - n * u0 * u1;  // P_12
                r[11] = 0.0;
            }
        }
        // ---- 3. Fischer-Methfessel density (Eq. fm) and chi (Eqs. chi, chi_ret): a warp per cell
        if (!I.chi_local) {
            for (int t = warp; t < nh; t += nwarps) {
                const int c = h0 + t;
                const int lo = A.band_lo[I.cell_off + c];
                const int kmax = min(I.band_w, jhi - lo + 1);
                const T* Wr = band + I.band_off + (long long)c * I.band_w;
                const T* nb = nbuf + (lo - jlo);
                T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
                int k = lane;
                for (; k + 96 < kmax; k += 128) {
                    a0 += Wr[k] * nb[k];
                    a1 += Wr[k + 32] * nb[k + 32];
                    a2 += Wr[k + 64] * nb[k + 64];
                    a3 += Wr[k + 96] * nb[k + 96];
                }
                for (; k < kmax; k += 32) a0 += Wr[k] * nb[k];
                const T acc = warp_sum((a0 + a1) + (a2 + a3));
                if (lane == 0) {
                    cb[8 * CH + t] = (double)acc;
                    cb[5 * CH + t] = chi_cs(I.etafac * (double)acc);
                }
            }
        }
        __syncthreads();
        for (int t = tid; t < nh; t += NT) {
            const double n = cb[t], Tc = cb[4 * CH + t], chi = cb[5 * CH + t];
            cb[6 * CH + t] = log(n * n * chi * Tc);
            cb[7 * CH + t] = log(Tc);
        }
        __syncthreads();
        // ---- 4. own cells: warp job 0 = gradients, transport, strain (Eqs. j1, viscosity,
        // prandtl, tau); jobs 1..4 = expansion coefficients of the equilibria (Sec. III.C)
        const int rs = A.rec_stride;
        T* rec = rec_all + (long long)I.cell_off * rs;
        for (int job = warp; job < 5; job += nwarps) {
            for (int t = lane; t < cnt; t += 32) {
                const int c = c0 + t, lt = c - h0;
                const double n = cb[lt], u0 = cb[CH + lt], u1 = cb[2 * CH + lt], u2 = cb[3 * CH + lt];
                const double Tc = cb[4 * CH + lt], chi = cb[5 * CH + lt];
                if (job == 0) {
                    int idx[5];
                    double sw[5];
                    stencil5(c, N, idx, sw);
                    const double* gc = A.geo + (long long)(I.cell_off + c) * kGeo;
                    const double R = gc[0], sc = gc[1] / I.ds;
                    double X = 0.0, Y = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0;
                    for (int q = 0; q < 5; ++q) {
                        const int k = idx[q] - h0;
                        X += sw[q] * cb[6 * CH + k];
                        Y += sw[q] * cb[7 * CH + k];
                        d0 += sw[q] * cb[1 * CH + k];
                        d1 += sw[q] * cb[2 * CH + k];
                        d2 += sw[q] * cb[3 * CH + k];
                    }
                    X *= sc;
                    Y *= sc;
                    d0 *= sc;
                    d1 *= sc;
                    d2 *= sc;
                    // transport, strain and Shakhov coefficient in the populations' precision
                    // (they are stored in it); FP64 above only for the gradients of logarithms
                    using C = T;
                    const C cn = (C)n, cT = (C)Tc, cchi = (C)chi, iR = (C)(1.0 / R);
                    const C cu0 = (C)u0, cu1 = (C)u1, cu2 = (C)u2, sg = (C)I.sigma;
                    const C br = (C)I.bfac * cn, x = br * cchi;
                    const C pi = C(3.14159265358979323846);
                    const C mu = C(5) / (C(16) * sg * sg) * sqrt(cT / pi) *
                                 (C(1) / cchi + C(0.8) * br + C(4.0 / 25.0) * (C(1) + C(12) / pi) * br * br * cchi);
                    const C Pr = C(2.0 / 3.0) * (C(1) + C(0.8) * x + C(4.0 / 25.0) * (C(1) + C(12) / pi) * x * x) /
                                 (C(1) + C(1.2) * x + C(9.0 / 25.0) * (C(1) + C(32) / (C(9) * pi)) * x * x);
                    const C itau = cn * cT / mu;
                    C S11, S22, S01, S02, div;
                    const C cd0 = (C)d0, cd1 = (C)d1, cd2 = (C)d2;
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
                    const double* rc = ca + (long long)c * kCA;
                    T* ct = rec + (long long)c * rs;
                    const C iT = C(1) / cT;
                    ct[0] = cn;
                    ct[1] = cu0;
                    ct[2] = cu1;
                    ct[3] = cu2;
                    ct[4] = iT;
                    ct[5] = itau;
                    ct[6] = (C(1) - Pr) * iT * iT / cn;
                    ct[7] = (T)rc[5];
                    ct[8] = (T)rc[6];
                    ct[9] = (T)rc[7];
                    ct[10] = x;
                    ct[11] = (T)X;
                    ct[12] = (T)Y;
                    ct[13] = cd0;
                    ct[14] = S11;
                    ct[15] = S22;
                    ct[16] = S01;
                    ct[17] = S02;
                    ct[18] = T(0);
                    ct[19] = div;
                    ca[(long long)c * kCA + 9] = chi;
                    ca[(long long)c * kCA + 10] = cb[8 * CH + lt];
                } else if (job <= 2) {
                    // half range, half line of sign s (job 1: +, job 2: -), v = s u_R:
                    //   e_0 = h_0 (1 + erf(v/sqrt(2T)))/2,
                    //   b_{l+1} e_{l+1} = (v - a_l) e_l + (T - 1) b_l e_{l-1}
                    //                     + T h_l(0) [G_v(0) - sum_{k<l} h_k(0) e_k / sqrt(2 pi)]
                    // (in the populations' precision)
                    using C = T;
                    T* e = ec + ((long long)t * 4 + (job - 1)) * kMaxE;
                    const T* ha = tabT + M.o_ha;
                    const T* hb = tabT + M.o_hb;
                    const T* h0t = tabT + M.o_h0;
                    for (int l = 0; l < kMaxE; ++l) e[l] = C(0);
                    const C cT = (C)Tc, v = job == 1 ? (C)u0 : -(C)u0;
                    const C G0 = exp(-v * v / (C(2) * cT)) / sqrt(C(6.283185307179586477) * cT);
                    e[0] = h0t[0] * C(0.5) * (C(1) + erf(v / sqrt(C(2) * cT)));
                    C run = C(0);
                    for (int l = 0; l < M.NR; ++l) {
                        const C em1 = l ? e[l - 1] : C(0);
                        const C bl = l ? hb[l] : C(0);
                        const C val = (v - ha[l]) * e[l] + (cT - C(1)) * bl * em1 +
                                      cT * h0t[l] * (G0 - run * C(0.39894228040143267794));
                        e[l + 1] = val / hb[l + 1];
                        run += h0t[l] * e[l];
                    }
                } else {
                    // full range: e_l = E[He_l(X)], X ~ N(u, T): e_{l+1} = u e_l + l (T - 1) e_{l-1}
                    using C = T;
                    T* e = ec + ((long long)t * 4 + (job - 1)) * kMaxE;
                    for (int l = 0; l < kMaxE; ++l) e[l] = C(0);
                    const C u = job == 3 ? (C)u1 : (C)u2, cT = (C)Tc;
                    const int Nax = job == 3 ? M.N2 : M.N3;
                    e[0] = C(1);
                    if (Nax >= 1) e[1] = u;
                    for (int l = 1; l < Nax; ++l) e[l + 1] = u * e[l] + C(l) * (cT - C(1)) * e[l - 1];
                }
            }
        }
        __syncthreads();
        // ---- 5. per-axis equilibrium vectors of the own cells, in the populations' precision
        const int ng = nR + n2 + n3;
        for (int e = tid; e < cnt * ng; e += NT) {
            const int t = e / ng, k = e % ng;
            const T* e4 = ec + (long long)t * 4 * kMaxE;
            T acc = T(0);
            int dst;
            if (k < nR) {
                const T* eh = e4 + (k >= QR ? kMaxE : 0);
                for (int l = 0; l <= M.NR; ++l) acc += tabT[M.o_GR + k * kMaxE + l] * eh[l];
                dst = rec_off_gR(n2) + k;
            } else if (k < nR + n2) {
                const int j = k - nR;
                for (int l = 0; l <= M.N2; ++l) acc += tabT[M.o_G2 + j * kMaxE + l] * e4[2 * kMaxE + l];
                dst = rec_off_g2() + j;
            } else {
                const int j = k - nR - n2;
                for (int l = 0; l <= M.N3; ++l) acc += tabT[M.o_G3 + j * kMaxE + l] * e4[3 * kMaxE + l];
                dst = rec_off_g3(nR, n2) + j;
            }
            rec[(long long)(c0 + t) * rs + dst] = acc;
        }
        // ---- 6. wall densities (diffuse walls): n_w = sum_out |p_R| w vhat_wall / sum_in |p_R| g_wall
        const T* fin = fin_all + I.f_off;
        for (int side = 0; side < 2; ++side) {
            const bool here = side == 0 ? (c0 == 0) : (c0 + cnt == N);
            if (!here) continue;
            double acc = 0.0;
            for (int m = tid; m < Np; m += NT) {
                const int k = m / (nR * n2), rem = m % (nR * n2), i = rem / n2, j = rem % n2;
                const T pr = (T)tab[M.o_pR + i];
                if (side == 0 ? !(pr < T(0)) : !(pr > T(0))) continue;
                const T wm = (T)tab[M.o_wR + i] * (T)tab[M.o_w2 + j] * (T)tab[M.o_w3 + k], iw = T(1) / wm;
                const long long b = side == 0 ? (long long)m : (long long)(N - 1) * Np + m;
                const long long st = side == 0 ? (long long)Np : -(long long)Np;
                const T f0 = fin[b], f1 = fin[b + st], f2 = fin[b + 2 * st], f3 = fin[b + 3 * st];
                const T g1 = T(4) * f0 - T(6) * f1 + T(4) * f2 - f3;
                const T g2 = T(10) * f0 - T(20) * f1 + T(15) * f2 - T(4) * f3;
                const T vh = weno5(f2 * iw, f1 * iw, f0 * iw, g1 * iw, g2 * iw);
                acc += (double)(fabs(pr) * wm * vh);
            }
            acc = warp_sum(acc);
            if (lane == 0) red[warp] = acc;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int ww = 0; ww < nwarps; ++ww) tot += red[ww];
                A.nw[w.x * 2 + side] = tot / I.nw_den[side];
            }
            __syncthreads();
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------ stream
// ------------------------------------------------------------------------------ residual
// Per instance: the profile moments (n, u_2, T, q_R) of the populations whose raw sums are
// given, the largest change since the saved profile, the largest saved value, the total mass
// sum_c V_c n_c and a non-finite flag; the current profile replaces the saved one.
__global__ void residual_kernel(const double* __restrict__ sums, int slices, const InstDev* __restrict__ inst,
                                const double* __restrict__ geo, double* __restrict__ prev, double* __restrict__ out,
                                int n_inst, int save) {
    __shared__ double red[kMaxRed][10];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = blockIdx.x; q < n_inst; q += gridDim.x) {
        const InstDev I = inst[q];
        double loc[10];
        for (int e = 0; e < 10; ++e) loc[e] = 0.0;
        for (int c = threadIdx.x; c < I.n_cells; c += blockDim.x) {
            double s[kSums];
            for (int e = 0; e < kSums; ++e) s[e] = 0.0;
            for (int sl = 0; sl < slices; ++sl)
                for (int e = 0; e < kSums; ++e) s[e] += sums[((long long)(I.cell_off + c) * slices + sl) * kSums + e];
            const double n = s[0], u0 = s[1] / n, u1 = s[2] / n, u2 = s[3] / n;
            const double tr = s[4] + s[5] + s[6], uu = u0 * u0 + u1 * u1 + u2 * u2;
            const double Tc = (tr - n * uu) / (3.0 * n);
            const double m0 = s[4] * u0 + s[7] * u1 + s[8] * u2;
            const double qR = 0.5 * (s[10] - 2.0 * m0 - u0 * tr + 2.0 * n * uu * u0);
            const double cur[4] = {n, u1, Tc, qR};
            double* pv = prev + (long long)(I.cell_off + c) * 4;
            for (int e = 0; e < 4; ++e) {
                double d = fabs(cur[e] - pv[e]);
                if (!(d == d)) d = 1e300;
                loc[e] = fmax(loc[e], d);
                loc[4 + e] = fmax(loc[4 + e], fabs(pv[e]));
                if (save) pv[e] = cur[e];
            }
            loc[8] += geo[(long long)(I.cell_off + c) * kGeo + 5] * n;
            if (!isfinite(n) || !isfinite(Tc) || !isfinite(qR) || !isfinite(u1)) loc[9] = 1.0;
        }
        for (int e = 0; e < 10; ++e) {
            double v = loc[e];
            for (int o = 16; o > 0; o >>= 1) {
                const double w = __shfl_xor_sync(0xffffffffu, v, o);
                v = (e == 8) ? v + w : fmax(v, w);
            }
            if (lane == 0) red[warp][e] = v;
        }
        __syncthreads();
        if (threadIdx.x < 10) {
            double v = threadIdx.x == 8 ? 0.0 : 0.0;
            for (int w = 0; w < nw; ++w) v = (threadIdx.x == 8) ? v + red[w][threadIdx.x] : fmax(v, red[w][threadIdx.x]);
            out[q * 10 + threadIdx.x] = v;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------ launchers
template <typename T>
void launch_moments(const T* f, double* sums, const int4* items, const int* n_items, int grid, const InstDev* inst,
                    const double* tab, const MomSet& M, cudaStream_t s) {
    moments_kernel<T><<<grid, 256, 0, s>>>(f, sums, items, n_items, inst, tab, M);
}

template <typename T>
void launch_closure(const ClosureArgs& A, const MomSet& M, int grid, int threads, size_t smem, cudaStream_t s) {
    if (smem > 48 * 1024) cudaFuncSetAttribute(closure_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    closure_kernel<T><<<grid, threads, smem, s>>>(A, M);
}

size_t closure_smem(int max_cells, int max_union, int tsize) { return closure_smem_bytes(max_cells, max_union, tsize); }

void launch_residual(const double* sums, int slices, const InstDev* inst, const double* geo, double* prev, double* out,
                     int n_inst, int save, cudaStream_t s) {
    residual_kernel<<<n_inst < 1024 ? n_inst : 1024, 256, 0, s>>>(sums, slices, inst, geo, prev, out, n_inst, save);
}

template void launch_moments<float>(const float*, double*, const int4*, const int*, int, const InstDev*,
                                    const double*, const MomSet&, cudaStream_t);
template void launch_moments<double>(const double*, double*, const int4*, const int*, int, const InstDev*,
                                     const double*, const MomSet&, cudaStream_t);
template void launch_closure<float>(const ClosureArgs&, const MomSet&, int, int, size_t, cudaStream_t);
template void launch_closure<double>(const ClosureArgs&, const MomSet&, int, int, size_t, cudaStream_t);

}  // namespace fdlb
