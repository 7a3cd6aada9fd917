// The fused stage kernel: one SSP-RK3 stage for a tile of radial cells x one momentum slice.
//
// Per work item (instance, first cell c0, cells Be, slice sl):
//  1. the TMA engine copies the populations of cells c0-3 .. c0+Be+2 (this slice) into shared
//     memory (one bulk copy when the slice is the whole cell, else one per cell);
//  2. meanwhile the block loads the per-cell collision records written by the closure kernel
//     (J1 gradients, tau, Pr, strain, equilibrium vectors) and the wall densities;
//  3. ghost rows at a wall: incoming directions carry n_w times the wall Maxwellian, outgoing
//     directions the cubic extrapolation of the four cells next to the wall;
//  4. per population: WENO5 face values of f/w upwinded by sign(p_R), conservative advection
//     with the face areas and cell volume (Sec. II.B/C), the curvature force with the K matrices
//     (Sec. III.B), the Shakhov + J1 collision (Eqs. j0, j1), the RK combination and the store;
//  5. the 13 raw sums of the new populations per cell (warp tree in the populations' precision,
//     FP64 across warps).
#pragma once

#include "device_common.cuh"
#include "kernels_decl.h"

namespace fdlb {

// Outgoing-direction ghost values (cubic extrapolation in the cell index) from the four
// populations next to a wall, f0 being the wall cell.
template <typename T>
__device__ __forceinline__ void wall_ghosts(T f0, T f1, T f2, T f3, T& g1, T& g2) {
    g1 = T(4) * f0 - T(6) * f1 + T(4) * f2 - f3;
    g2 = T(10) * f0 - T(20) * f1 + T(15) * f2 - T(4) * f3;
}

template <typename T, int GEOM, int MPT>
__global__ void __launch_bounds__(512, 1) stream_kernel(StageArgs A, MomSet M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NT = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;
    const int nR = M.nR, n2 = M.n2, n3 = M.n3, Ms = M.Ms, Np = M.Np;
    const StreamSmem P = stream_smem_plan(A.B, Ms, nR, n2, n3, nwarps, (int)sizeof(T));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    T* fs = reinterpret_cast<T*>(smem_raw + P.fs);  // rows: cells c0-3 .. c0+B+2
    T* sp_R = reinterpret_cast<T*>(smem_raw + P.tabs);
    T* sp_2 = sp_R + nR;
    T* sp_3 = sp_2 + n2;
    T* sw_R = sp_3 + n3;
    T* sw_2 = sw_R + nR;
    T* sw_3 = sw_2 + n2;
    T* sKR = sw_3 + n3;
    T* sK2 = sKR + nR * nR;
    T* sK3 = sK2 + n2 * n2;
    T* sgw = sK3 + n3 * n3;  // [2][nR + n2 + n3]: inner and outer wall Maxwellian per axis
    T* cellT = reinterpret_cast<T*>(smem_raw + P.cell);
    const int cstride = kCellScalars + nR + n2 + n3;
    T* sgeo = reinterpret_cast<T*>(smem_raw + P.geo);
    T* red = reinterpret_cast<T*>(smem_raw + P.red);  // warp partials of the raw sums
    const T* __restrict__ f_in = reinterpret_cast<const T*>(A.f_in);
    const T* __restrict__ f_n = reinterpret_cast<const T*>(A.f_n);
    T* __restrict__ f_out = reinterpret_cast<T*>(A.f_out);
    const double* __restrict__ tab = A.tab;
    const int gwstride = nR + n2 + n3;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    for (int e = tid; e < nR; e += NT) {
        sp_R[e] = (T)tab[M.o_pR + e];
        sw_R[e] = (T)tab[M.o_wR + e];
    }
    for (int e = tid; e < n2; e += NT) {
        sp_2[e] = (T)tab[M.o_p2 + e];
        sw_2[e] = (T)tab[M.o_w2 + e];
    }
    for (int e = tid; e < n3; e += NT) {
        sp_3[e] = (T)tab[M.o_p3 + e];
        sw_3[e] = (T)tab[M.o_w3 + e];
    }
    for (int e = tid; e < nR * nR; e += NT) sKR[e] = (T)tab[M.o_KR + e];
    for (int e = tid; e < n2 * n2; e += NT) sK2[e] = (T)tab[M.o_K2 + e];
    for (int e = tid; e < n3 * n3; e += NT) sK3[e] = (T)tab[M.o_K3 + e];
    __syncthreads();

    uint32_t phase = 0;
    const int nit = *A.n_items;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 wi = A.items[it];
        const InstDev I = A.inst[wi.x];
        const int N = I.n_cells, c0 = wi.y, Be = wi.z, sl = wi.w;
        const T* fin = f_in + I.f_off;
        const long long slice_off = (long long)sl * Ms;
        const int lo = c0 >= 3 ? c0 - 3 : 0;
        const int hi = min(c0 + Be + 3, N);  // staged cells [lo, hi)
        T* const frow0 = fs + (long long)(lo - c0 + 3) * Ms;

        // ---- 1. stage the cells (this slice) into shared memory
        if (A.use_bulk) {
            if (tid == 0) {
                fence_proxy_async();
                mbar_expect_tx(bar, (uint32_t)((hi - lo) * Ms * sizeof(T)));
                if (M.slices == 1) {
                    bulk_g2s(frow0, fin + (long long)lo * Np, (uint32_t)((hi - lo) * Np * sizeof(T)), bar);
                } else {
                    for (int cc = lo; cc < hi; ++cc)
                        bulk_g2s(frow0 + (long long)(cc - lo) * Ms, fin + (long long)cc * Np + slice_off,
                                 (uint32_t)(Ms * sizeof(T)), bar);
                }
            }
        } else {
            for (int cc = lo; cc < hi; ++cc)
                for (int e = tid; e < Ms; e += NT)
                    frow0[(long long)(cc - lo) * Ms + e] = ldg_t(fin + (long long)cc * Np + slice_off + e);
        }

        // ---- 2. per-cell collision records and geometry of the tile (overlapping the copy)
        const double* gwi = A.gw + (long long)wi.x * 2 * gwstride;
        for (int e = tid; e < 2 * gwstride; e += NT) sgw[e] = (T)gwi[e];
        for (int c = tid; c < Be; c += NT) {
            const double* g = A.geo + (long long)(I.cell_off + c0 + c) * kGeo;
            sgeo[c * 3 + 0] = (T)g[2];
            sgeo[c * 3 + 1] = (T)g[3];
            sgeo[c * 3 + 2] = (T)g[4];
        }
        {
            const T* rsrc = reinterpret_cast<const T*>(A.rec) + (long long)(I.cell_off + c0) * A.rec_stride;
            for (int e = tid; e < Be * cstride; e += NT) {
                const int cl = e / cstride, q = e % cstride;
                cellT[e] = rsrc[(long long)cl * A.rec_stride + q];
            }
        }
        const double nwall[2] = {A.nw[wi.x * 2], A.nw[wi.x * 2 + 1]};

        // ---- wait for the staged cells
        if (A.use_bulk) {
            const bool ok = mbar_wait_bounded(bar, phase);
            // every thread takes the same exit: a block-wide vote on the outcome
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(A.err, 1);
                mbar_wait_bounded(bar, phase);  // bounded wait for the copy still in flight
                return;
            }
            phase ^= 1u;
        }
        __syncthreads();

        // ---- 3. ghost rows at the walls
        const T nwL = (T)nwall[0], nwR = (T)nwall[1];
        const T* gwL = sgw;
        const T* gwR = sgw + gwstride;
        if (c0 == 0 || c0 + Be == N) {
            for (int ml = tid; ml < Ms; ml += NT) {
                const int kk = ml / (nR * n2), rem = ml % (nR * n2), i = rem / n2, j = rem % n2;
                const int k = sl * M.KS + kk;
                const T pr = sp_R[i];
                if (c0 == 0) {
                    T g1, g2;
                    if (pr > T(0)) {
                        g1 = g2 = nwL * gwL[i] * gwL[nR + j] * gwL[nR + n2 + k];
                    } else {
                        const T* r0 = fs + 3 * Ms + ml;
                        wall_ghosts(r0[0], r0[Ms], r0[2 * Ms], r0[3 * Ms], g1, g2);
                    }
                    fs[2 * Ms + ml] = g1;  // cell -1
                    fs[1 * Ms + ml] = g2;  // cell -2
                }
                if (c0 + Be == N) {
                    T g1, g2;
                    if (pr < T(0)) {
                        g1 = g2 = nwR * gwR[i] * gwR[nR + j] * gwR[nR + n2 + k];
                    } else {
                        const T* r0 = fs + (long long)(N - 1 - c0 + 3) * Ms + ml;
                        wall_ghosts(r0[0], r0[-Ms], r0[-2 * Ms], r0[-3 * Ms], g1, g2);
                    }
                    fs[(long long)(N - c0 + 3) * Ms + ml] = g1;      // cell N
                    fs[(long long)(N + 1 - c0 + 3) * Ms + ml] = g2;  // cell N+1
                }
            }
            __syncthreads();
        }

        // ---- 4. per-thread momenta of this slice; value of the left face of c0
        int code[MPT];
        T pr_[MPT], wm_[MPT], iw_[MPT], vl_[MPT];
#pragma unroll
        for (int r = 0; r < MPT; ++r) {
            const int ml = tid + r * NT;
            code[r] = 0;
            pr_[r] = wm_[r] = iw_[r] = vl_[r] = T(0);
            if (ml < Ms) {
                const int kk = ml / (nR * n2), rem = ml % (nR * n2), i = rem / n2, j = rem % n2;
                const int k = sl * M.KS + kk;
                code[r] = (kk << 16) | (i << 8) | j;
                const T pr = sp_R[i];
                pr_[r] = pr;
                wm_[r] = sw_R[i] * sw_2[j] * sw_3[k];
                const T iw = T(1) / wm_[r];
                iw_[r] = iw;
                if (c0 == 0 && pr > T(0)) {
                    vl_[r] = nwL * gwL[i] * gwL[nR + j] * gwL[nR + n2 + k] * iw;
                } else {
                    // rows of cells c0-3..c0+1 (p_R > 0) or c0+2..c0-2 (p_R < 0)
                    const T* b = fs + (long long)(pr > T(0) ? 0 : 5) * Ms + ml;
                    const long long s = pr > T(0) ? (long long)Ms : -(long long)Ms;
                    vl_[r] = weno5(b[0] * iw, b[s] * iw, b[2 * s] * iw, b[3 * s] * iw, b[4 * s] * iw);
                }
            }
        }

        const T dt = (T)I.dt, ca_ = (T)A.a, cb_ = (T)A.b;
        for (int cl = 0; cl < Be; ++cl) {
            const int c = c0 + cl;
            const T* ct = cellT + cl * cstride;
            const T n = ct[0], u0 = ct[1], u1 = ct[2], u2 = ct[3], iT = ct[4], itau = ct[5], cS = ct[6];
            const T q0 = ct[7], q1 = ct[8], q2 = ct[9], brchi = ct[10], X = ct[11], Y = ct[12];
            const T S00 = ct[13], S11 = ct[14], S22 = ct[15], S01 = ct[16], S02 = ct[17], dv = ct[19];
            const T* gR = ct + kCellScalars;
            const T* g2 = gR + nR;
            const T* g3 = g2 + n2;
            const T Ap = sgeo[cl * 3 + 0], Am = sgeo[cl * 3 + 1], kf = sgeo[cl * 3 + 2];
            const T* fc = fs + (long long)(cl + 3) * Ms;  // row of cell c
            T acc[kSums];
#pragma unroll
            for (int q = 0; q < kSums; ++q) acc[q] = T(0);
#pragma unroll
            for (int r = 0; r < MPT; ++r) {
                const int ml = tid + r * NT;
                if (ml < Ms) {
                    const int cd = code[r];
                    const int i = (cd >> 8) & 0xff, j = cd & 0xff, kk = (cd >> 16) & 0xff;
                    const int k = sl * M.KS + kk;
                    const T pr = pr_[r], iw = iw_[r];
                    // advection: WENO5 value at the right face, upwind by sign(p_R)
                    T vr;
                    if (c == N - 1 && pr < T(0)) {
                        vr = nwR * gwR[i] * gwR[nR + j] * gwR[nR + n2 + k] * iw;
                    } else {
                        const T* b = fc + (pr > T(0) ? -2LL : 3LL) * Ms + ml;
                        const long long s = pr > T(0) ? (long long)Ms : -(long long)Ms;
                        vr = weno5(b[0] * iw, b[s] * iw, b[2 * s] * iw, b[3 * s] * iw, b[4 * s] * iw);
                    }
                    const T adv = pr * wm_[r] * (Ap * vr - Am * vl_[r]);
                    vl_[r] = vr;
                    // curvature force with the derivative matrices
                    const T p2v = sp_2[j], p3v = sp_3[k];
                    const T* colR = fc + (kk * nR) * n2 + j;
                    T KRf = T(0);
#pragma unroll 8
                    for (int a = 0; a < nR; ++a) KRf += sKR[i * nR + a] * colR[a * n2];
                    const T* row2 = fc + (kk * nR + i) * n2;
                    T K2f = T(0);
#pragma unroll 8
                    for (int a = 0; a < n2; ++a) K2f += sK2[j * n2 + a] * row2[a];
                    T frc;
                    if (GEOM == 0) {
                        frc = kf * (p2v * p2v * KRf - pr * K2f);
                    } else {
                        const T* col3 = fc + i * n2 + j;
                        T K3f = T(0);
#pragma unroll 4
                        for (int a = 0; a < n3; ++a) K3f += sK3[k * n3 + a] * col3[a * nR * n2];
                        frc = kf * ((p2v * p2v + p3v * p3v) * KRf - pr * (K2f + K3f));
                    }
                    // collision: -(f - f^S)/tau + J1[f^MB]
                    const T f = fc[ml];
                    const T x0 = pr - u0, x1 = p2v - u1, x2 = p3v - u2;
                    const T xs = x0 * x0 + x1 * x1 + x2 * x2;
                    const T xq = x0 * q0 + x1 * q1 + x2 * q2;
                    const T fmb = n * gR[i] * g2[j] * g3[k];
                    const T z2 = T(0.5) * xs * iT;
                    const T strain = iT * (x0 * x0 * S00 + x1 * x1 * S11 + x2 * x2 * S22 + T(2) * (x0 * x1 * S01 + x0 * x2 * S02));
                    const T j1 = -brchi * (x0 * (X + T(0.6) * (z2 - T(2.5)) * Y) + T(0.4) * (strain + (z2 - T(2.5)) * dv));
                    const T fS = fmb * (T(1) + cS * (T(0.2) * xs * iT - T(1)) * xq);
                    const T L = -adv - frc - (f - fS) * itau + fmb * j1;
                    const long long gidx = I.f_off + (long long)c * Np + slice_off + ml;
                    T out;
                    if (A.mode == 1) {
                        out = L;
                    } else {
                        const T fnv = ca_ != T(0) ? ldg_t(f_n + gidx) : T(0);
                        out = ca_ * fnv + cb_ * (f + dt * L);
                    }
                    f_out[gidx] = out;
                    const T ps = pr * pr + p2v * p2v + p3v * p3v;
                    acc[0] += out;
                    acc[1] += out * pr;
                    acc[2] += out * p2v;
                    acc[3] += out * p3v;
                    acc[4] += out * pr * pr;
                    acc[5] += out * p2v * p2v;
                    acc[6] += out * p3v * p3v;
                    acc[7] += out * pr * p2v;
                    acc[8] += out * pr * p3v;
                    acc[9] += out * p2v * p3v;
                    acc[10] += out * ps * pr;
                    acc[11] += out * ps * p2v;
                    acc[12] += out * ps * p3v;
                }
            }
            // ---- 5. raw sums of the new populations: per-thread partial and warp tree in the
            // populations' precision, FP64 sum over the warps in a fixed order
            if (A.mode == 0) {
                T* rb = red + (cl & 1) * nwarps * kSums;
#pragma unroll
                for (int q = 0; q < kSums; ++q) {
                    const T s = warp_sum(acc[q]);  // warp tree in the populations' precision
                    if (lane == 0) rb[warp * kSums + q] = s;
                }
                __syncthreads();
                if (tid < kSums) {
                    double s = 0.0;  // FP64 sum over the warps, fixed order
                    for (int ww = 0; ww < nwarps; ++ww) s += (double)rb[ww * kSums + tid];
                    A.sums_out[((long long)(I.cell_off + c) * M.slices + sl) * kSums + tid] = s;
                }
            }
        }
        __syncthreads();  // the next item overwrites the staged rows and the cell data
    }
}

template <typename T, int GEOM, int MPT>
cudaError_t launch_stream_t(const StageArgs& A, const MomSet& M, int grid, int threads, size_t smem, cudaStream_t s) {
    auto kern = stream_kernel<T, GEOM, MPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, s>>>(A, M);
    return cudaGetLastError();
}

#define FDLB_STREAM_INSTANCE(T, G)                                                                            \
    cudaError_t launch_stream_##T##_##G(int mpt, const StageArgs& A, const MomSet& M, int grid, int threads, \
                                        size_t smem, cudaStream_t s) {                                       \
        switch (mpt) {                                                                                        \
            case 1: return launch_stream_t<T, G, 1>(A, M, grid, threads, smem, s);                          \
            case 2: return launch_stream_t<T, G, 2>(A, M, grid, threads, smem, s);                          \
            case 4: return launch_stream_t<T, G, 4>(A, M, grid, threads, smem, s);                          \
            case 8: return launch_stream_t<T, G, 8>(A, M, grid, threads, smem, s);                          \
            default: return cudaErrorInvalidValue;                                                            \
        }                                                                                                     \
    }

}  // namespace fdlb
