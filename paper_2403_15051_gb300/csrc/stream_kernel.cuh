// The fused stage kernel: one SSP-RK3 stage for a tile of radial cells x one momentum slice.
//
// Per work item (instance, first cell c0, cells Be, slice sl):
//  1. the TMA engine copies the populations of cells c0-3 .. c0+Be+2 (this slice) and the
//     tile's collision records (written by the closure kernel) into shared memory (a block's
//     first rows before its dependency wait, the records after it);
//  2. meanwhile the block loads the cell geometry and the wall densities;
//  3. ghost rows where the tile's stencils leave the domain: incoming directions carry n_w times
//     the wall Maxwellian, outgoing directions the cubic extrapolation of the four cells next to
//     the wall;
//  4. per population: WENO5 face values of f/w upwinded by sign(p_R), conservative advection
//     with the face areas and cell volume (Sec. II.B/C), the curvature force with the K matrices
//     (Sec. III.B), the Shakhov + J1 collision (Eqs. j0, j1), the RK combination and the store;
//  5. the 13 raw sums of the new populations per cell: per-thread partials, a transposing warp
//     reduction in the populations' precision, across the warps at the end of the item in a
//     fixed tree (double-float for FP32 populations, FP64 for FP64), stored as FP64 sums and, for
//     FP32 populations, as the double-float pairs the closure reads.
//
// Thread mapping: a "vector" is VW momenta with the same (k, i) and consecutive j, which are
// contiguous in the [k][i][j] layout.  A thread owns up to NV vectors for the whole kernel, so
// every shared-memory access is a VW-wide load: the five WENO rows, the column of the K^h
// contraction (shared by the VW momenta), the row of the K_2 contraction and, from K_2 stored
// transposed, each input's coefficients for the vector's outputs.  All momenta of a vector share
// p_R and hence the upwind direction.  A vector's momenta are processed in pairs of lanes (packed
// FP32x2 operations for FP32 populations), every operation written out, so that a lane's result
// does not depend on the pairing.
#pragma once

#include <type_traits>

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

// VW consecutive elements (16-byte aligned for VW * sizeof(T) >= 16; 8-byte for float2).
template <typename T, int VW>
__device__ __forceinline__ void ld_vec(const T* p, T (&o)[VW]) {
    if constexpr (sizeof(T) == 4 && VW == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
    } else if constexpr (sizeof(T) == 4 && VW == 8) {
        const float4 x = reinterpret_cast<const float4*>(p)[0], y = reinterpret_cast<const float4*>(p)[1];
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w; o[4] = y.x; o[5] = y.y; o[6] = y.z; o[7] = y.w;
    } else if constexpr (sizeof(T) == 4 && VW == 2) {
        const float2 x = *reinterpret_cast<const float2*>(p);
        o[0] = x.x; o[1] = x.y;
    } else if constexpr (sizeof(T) == 8 && VW >= 2) {
#pragma unroll
        for (int h = 0; h < VW / 2; ++h) {
            const double2 x = *reinterpret_cast<const double2*>(p + 2 * h);
            o[2 * h] = x.x; o[2 * h + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) o[e] = p[e];
    }
}

template <typename T, int VW>
__device__ __forceinline__ void ldg_vec(const T* p, T (&o)[VW]) {
    if constexpr (sizeof(T) == 4 && VW == 4) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(p));
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
    } else if constexpr (sizeof(T) == 4 && VW == 8) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(p)), y = __ldg(reinterpret_cast<const float4*>(p) + 1);
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w; o[4] = y.x; o[5] = y.y; o[6] = y.z; o[7] = y.w;
    } else if constexpr (sizeof(T) == 4 && VW == 2) {
        const float2 x = __ldg(reinterpret_cast<const float2*>(p));
        o[0] = x.x; o[1] = x.y;
    } else if constexpr (sizeof(T) == 8 && VW >= 2) {
#pragma unroll
        for (int h = 0; h < VW / 2; ++h) {
            const double2 x = __ldg(reinterpret_cast<const double2*>(p + 2 * h));
            o[2 * h] = x.x; o[2 * h + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) o[e] = __ldg(p + e);
    }
}

// The same through L2 only (data written earlier in the same launch by other blocks).
template <typename T, int VW>
__device__ __forceinline__ void ldcg_vec(const T* p, T (&o)[VW]) {
    if constexpr (sizeof(T) == 4 && VW == 4) {
        const float4 x = __ldcg(reinterpret_cast<const float4*>(p));
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w;
    } else if constexpr (sizeof(T) == 4 && VW == 8) {
        const float4 x = __ldcg(reinterpret_cast<const float4*>(p)), y = __ldcg(reinterpret_cast<const float4*>(p) + 1);
        o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w; o[4] = y.x; o[5] = y.y; o[6] = y.z; o[7] = y.w;
    } else if constexpr (sizeof(T) == 4 && VW == 2) {
        const float2 x = __ldcg(reinterpret_cast<const float2*>(p));
        o[0] = x.x; o[1] = x.y;
    } else if constexpr (sizeof(T) == 8 && VW >= 2) {
#pragma unroll
        for (int h = 0; h < VW / 2; ++h) {
            const double2 x = __ldcg(reinterpret_cast<const double2*>(p + 2 * h));
            o[2 * h] = x.x; o[2 * h + 1] = x.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) o[e] = __ldcg(p + e);
    }
}

template <typename T, int VW>
__device__ __forceinline__ void st_vec(T* p, const T (&o)[VW]) {
    if constexpr (sizeof(T) == 4 && VW == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (sizeof(T) == 4 && VW == 8) {
        reinterpret_cast<float4*>(p)[0] = make_float4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<float4*>(p)[1] = make_float4(o[4], o[5], o[6], o[7]);
    } else if constexpr (sizeof(T) == 4 && VW == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(o[0], o[1]);
    } else if constexpr (sizeof(T) == 8 && VW >= 2) {
#pragma unroll
        for (int h = 0; h < VW / 2; ++h) *reinterpret_cast<double2*>(p + 2 * h) = make_double2(o[2 * h], o[2 * h + 1]);
    } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) p[e] = o[e];
    }
}

// A vector as (VW + 1) / 2 pairs of lanes: (e0, e1), (e2, e3), ...; for VW = 1 one pair whose
// second lane repeats the first (computed alongside and never stored).  The loads go through the
// VW-wide forms above, whose registers the pairs then name without a move.
template <typename T, int VW>
__device__ __forceinline__ void pairs_of(const T (&v)[VW], Pair<T> (&o)[(VW + 1) / 2]) {
#pragma unroll
    for (int h = 0; h < (VW + 1) / 2; ++h) o[h] = p_make(v[2 * h], v[VW == 1 ? 0 : 2 * h + 1]);
}
template <typename T, int VW>
__device__ __forceinline__ void ld_pairs(const T* p, Pair<T> (&o)[(VW + 1) / 2]) {
    T v[VW];
    ld_vec<T, VW>(p, v);
    pairs_of<T, VW>(v, o);
}
template <typename T, int VW>
__device__ __forceinline__ void ldg_pairs(const T* p, Pair<T> (&o)[(VW + 1) / 2]) {
    T v[VW];
    ldg_vec<T, VW>(p, v);
    pairs_of<T, VW>(v, o);
}
template <typename T, int VW>
__device__ __forceinline__ void ldcg_pairs(const T* p, Pair<T> (&o)[(VW + 1) / 2]) {
    T v[VW];
    ldcg_vec<T, VW>(p, v);
    pairs_of<T, VW>(v, o);
}
template <typename T, int VW>
__device__ __forceinline__ void st_pairs(T* p, const Pair<T> (&o)[(VW + 1) / 2]) {
    T v[VW];
#pragma unroll
    for (int h = 0; h < (VW + 1) / 2; ++h) {
        v[2 * h] = o[h].x;
        if (2 * h + 1 < VW) v[2 * h + 1] = o[h].y;
    }
    st_vec<T, VW>(p, v);
}

// Local names of the stage's dimensions and of its shared-memory plan (StreamSmem): fs the
// staged rows of cells c0-3 .. c0+B+2, cellT the tile's records, sp_2 the p_2 nodes (first in the
// tables: aligned vector loads), sK2 K_2 in the vector-swizzled
// transposed, [b][j] (the coefficients of input b for a vector's outputs: one aligned vector load),
// sKR K^h with row stride krs,
// sK3 K_3 with row stride n3+1, nodes and weights, sgw the inner and outer wall Maxwellians per
// axis [2][nR + n2 + n3], sgeo the tile's geometry, red the per-warp sums [cell][warp][16], skrf
// K^h f of the own cells (tensor-core path).  NR_, N2_, N3_: compile-time axis sizes (0: taken
// from M at run time).  The sphere couples every axis: one slice (KS = n3), unless K_3 f comes from
// its own contraction kernel (A.k3f).
#define FDLB_STREAM_LAYOUT                                                                                       \
    extern __shared__ __align__(16) unsigned char smem_raw[];                                                    \
    const int NT = blockDim.x;                                                                                   \
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = NT >> 5;                             \
    const int nR = NR_ ? NR_ : M.nR, n2 = N2_ ? N2_ : M.n2, n3 = N3_ ? N3_ : M.n3;                               \
    const int KS = M.KS;                                                                                         \
    const int Ms = nR * n2 * KS, Np = nR * n2 * n3;                                                              \
    const int n2v = n2 / VW;                                                                                     \
    const int Vs = Ms / VW;                                                                                      \
    const int rs = record_stride(nR, n2, n3);                                                                    \
    constexpr bool kMMA = sizeof(T) == 4 && NR_ > 0 && NR_ % 8 == 0 && VW == 4;                                  \
    const bool use_mma = kMMA && A.mma;                                                                          \
    const StreamSmem P = stream_smem_plan(A.B, Ms, nR, n2, n3, nwarps, (int)sizeof(T), use_mma ? 1 : 0,          \
                                          A.krf ? 1 : 0);                                                        \
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);                                                       \
    T* fs = reinterpret_cast<T*>(smem_raw + P.fs);                                                               \
    T* cellT = reinterpret_cast<T*>(smem_raw + P.rec);                                                           \
    T* sp_2 = reinterpret_cast<T*>(smem_raw + P.tabs);                                                           \
    T* sK2 = sp_2 + p2_span(n2);                                                                                 \
    const int krs = kr_stride(nR);                                                                               \
    T* sKR = sK2 + kr_offset(n2, (int)sizeof(T));                                                                \
    T* sK3 = sKR + (A.krf ? 0 : nR) * krs;                                                                       \
    T* sp_R = sK3 + n3 * (n3 + 1);                                                                               \
    T* sp_3 = sp_R + nR;                                                                                         \
    T* sw_R = sp_3 + n3;                                                                                         \
    T* sw_2 = sw_R + nR;                                                                                         \
    T* sw_3 = sw_2 + n2;                                                                                         \
    T* sgw = sw_3 + n3;                                                                                          \
    T* sgeo = reinterpret_cast<T*>(smem_raw + P.geo);                                                            \
    T* red = reinterpret_cast<T*>(smem_raw + P.red);                                                             \
    T* skrf = reinterpret_cast<T*>(smem_raw + P.kr);                                                             \
    const T* __restrict__ f_in = reinterpret_cast<const T*>(A.f_in);                                             \
    const T* __restrict__ f_n = reinterpret_cast<const T*>(A.f_n);                                               \
    T* __restrict__ f_out = reinterpret_cast<T*>(A.f_out);                                                       \
    const T* __restrict__ rec_all = reinterpret_cast<const T*>(A.rec);                                           \
    const T* __restrict__ tab = reinterpret_cast<const T*>(A.tabT);                                              \
    const int gwstride = nR + n2 + n3;                                                                           \
    (void)0

// Tables of the stage (nodes, weights, K matrices) into shared memory and the copy barrier;
// the caller synchronises.
template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
__device__ __forceinline__ void stream_tables(const StageArgs& A, const MomSet& M) {
    FDLB_STREAM_LAYOUT;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    for (int e = tid; e < nR; e += NT) {
        sp_R[e] = tab[M.o_pR + e];
        sw_R[e] = tab[M.o_wR + e];
    }
    for (int e = tid; e < n2; e += NT) {
        sp_2[e] = tab[M.o_p2 + e];
        sw_2[e] = tab[M.o_w2 + e];
    }
    for (int e = tid; e < n3; e += NT) {
        sp_3[e] = tab[M.o_p3 + e];
        sw_3[e] = tab[M.o_w3 + e];
    }
    if (!A.krf)
        for (int e = tid; e < nR * nR; e += NT) sKR[(e / nR) * krs + e % nR] = tab[M.o_KR + e];
    for (int e = tid; e < n2 * n2; e += NT) sK2[(e % n2) * n2 + e / n2] = tab[M.o_K2 + e];  // transposed
    if (GEOM == 1)
        for (int e = tid; e < n3 * n3; e += NT) sK3[(e / n3) * (n3 + 1) + e % n3] = tab[M.o_K3 + e];
}

// Staging of a work item: the cells c0-3 .. c0+Be+2 of its slice and, when `records`, the
// tile's collision records (the bulk engine, completion on the copy barrier; else plain loads).
// With the bulk engine the two can be requested apart: part 1 expects the whole item and copies
// the rows, part 2 copies the records, part 3 does both.
template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
__device__ __forceinline__ void stream_issue(const StageArgs& A, const MomSet& M, int4 wi, const InstDev& I,
                                             bool records, int part = 3) {
    FDLB_STREAM_LAYOUT;
    const int N = I.n_cells, c0 = wi.y, Be = wi.z, sl = wi.w;
    const T* fin = f_in + I.f_off;
    const long long slice_off = (long long)sl * Ms;
    const int lo = c0 >= 3 ? c0 - 3 : 0;
    const int hi = min(c0 + Be + 3, N);  // staged cells [lo, hi)
    T* const frow0 = fs + (long long)(lo - c0 + 3) * Ms;
    const T* rsrc = rec_all + (long long)(I.cell_off + c0) * rs;
    // ---- 1. stage the cells (this slice) and the tile's collision records
    if (A.use_bulk) {
        if (tid == 0) {
            if (part & 1) {
                fence_proxy_async();
                mbar_expect_tx(bar, (uint32_t)(((hi - lo) * Ms + (records ? Be * rs : 0)) * sizeof(T)) + (uint32_t)A.tx_extra);
                if (M.slices == 1) {
                    bulk_g2s(frow0, fin + (long long)lo * Np, (uint32_t)((hi - lo) * Np * sizeof(T)), bar);
                } else {
                    for (int cc = lo; cc < hi; ++cc)
                        bulk_g2s(frow0 + (long long)(cc - lo) * Ms, fin + (long long)cc * Np + slice_off,
                                 (uint32_t)(Ms * sizeof(T)), bar);
                }
            }
            if (records && (part & 2)) bulk_g2s(cellT, rsrc, (uint32_t)(Be * rs * sizeof(T)), bar);
            // the tile's f_n (read once per population at the end of its update, from HBM) into L2
            // while the item is staged and computed
            if ((part & 1) && A.mode == 0 && (sizeof(T) == 4 ? A.fa : (float)A.a) != 0.f) {
                const T* fn = f_n + I.f_off + (long long)c0 * Np;
                if (M.slices == 1)
                    bulk_prefetch_l2(fn, (uint32_t)(Be * Np * sizeof(T)));
                else
                    for (int cl = 0; cl < Be; ++cl) bulk_prefetch_l2(fn + (long long)cl * Np + slice_off, (uint32_t)(Ms * sizeof(T)));
            }
        }
    } else {
        for (int cc = lo; cc < hi; ++cc)
            for (int e = tid; e < Ms; e += NT)
                frow0[(long long)(cc - lo) * Ms + e] = ldg_t(fin + (long long)cc * Np + slice_off + e);
        if (records)
            for (int e = tid; e < Be * rs; e += NT) cellT[e] = rsrc[e];
    }
}

// Geometry of the tile and the instance's wall Maxwellians into shared memory.
template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
__device__ __forceinline__ void stream_statics(const StageArgs& A, const MomSet& M, int4 wi, const InstDev& I) {
    FDLB_STREAM_LAYOUT;
    const int c0 = wi.y, Be = wi.z;
    const T* gwi = reinterpret_cast<const T*>(A.gwT) + (long long)wi.x * 2 * gwstride;
    for (int e = tid; e < 2 * gwstride; e += NT) sgw[e] = gwi[e];
    for (int c = tid; c < Be; c += NT) {
        const T* g = reinterpret_cast<const T*>(A.geoT) + (long long)(I.cell_off + c0 + c) * kGeo;
        sgeo[c * 3 + 0] = g[2];
        sgeo[c * 3 + 1] = g[3];
        sgeo[c * 3 + 2] = g[4];
    }
}

// Completion of the staged copy; false (on every thread, A.err set) when it never completes.  With
// the bulk engine the outcome is voted on block-wide, which is also the block's barrier after the
// copy; the plain-load path needs a barrier of its own.
template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
__device__ __forceinline__ bool stream_wait(const StageArgs& A, const MomSet& M, uint32_t& phase) {
    FDLB_STREAM_LAYOUT;
    // ---- wait for the staged cells
    if (A.use_bulk) {
        const bool ok = mbar_wait_bounded(bar, phase);
        // every thread takes the same exit: a block-wide vote on the outcome
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(A.err, 1);
            mbar_wait_bounded(bar, phase);  // bounded wait for the copy still in flight
            return false;
        }
        phase ^= 1u;
    }
    return true;
}

// Steps 3-5 of the item on the staged cells and records: ghost rows, the populations of the
// new stage, their raw sums.  nwL, nwR: the wall densities of the item's instance.
template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_, bool kCoherent = false>
__device__ __forceinline__ void stream_compute(const StageArgs& A, const MomSet& M, int4 wi, const InstDev& I,
                                               T nwL, T nwR) {
    FDLB_STREAM_LAYOUT;
    const int N = I.n_cells, c0 = wi.y, Be = wi.z, sl = wi.w;
    const long long slice_off = (long long)sl * Ms;
    // ---- 3. ghost rows: the tile's stencils span cells c0-3 .. c0+Be+2 (rows 0 .. Be+5, row =
    // cell - c0 + 3); the cells outside the domain among them (-2, -1 and N, N+1) hold n_w times
    // the wall Maxwellian for directions into the domain, the cubic extrapolation of the four
    // cells next to the wall for directions out of it.  Tiles near a wall need them whether or
    // not they touch it (a tile of two cells starting at cell 2 reaches cell -1).
    const T* gwL = sgw;
    const T* gwR = sgw + gwstride;
    const bool ghL = c0 < 3, ghR = c0 + Be + 2 >= N;
    if (ghL || ghR) {
        for (int ml = tid; ml < Ms; ml += NT) {
            const int kk = ml / (nR * n2), rem = ml % (nR * n2), i = rem / n2, j = rem % n2;
            const int k = sl * KS + kk;
            const T pr = sp_R[i];
            if (ghL) {
                T g1, g2;
                if (pr > T(0)) {
                    g1 = g2 = nwL * gwL[i] * gwL[nR + j] * gwL[nR + n2 + k];
                } else {
                    const T* r0 = fs + (long long)(3 - c0) * Ms + ml;  // cell 0
                    wall_ghosts(r0[0], r0[Ms], r0[2 * Ms], r0[3 * Ms], g1, g2);
                }
                fs[(long long)(2 - c0) * Ms + ml] = g1;                 // cell -1
                if (c0 <= 1) fs[(long long)(1 - c0) * Ms + ml] = g2;    // cell -2
            }
            if (ghR) {
                T g1, g2;
                if (pr < T(0)) {
                    g1 = g2 = nwR * gwR[i] * gwR[nR + j] * gwR[nR + n2 + k];
                } else {
                    const T* r0 = fs + (long long)(N - 1 - c0 + 3) * Ms + ml;  // cell N-1
                    wall_ghosts(r0[0], r0[-Ms], r0[-2 * Ms], r0[-3 * Ms], g1, g2);
                }
                fs[(long long)(N - c0 + 3) * Ms + ml] = g1;                           // cell N
                if (N + 1 <= c0 + Be + 2) fs[(long long)(N + 1 - c0 + 3) * Ms + ml] = g2;  // cell N+1
            }
        }
        __syncthreads();
    }

    // ---- 3b. tensor cores: (K^h f)[i][(k, j)] = sum_a K^h[i][a] f[k][a][j] for the own cells,
    // a GEMM of the nR x nR matrix with the cell's nR x (n2 KS) slice, in split TF32
    // (K = Kh + Kl, f = fh + fl; Kh fh + Kh fl + Kl fh with FP32 accumulation: FP32-level
    // products), n-tiles of 8 columns spread over the warps, results to shared memory.
    if constexpr (kMMA) {
      if (use_mma) {
        constexpr int MT = (NR_ + 15) / 16, KT = NR_ / 8;
        const int g = lane >> 2, tg = lane & 3;
        uint32_t ah[MT][KT][4], alo[MT][KT][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int ks = 0; ks < KT; ++ks)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = mt * 16 + g + ((q & 1) ? 8 : 0), cidx = ks * 8 + tg + ((q & 2) ? 4 : 0);
                    const float x = r < NR_ ? sKR[r * krs + cidx] : 0.f;
                    ah[mt][ks][q] = to_tf32(x);
                    alo[mt][ks][q] = to_tf32(x - __uint_as_float(ah[mt][ks][q]));
                }
        const int ncol = n2 * KS, ntc = ncol / 8;
        for (int tt = warp; tt < Be * ntc; tt += nwarps) {
            const int cl = tt / ntc, nt = tt % ntc;
            const int colb = nt * 8 + g;  // this lane's B column (k, j)
            const T* bsrc = fs + (long long)(cl + 3) * Ms + ((colb / n2) * nR) * n2 + colb % n2;
            float acc[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) acc[mt][0] = acc[mt][1] = acc[mt][2] = acc[mt][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < KT; ++ks) {
                const float x0 = bsrc[(ks * 8 + tg) * n2], x1 = bsrc[(ks * 8 + tg + 4) * n2];
                const uint32_t bh0 = to_tf32(x0), bh1 = to_tf32(x1);
                const uint32_t bl0 = to_tf32(x0 - __uint_as_float(bh0)), bl1 = to_tf32(x1 - __uint_as_float(bh1));
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    mma_tf32(acc[mt], alo[mt][ks], bh0, bh1);
                    mma_tf32(acc[mt], ah[mt][ks], bl0, bl1);
                    mma_tf32(acc[mt], ah[mt][ks], bh0, bh1);
                }
            }
            T* dst = skrf + (long long)cl * Ms;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = mt * 16 + g + ((q & 2) ? 8 : 0), cc = nt * 8 + 2 * tg + (q & 1);
                    if (r < NR_) dst[((cc / n2) * nR + r) * n2 + cc % n2] = acc[mt][q];
                }
        }
        __syncthreads();
      }
    }

    // ---- 4. the thread's vectors in this slice; WENO value at the left face of c0.  A vector's
    // momenta are processed in pairs of lanes (packed FP32x2 operations for FP32 populations).
    using V2 = Pair<T>;
    constexpr int NP = (VW + 1) / 2;
    int vcode[NV];  // (kk << 20) | (i << 10) | jb, -1 if none
    T pr_[NV], p3_[NV];
    V2 e4w_[NV][NP], vl_[NV][NP];
#pragma unroll
    for (int g = 0; g < NV; ++g) {
        const int v = tid + g * NT;
        vcode[g] = -1;
        pr_[g] = p3_[g] = T(0);
#pragma unroll
        for (int h = 0; h < NP; ++h) e4w_[g][h] = vl_[g][h] = p_splat(T(0));
        if (v < Vs) {
            const int kk = v / (nR * n2v), rem = v % (nR * n2v), i = rem / n2v, jb = rem % n2v;
            const int k = sl * KS + kk;
            vcode[g] = (kk << 20) | (i << 10) | jb;
            const T pr = sp_R[i];
            pr_[g] = pr;
            p3_[g] = sp_3[k];
            const T wik = sw_R[i] * sw_3[k];
#pragma unroll
            for (int h = 0; h < NP; ++h) {
                const int ja = jb * VW + 2 * h, jc = VW == 1 ? ja : ja + 1;
                // WENO5 of f / w (Sec. II.C) taken on f itself: with eps scaled by w^2 the face value
                // of f is w times that of f / w, and the flux needs no division by the weight.  In
                // FP32 eps w^2 is kept above the float range's floor (weights below ~1e-16 at large
                // radial orders, whose populations are negligible, reconstruct with linear weights)
                const T wa = wik * sw_2[ja], wc = wik * sw_2[jc];
                e4w_[g][h] = sizeof(T) == 4 ? p_make(fmax(T(4e-6) * wa * wa, T(1e-37)), fmax(T(4e-6) * wc * wc, T(1e-37)))
                                            : p_make(T(4e-6) * wa * wa, T(4e-6) * wc * wc);
            }
            if (c0 == 0 && pr > T(0)) {
                const V2 gik = p_splat(nwL * gwL[i] * gwL[nR + n2 + k]);
#pragma unroll
                for (int h = 0; h < NP; ++h) {
                    const int ja = jb * VW + 2 * h, jc = VW == 1 ? ja : ja + 1;
                    vl_[g][h] = p_mul(gik, p_make(gwL[nR + ja], gwL[nR + jc]));
                }
            } else {
                // rows of cells c0-3..c0+1 (p_R > 0) or c0-2..c0+2 (p_R < 0), ascending
                const T* b = fs + (long long)(pr > T(0) ? 0 : 1) * Ms + v * VW;
                const V2 s3 = p_splat(pr > T(0) ? T(3) : T(-3)), ns3 = p_splat(pr > T(0) ? T(-3) : T(3));
                const V2 dL = p_splat(pr > T(0) ? T(0.1) : T(0.3)), dR = p_splat(pr > T(0) ? T(0.3) : T(0.1));
                V2 r0[NP], r1[NP], r2[NP], r3[NP], r4[NP];
                ld_pairs<T, VW>(b, r0);
                ld_pairs<T, VW>(b + Ms, r1);
                ld_pairs<T, VW>(b + 2 * Ms, r2);
                ld_pairs<T, VW>(b + 3 * Ms, r3);
                ld_pairs<T, VW>(b + 4 * Ms, r4);
#pragma unroll
                for (int h = 0; h < NP; ++h)
                    vl_[g][h] = weno5_pair<T>(r0[h], r1[h], r2[h], r3[h], r4[h], s3, ns3, dL, dR, e4w_[g][h]);
            }
        }
    }

    const T dt = sizeof(T) == 4 ? (T)I.f_dt : (T)I.dt;
    const T ca_ = sizeof(T) == 4 ? (T)A.fa : (T)A.a, cb_ = sizeof(T) == 4 ? (T)A.fb : (T)A.b;
    for (int cl = 0; cl < Be; ++cl) {
        const int c = c0 + cl;
        const T* ct = cellT + cl * rs;
        T sc[20];
#pragma unroll
        for (int q = 0; q < 20; q += 4) {
            T t4[4];
            ld_vec<T, 4>(ct + q, t4);
            sc[q] = t4[0]; sc[q + 1] = t4[1]; sc[q + 2] = t4[2]; sc[q + 3] = t4[3];
        }
        const T n = sc[0], u0 = sc[1], u1 = sc[2], u2 = sc[3], iT = sc[4], itau = sc[5], cS = sc[6];
        const T q0 = sc[7], q1 = sc[8], q2 = sc[9], nbr = sc[10], X = sc[11], Y = sc[12];
        const T S00 = sc[13], J2c = sc[14], S22 = sc[15], g1c = sc[16], S02 = sc[17], hiT = sc[18], dv = sc[19];
        // collision terms of the cell that do not depend on the momentum (see below; the closure
        // stores -b rho chi, 0.4 S_11 / T, 2 S_01 / T and 1 / (2T) as they are used here)
        const T fiT = T(0.2) * iT, F3 = cS * fiT * q1;
        const T* g2c = ct + rec_off_g2();
        const T* gRc = ct + rec_off_gR(n2);
        const T* g3c = ct + rec_off_g3(nR, n2);
        const T Ap = sgeo[cl * 3 + 0], Am = sgeo[cl * 3 + 1], kf = sgeo[cl * 3 + 2];
        const T* fc = fs + (long long)(cl + 3) * Ms;  // row of cell c
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = T(0);
#pragma unroll
        for (int g = 0; g < NV; ++g) {
            const int cd = vcode[g];
            if (cd >= 0) {
                const int kk = cd >> 20, i = (cd >> 10) & 1023, jb = cd & 1023;
                const int k = sl * KS + kk;
                const int vb = ((kk * nR + i) * n2v + jb) * VW;  // element offset in the slice
                const long long gidx = I.f_off + (long long)c * Np + slice_off + vb;
                const T pr = pr_[g], p3v = p3_[g];
                // f_n for the RK combination, requested first so that its latency overlaps the update.
                // f_n: read-only for the stage kernel; written earlier in the same launch for the
                // persistent step kernel, which reads it coherently (L2)
                V2 fnv[NP];
                const bool use_fn = A.mode == 0 && ca_ != T(0);
                if (use_fn) {
                    if constexpr (kCoherent)
                        ldcg_pairs<T, VW>(f_n + gidx, fnv);
                    else
                        ldg_pairs<T, VW>(f_n + gidx, fnv);
                }
                // advection: WENO5 value at the right face, upwind by sign(p_R)
                V2 vr[NP];
                if (c == N - 1 && pr < T(0)) {
                    const V2 gik = p_splat(nwR * gwR[i] * gwR[nR + n2 + k]);
#pragma unroll
                    for (int h = 0; h < NP; ++h) {
                        const int ja = jb * VW + 2 * h, jc = VW == 1 ? ja : ja + 1;
                        vr[h] = p_mul(gik, p_make(gwR[nR + ja], gwR[nR + jc]));
                    }
                } else {
                    // rows of cells c-2..c+2 (p_R > 0) or c-1..c+3 (p_R < 0), ascending
                    const T* b = fc + (pr > T(0) ? -2 * Ms : -Ms) + vb;
                    const V2 s3 = p_splat(pr > T(0) ? T(3) : T(-3)), ns3 = p_splat(pr > T(0) ? T(-3) : T(3));
                    const V2 dL = p_splat(pr > T(0) ? T(0.1) : T(0.3)), dR = p_splat(pr > T(0) ? T(0.3) : T(0.1));
                    V2 r0[NP], r1[NP], r2[NP], r3[NP], r4[NP];
                    ld_pairs<T, VW>(b, r0);
                    ld_pairs<T, VW>(b + Ms, r1);
                    ld_pairs<T, VW>(b + 2 * Ms, r2);
                    ld_pairs<T, VW>(b + 3 * Ms, r3);
                    ld_pairs<T, VW>(b + 4 * Ms, r4);
#pragma unroll
                    for (int h = 0; h < NP; ++h)
                        vr[h] = weno5_pair<T>(r0[h], r1[h], r2[h], r3[h], r4[h], s3, ns3, dL, dR, e4w_[g][h]);
                }
                // curvature force: K^h along i (one column shared by the vector), K_2 along j; each
                // output sums its terms in the order of the contracted index
                V2 KRf[NP], K2f[NP], K3f[NP];
#pragma unroll
                for (int h = 0; h < NP; ++h) KRf[h] = K2f[h] = K3f[h] = p_splat(T(0));
                {
                    if (kMMA && use_mma) {
                        ld_pairs<T, VW>(skrf + (long long)cl * Ms + vb, KRf);
                    } else if (A.krf) {
                        // from the contraction kernel, in the layout of f
                        ldg_pairs<T, VW>(reinterpret_cast<const T*>(A.krf) + I.f_off + (long long)c * Np + slice_off + vb, KRf);
                    } else {
                        const T* col = fc + kk * nR * n2 + jb * VW;
                        const T* kr = sKR + i * krs;
                        if constexpr (sizeof(T) == 4 && NR_ > 0 && NR_ % 4 == 0) {
                            // four entries of the K^h row per vector load
#pragma unroll 2
                            for (int a4 = 0; a4 < NR_; a4 += 4) {
                                T kq[4];
                                ld_vec<T, 4>(kr + a4, kq);
#pragma unroll
                                for (int t = 0; t < 4; ++t) {
                                    V2 cv[NP];
                                    ld_pairs<T, VW>(col + (a4 + t) * n2, cv);
                                    const V2 kv = p_splat(kq[t]);
#pragma unroll
                                    for (int h = 0; h < NP; ++h) KRf[h] = p_fma(kv, cv[h], KRf[h]);
                                }
                            }
                        } else {
#pragma unroll 8
                            for (int a = 0; a < nR; ++a) {
                                V2 cv[NP];
                                ld_pairs<T, VW>(col + a * n2, cv);
                                const V2 kv = p_splat(kr[a]);
#pragma unroll
                                for (int h = 0; h < NP; ++h) KRf[h] = p_fma(kv, cv[h], KRf[h]);
                            }
                        }
                    }
                    // K_2 from its transpose: input b's coefficients for the vector's outputs
                    const T* row = fc + (kk * nR + i) * n2;
                    const T* k2 = sK2 + jb * VW;
#pragma unroll 2
                    for (int b4 = 0; b4 < n2v; ++b4) {
                        T rv[VW];
                        ld_vec<T, VW>(row + b4 * VW, rv);
#pragma unroll
                        for (int t = 0; t < VW; ++t) {
                            V2 kq[NP];
                            ld_pairs<T, VW>(k2 + (b4 * VW + t) * n2, kq);
                            const V2 fv1 = p_splat(rv[t]);
#pragma unroll
                            for (int h = 0; h < NP; ++h) K2f[h] = p_fma(kq[h], fv1, K2f[h]);
                        }
                    }
                    if (GEOM == 1 && A.k3f) {
                        // sliced along p_3: from the contraction kernel, in the layout of f
                        ldg_pairs<T, VW>(reinterpret_cast<const T*>(A.k3f) + I.f_off + (long long)c * Np + slice_off + vb, K3f);
                    } else if (GEOM == 1) {
                        const T* k3 = sK3 + k * (n3 + 1);
                        const T* c3 = fc + i * n2 + jb * VW;
#pragma unroll 4
                        for (int b = 0; b < n3; ++b) {
                            V2 cv[NP];
                            ld_pairs<T, VW>(c3 + b * nR * n2, cv);
                            const V2 kv = p_splat(k3[b]);
#pragma unroll
                            for (int h = 0; h < NP; ++h) K3f[h] = p_fma(kv, cv[h], K3f[h]);
                        }
                    }
                }
                // collision: -(f - f^S)/tau + J1[f^MB] (Eqs. j0, j1).  With x = p - u and
                // x1 = p_2 - u_2 the only coordinate that varies along the vector, the Shakhov
                // factor f^S / f^MB = 1 + c_S (|x|^2 / (5 T) - 1) x.q is a cubic in x1 and J1 / f^MB
                // (which holds |x|^2 / (2T) - 5/2 and the strain x.S.x / T) a quadratic: their
                // coefficients are formed once per vector, then two Horner evaluations per momentum.
                V2 fv[NP], g2v[NP], p2v[NP], p2q[NP];
                ld_pairs<T, VW>(fc + vb, fv);
                ld_pairs<T, VW>(g2c + jb * VW, g2v);
                ld_pairs<T, VW>(sp_2 + jb * VW, p2v);
#pragma unroll
                for (int h = 0; h < NP; ++h) p2q[h] = p_mul(p2v[h], p2v[h]);
                const T x0 = pr - u0, x2 = p3v - u2;
                T xsA = x0 * x0 + x2 * x2;
                const T xqA = x0 * q0 + x2 * q2;
                if (N3_ == 0 && M.reduced) {
                    // cylinder with p_z integrated out (p_3 = u_3 = 0 here): the p_z^2 in |x|^2
                    // becomes T for phi (k = 0), 3T for chi (k = 1); chi's T factor is in g_3
                    xsA += (k == 0 ? T(1) : T(3)) / iT;
                }
                const T stA = x0 * x0 * S00 + x2 * x2 * S22 + T(2) * x0 * x2 * S02;
                const T fmbA = n * gRc[i] * g3c[k];
                const T Yd = T(0.6) * x0 * Y + T(0.4) * dv;
                const T J0 = nbr * (x0 * X + Yd * (hiT * xsA - T(2.5)) + T(0.4) * iT * stA);
                const T J1 = nbr * T(0.4) * g1c * x0;
                const T J2 = nbr * (Yd * hiT + J2c);
                const T b0 = fiT * xsA - T(1), cb0 = cS * b0;
                const T F0 = T(1) + cb0 * xqA, F1 = cb0 * q1, F2 = cS * fiT * xqA;
                // the advection and force terms enter negated: -(p_R A+/V vr - p_R A-/V vl) (face
                // values are of f) and -frc, each formed with one rounding like its positive
                const V2 npAp = p_splat(-(pr * Ap)), pAm = p_splat(pr * Am);
                const V2 pu1 = p_splat(u1), pfmbA = p_splat(fmbA), pitau = p_splat(itau);
                const V2 pF0 = p_splat(F0), pF1 = p_splat(F1), pF2 = p_splat(F2), pF3 = p_splat(F3);
                const V2 pJ0 = p_splat(J0), pJ1 = p_splat(J1), pJ2 = p_splat(J2);
                V2 out[NP];
#pragma unroll
                for (int h = 0; h < NP; ++h) {
                    const V2 nadv = p_fma(npAp, vr[h], p_mul(pAm, vl_[g][h]));
                    vl_[g][h] = vr[h];
                    V2 nfrc;
                    if (GEOM == 0) {
                        // -kf (p_2^2 K^h f - p_R K_2 f)
                        nfrc = p_mul(p_splat(-kf), p_fma(p2q[h], KRf[h], p_mul(p_splat(-pr), K2f[h])));
                    } else {
                        // -((kf p_2^2 + kf p_3^2) K^h f - kf p_R (K_2 f + K_3 f))
                        const V2 na = p_fma(p_splat(-kf), p2q[h], p_splat(-(kf * p3v * p3v)));
                        nfrc = p_fma(na, KRf[h], p_mul(p_splat(kf * pr), p_add(K2f[h], K3f[h])));
                    }
                    const V2 x1 = p_sub(p2v[h], pu1);
                    const V2 fmb = p_mul(pfmbA, g2v[h]);
                    const V2 fS = p_mul(fmb, p_fma(p_fma(p_fma(pF3, x1, pF2), x1, pF1), x1, pF0));
                    const V2 j1 = p_fma(p_fma(pJ2, x1, pJ1), x1, pJ0);
                    out[h] = p_fma(fmb, j1, p_fma(p_sub(fS, fv[h]), pitau, p_add(nadv, nfrc)));
                }
                if (A.mode == 0) {
                    // a f_n + b (f + dt L) with a = 1 - b, written as f_n + b ((f - f_n) + dt L):
                    // exactly affine whatever the rounding of b (in FP32, fl(1/3) + fl(2/3)
                    // exceeds one by 3e-8, which would scale the state by that much every step)
                    const V2 pdt = p_splat(dt);
                    if (use_fn) {
                        const V2 pcb = p_splat(cb_);
#pragma unroll
                        for (int h = 0; h < NP; ++h) out[h] = p_fma(pcb, p_fma(pdt, out[h], p_sub(fv[h], fnv[h])), fnv[h]);
                    } else {
#pragma unroll
                        for (int h = 0; h < NP; ++h) out[h] = p_fma(pdt, out[h], fv[h]);
                    }
                }
                st_pairs<T, VW>(f_out + gidx, out);
                // raw sums: power sums over the vector's p_2 (per lane of the pairs, then the two
                // lanes), then the 13 moments
                V2 ps1 = p_mul(out[0], p2v[0]);
                V2 ps0 = out[0], ps2 = p_mul(out[0], p2q[0]), ps3 = p_mul(ps1, p2q[0]);
#pragma unroll
                for (int h = 1; h < NP; ++h) {
                    const V2 o1 = p_mul(out[h], p2v[h]);
                    ps0 = p_add(ps0, out[h]);
                    ps1 = p_add(ps1, o1);
                    ps2 = p_fma(out[h], p2q[h], ps2);
                    ps3 = p_fma(o1, p2q[h], ps3);
                }
                const T s0 = VW == 1 ? ps0.x : ps0.x + ps0.y, s1 = VW == 1 ? ps1.x : ps1.x + ps1.y;
                const T s2 = VW == 1 ? ps2.x : ps2.x + ps2.y, s3 = VW == 1 ? ps3.x : ps3.x + ps3.y;
                const T prs0 = pr * s0, p3s0 = p3v * s0, rr = pr * pr + p3v * p3v;
                const T e10 = rr * s0 + s2;  // sum out (p_R^2 + p_2^2 + p_3^2)
                if (N3_ == 0 && M.reduced && k == 1) {
                    // chi = int p_z^2 f: it enters S2_zz and the p_z^2 p_a part of S3_a only
                    acc[6] += s0;
                    acc[10] += prs0;
                    acc[11] += s1;
                    continue;
                }
                acc[0] += s0;
                acc[1] += prs0;
                acc[2] += s1;
                acc[3] += p3s0;
                acc[4] += pr * prs0;
                acc[5] += s2;
                acc[6] += p3v * p3s0;
                acc[7] += pr * s1;
                acc[8] += pr * p3s0;
                acc[9] += p3v * s1;
                acc[10] += pr * e10;
                acc[11] += rr * s1 + s3;
                acc[12] += p3v * e10;
            }
        }
        // ---- 5. warp sums of the 13 raw moments of this cell (lane L holds sum L/2)
        if (A.mode == 0) {
            const T s = warp_sum16_transposed(acc, lane);
            if (!(lane & 1) && (lane >> 1) < kSums) red[(cl * nwarps + warp) * 16 + (lane >> 1)] = s;
        }
    }
    __syncthreads();
    if (A.mode == 0) {
        // sums over the warps in a fixed pairwise tree, to FP64.  FP32 partials: a double-float
        // tree (error-free first level, ~44 bits after), converted once (exact); the FP64 pipe is
        // slow on this part and the sums are the tail of every item.  FP64 partials: FP64.
        // The tree over 16 slots (at most 512 threads), the slots beyond the block's warps zero; it
        // is taken over the smallest power of two of slots that holds the warps, since the levels
        // above add exact zeros (the same sums bit for bit, without their instructions).
        auto tree = [&](auto kWc, int cl, int q) -> double {
            constexpr int kW = decltype(kWc)::value;
            if constexpr (sizeof(T) == 4) {
                Wide<float> v[kW];
#pragma unroll
                for (int ww = 0; ww < kW; ++ww) v[ww] = w_from_t(ww < nwarps ? (float)red[(cl * nwarps + ww) * 16 + q] : 0.f);
#pragma unroll
                for (int h = kW / 2; h > 0; h >>= 1)
#pragma unroll
                    for (int ww = 0; ww < h; ++ww) v[ww] = w_add(v[ww], v[ww + h]);
                // the pair itself for the closure (its split of the sum: hi = fl(s), lo = s - hi)
                const long long cs = (long long)(I.cell_off + c0 + cl) * M.slices + sl;
                reinterpret_cast<float2*>(A.sumsw_out)[cs * kSums + q] = make_float2(v[0].hi, v[0].lo);
                return (double)v[0].hi + (double)v[0].lo;
            } else {
                double v[kW];
#pragma unroll
                for (int ww = 0; ww < kW; ++ww) v[ww] = ww < nwarps ? (double)red[(cl * nwarps + ww) * 16 + q] : 0.0;
#pragma unroll
                for (int h = kW / 2; h > 0; h >>= 1)
#pragma unroll
                    for (int ww = 0; ww < h; ++ww) v[ww] = v[ww] + v[ww + h];
                return v[0];
            }
        };
        for (int e = tid; e < Be * kSums; e += NT) {
            const int cl = e / kSums, q = e % kSums;
            double s;
            if (nwarps <= 4)
                s = tree(std::integral_constant<int, 4>{}, cl, q);
            else if (nwarps <= 8)
                s = tree(std::integral_constant<int, 8>{}, cl, q);
            else
                s = tree(std::integral_constant<int, 16>{}, cl, q);
            const long long cs = (long long)(I.cell_off + c0 + cl) * M.slices + sl;
            A.sums_out[cs * kSums + q] = s;
            if (q == 0) reinterpret_cast<T*>(A.dens_out)[cs] = (T)s;
        }
    }
    __syncthreads();  // the next item overwrites the staged rows, the records and the sums
}

template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
__device__ __forceinline__ void stream_body(const StageArgs& A, const MomSet& M) {
    __shared__ T snw[2];  // wall densities of the item's instance
    const int tid = threadIdx.x;
    stream_tables<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M);
    // The rows of the first item are requested before the wait: they are the output of the stage
    // kernel two launches back, complete once the closure kernel in between has passed its own
    // wait, which it does before it lets this kernel start.  The records (the closure's output)
    // follow the wait.
    const int nit = *A.n_items;
    const bool early = A.use_bulk && blockIdx.x < nit;
    if (early) {
        const int4 wi = A.items[blockIdx.x];
        stream_issue<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, wi, A.inst[wi.x], true, 1);
    }
    __syncthreads();
    pdl_trigger();
    pdl_wait();  // everything below reads what the previous kernels wrote
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 wi = A.items[it];
        const InstDev I = A.inst[wi.x];
        stream_issue<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, wi, I, true, (early && it == blockIdx.x) ? 2 : 3);
        // geometry, wall Maxwellians and the wall densities from the parts of the outgoing
        // fluxes, overlapping the copy
        stream_statics<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, wi, I);
        if (tid < 2) {
            const T* pp = reinterpret_cast<const T*>(A.nwp) + ((long long)wi.x * 2 + tid) * A.wall_parts;
            T sum = T(0);
            for (int p = 0; p < A.wall_parts; ++p) sum += pp[p];
            const T iden = sizeof(T) == 4 ? (T)(tid ? I.f_nw_iden[1] : I.f_nw_iden[0])
                                          : (T)(tid ? I.nw_iden[1] : I.nw_iden[0]);
            snw[tid] = sum * iden;
        }
        if (!stream_wait<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, phase)) return;
        if (!A.use_bulk) __syncthreads();  // the bulk path's wait ends with a block-wide vote
        stream_compute<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, wi, I, snw[0], snw[1]);
    }
}

// The stage kernel; MINB = the blocks per SM the register allocation is bounded for: 1 (up to 512
// threads, 128 registers each: two blocks of 256 threads reside) or, for blocks of at most 256
// threads, 3 (at most 85 registers each); for the row kernel (VW = 8, blocks of at most 128
// threads) 5, 3 or 2 (at most 102, 170 or 255 registers each; five blocks fit in shared memory
// with tiles of up to three cells).  The arithmetic and its order are the same in all.
template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_, int MINB>
__global__ void __launch_bounds__(MINB == 1 ? 512 : (VW == 8 ? 128 : 256), MINB) stream_kernel(StageArgs A, MomSet M) {
    stream_body<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M);
}


template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_, int MINB = 1>
cudaError_t launch_stream_t(const StageArgs& A, const MomSet& M, int grid, int threads, size_t smem, cudaStream_t s) {
    auto kern = stream_kernel<T, GEOM, VW, NV, NR_, N2_, N3_, MINB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_maybe_programmatic(kern, grid, threads, smem, s, A.programmatic, A, M);
}

// Instantiations: generic shapes (VW 1, 2, 4 for float; 1, 2 for double) and the compile-time
// shapes of the cylinder (16 x 8 x 8) and sphere (24 x 12 x 12) workloads.
template <typename T, int G>
cudaError_t launch_stream_dispatch(const StreamCfg& cfg, const StageArgs& A, const MomSet& M, int grid, int threads,
                                   size_t smem, cudaStream_t s) {
    constexpr int VS = sizeof(T) == 4 ? 4 : 2;  // vector width of the compile-time shapes
    constexpr int SR = G == 0 ? 16 : 24, S2 = G == 0 ? 8 : 12, S3 = G == 0 ? 8 : 12;
    constexpr int NA = G == 0 ? 1 : 2, NB = G == 0 ? 2 : 4;
    if (cfg.spec) {
        if constexpr (sizeof(T) == 4 && G == 0) {
            // the cylinder's FP32 shape also as one vector of a whole p_2 row (8 momenta) per thread
            if (cfg.vw == 8 && cfg.nv == 1) {
                if (threads > 128 && cfg.minb != 1) return cudaErrorInvalidValue;
                if (cfg.minb == 5) return launch_stream_t<T, G, 8, 1, SR, S2, S3, 5>(A, M, grid, threads, smem, s);
                if (cfg.minb == 3) return launch_stream_t<T, G, 8, 1, SR, S2, S3, 3>(A, M, grid, threads, smem, s);
                if (cfg.minb == 2) return launch_stream_t<T, G, 8, 1, SR, S2, S3, 2>(A, M, grid, threads, smem, s);
                return launch_stream_t<T, G, 8, 1, SR, S2, S3>(A, M, grid, threads, smem, s);
            }
        }
        if (cfg.vw != VS) return cudaErrorInvalidValue;
        if constexpr (sizeof(T) == 4 && G == 0) {
            // the cylinder's FP32 shape also bounded for three blocks of 256 threads per SM
            if (cfg.minb == 3 && cfg.nv == NA && threads <= 256)
                return launch_stream_t<T, G, VS, NA, SR, S2, S3, 3>(A, M, grid, threads, smem, s);
        }
        if (cfg.nv == NA) return launch_stream_t<T, G, VS, NA, SR, S2, S3>(A, M, grid, threads, smem, s);
        if (cfg.nv == NB) return launch_stream_t<T, G, VS, NB, SR, S2, S3>(A, M, grid, threads, smem, s);
        return cudaErrorInvalidValue;
    }
    if (cfg.vw == 1 && cfg.nv == 4) return launch_stream_t<T, G, 1, 4, 0, 0, 0>(A, M, grid, threads, smem, s);
    if (cfg.vw == 2 && cfg.nv == 4) return launch_stream_t<T, G, 2, 4, 0, 0, 0>(A, M, grid, threads, smem, s);
    if constexpr (sizeof(T) == 4) {
        if (cfg.vw == 4 && cfg.nv == 2) return launch_stream_t<T, G, 4, 2, 0, 0, 0>(A, M, grid, threads, smem, s);
    }
    return cudaErrorInvalidValue;
}

#define FDLB_STREAM_INSTANCE(T, G)                                                                               \
    cudaError_t launch_stream_##T##_##G(const StreamCfg& cfg, const StageArgs& A, const MomSet& M, int grid,    \
                                        int threads, size_t smem, cudaStream_t s) {                              \
        return launch_stream_dispatch<T, G>(cfg, A, M, grid, threads, smem, s);                                  \
    }

}  // namespace fdlb
