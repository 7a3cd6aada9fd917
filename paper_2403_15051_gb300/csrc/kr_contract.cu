// The half-range momentum derivative of the curvature force as its own kernel: Y = K^h X for
// every (cell, p_3 value) block X = f[cell][k][.][.] (2Q_R radial momenta x Q_2 momenta of the
// second axis), with K^h the 2Q_R x 2Q_R matrix of Sec. III.B.  Taken out of the fused stage when
// the radial order is large (the paper's HHLB(7,20) .. HHLB(7,100), Sec. IV): K^h no longer fits
// beside the staged rows in shared memory, and the contraction (2 x 2Q_R flops per population)
// dominates the stage's arithmetic.  The result has the layout of f; the fused stage reads it in
// place of its own contraction.  FP32 populations use the weight-scaled form (see
// kr_cuda_core_kernel): K^h itself leaves the float range at the largest radial orders.
//
// Seen as one GEMM: rows i of K^h against the columns (block, j) of X, the blocks of a stage work
// item (instance, first cell, cells, slice) being contiguous in memory.  Two forms:
//  * CUDA cores (any precision): 64 x 64 output tiles, K^h and X chunks of 16 in shared memory,
//    4 x 4 outputs per thread;
//  * 5th-generation tensor cores (FP32 populations): tcgen05.mma kind::tf32 with the FP32 operands
//    split into TF32 pairs (x = x_hi + x_lo) and the three products K_hi X_hi + K_hi X_lo +
//    K_lo X_hi accumulated in FP32 in tensor memory, which keeps FP32-level accuracy (the dropped
//    K_lo X_lo and the TF32 rounding of the low parts are ~2^-22 of the product).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"
#include "kernels_decl.h"

namespace fdlb {
namespace {

constexpr int kTile = 64;   // output rows and columns per tile
constexpr int kChunk = 16;  // contraction chunk

// With isw and sw (FP32 populations) the product runs in the weight-scaled form
// (K^h f)_i = sw_i sum_a Khat_ia (isw_a f_a): Khat = K^h scaled by sqrt(w_a / w_i) (radial weights
// w) has entries of order one, where K^h itself spans ~1e-100 .. 1e+100 at the largest radial
// orders and leaves the float range; sw = sqrt(w), isw = 1/sqrt(w) (zero where it exceeds the
// float range: those populations are zero in FP32).  Without them, KR is K^h itself.
template <typename T>
__global__ void __launch_bounds__(256) kr_cuda_core_kernel(const T* __restrict__ f, T* __restrict__ out,
                                                           const int4* __restrict__ items, const int* __restrict__ n_items,
                                                           const InstDev* __restrict__ inst, const T* __restrict__ KR,
                                                           const T* __restrict__ isw, const T* __restrict__ sw,
                                                           MomSet M) {
    __shared__ T Ks[kChunk][kTile + 1];  // [a][i]: K^h chunk, transposed
    __shared__ T Xs[kChunk][kTile];      // [a][column]
    const int nR = M.nR, n2 = M.n2, KS = M.KS, Np = M.Np;
    const int tid = threadIdx.x, tr = tid / 16, tc = tid % 16;
    const int nit = *n_items;
    const int row_tiles = (nR + kTile - 1) / kTile;
    // work units: (item, row tile, column tile), column tiles counted up to the largest item
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = items[it];
        const InstDev I = inst[w.x];
        const int ncols = w.z * KS * n2;
        const T* fb = f + I.f_off;
        T* ob = out + I.f_off;
        for (int rt = 0; rt < row_tiles; ++rt)
            for (int col0 = 0; col0 < ncols; col0 += kTile) {
                const int r0 = rt * kTile;
                T acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[r][q] = T(0);
                for (int a0 = 0; a0 < nR; a0 += kChunk) {
                    for (int e = tid; e < kTile * kChunk; e += blockDim.x) {
                        const int row = e / kChunk, kk = e % kChunk, i = r0 + row, a = a0 + kk;
                        Ks[kk][row] = (i < nR && a < nR) ? KR[(long long)i * nR + a] : T(0);
                    }
                    for (int e = tid; e < kTile * kChunk; e += blockDim.x) {
                        const int kk = e / kTile, cc = e % kTile, a = a0 + kk, col = col0 + cc;
                        T v = T(0);
                        if (a < nR && col < ncols) {
                            const int blk = col / n2, j = col % n2;
                            const int c = w.y + blk / KS, k = w.w * KS + blk % KS;
                            v = fb[(long long)c * Np + ((long long)k * nR + a) * n2 + j];
                            if (isw) v *= isw[a];
                        }
                        Xs[kk][cc] = v;
                    }
                    __syncthreads();
#pragma unroll 4
                    for (int kk = 0; kk < kChunk; ++kk) {
                        T kv[4], xv[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) kv[r] = Ks[kk][tr * 4 + r];
#pragma unroll
                        for (int q = 0; q < 4; ++q) xv[q] = Xs[kk][tc * 4 + q];
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int q = 0; q < 4; ++q) acc[r][q] += kv[r] * xv[q];
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = r0 + tr * 4 + r, col = col0 + tc * 4 + q;
                        if (i < nR && col < ncols) {
                            const int blk = col / n2, j = col % n2;
                            const int c = w.y + blk / KS, k = w.w * KS + blk % KS;
                            ob[(long long)c * Np + ((long long)k * nR + i) * n2 + j] = sw ? sw[i] * acc[r][q] : acc[r][q];
                        }
                    }
            }
    }
}

// ------------------------------------------------------------------------ tensor cores
// One CTA of 128 threads per SM, persistent over the stage items.  A tile is 128 consecutive
// columns of an item's X (the MMA's M); the accumulator D[m][n] = sum_a X[a][m] K^h[n][a] holds the
// tile's K^h X transposed, M = 128 lanes by N = 2Q_R rounded up to 16 columns of tensor memory.
// The contraction runs in chunks of 32 values of a: per chunk the threads load the 32 x 128 block
// of X (coalesced), split it into TF32 pairs and write both parts into shared memory in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices, 128 bytes each: element
// (row r, k) at (r / 8) * 1024 + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4 bytes), while the bulk
// copy engine brings the chunk's K^h pair, laid out the same way on the host; one thread issues the
// chunk's MMAs (K = 8 each, three per K-step) and commits them to an mbarrier.  Two buffers: the
// next chunk is staged while the tensor cores work on this one.  The epilogue reads the
// accumulator with tcgen05.ld (warp w reads lanes 32w..32w+31) and stores K^h f in the layout of f.
// Every wait is bounded: a wait that runs out sets the error flag, the block drains what it issued
// (bounded), frees its tensor memory and leaves.
constexpr int kUM = 128;        // columns of X per tile (MMA M)
constexpr int kUK = 32;         // values of a per staged chunk
constexpr int kTmemCols = 256;  // accumulator columns allocated (N <= 208)
constexpr int kAPart = kUM * kUK * 4;  // bytes of one TF32 part of an X chunk (16 KB)

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    // shared-memory matrix descriptor: start address >> 4, leading byte offset (between the core
    // matrices along K) 128 >> 4, stride byte offset (between 8-row groups) 1024 >> 4, descriptor
    // version 1, no base offset, no swizzle
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128, 1) kr_tc_kernel(const float* __restrict__ f, float* __restrict__ out,
                                                       const int4* __restrict__ items, const int* __restrict__ n_items,
                                                       const InstDev* __restrict__ inst, const float* __restrict__ Bsplit,
                                                       const float* __restrict__ isw, const float* __restrict__ sw,
                                                       MomSet M, int Npad, int* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bfull[2], mdone[2], drain;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nR = M.nR, n2 = M.n2, KS = M.KS, Np = M.Np;
    const int Kp8 = (nR + 7) & ~7, nk = (Kp8 + kUK - 1) / kUK;
    const uint32_t bpart = (uint32_t)Npad * 128u, bbytes = 2u * bpart;  // one TF32 part, the pair
    // 1024-byte aligned buffers: X pairs [2][hi | lo], K^h pairs [2][hi | lo]
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const uint32_t sA[2] = {sbase, sbase + 2u * kAPart};
    const uint32_t sB[2] = {sbase + 4u * kAPart, sbase + 4u * kAPart + bbytes};
    unsigned char* gA[2] = {gbase, gbase + 2 * kAPart};
    if (tid == 0) {
        mbar_init(&bfull[0], 1);
        mbar_init(&bfull[1], 1);
        mbar_init(&mdone[0], 1);
        mbar_init(&mdone[1], 1);
        mbar_init(&drain, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = umma_idesc_tf32(kUM, Npad);
    bool fail = false;
    int g = 0;                  // chunks staged by this block so far
    int pend_b = -1;            // buffer of an outstanding K^h copy (thread 0), -1 none
    const int nit = *n_items;
    for (int it = blockIdx.x; it < nit && !fail; it += gridDim.x) {
        const int4 w = items[it];
        const InstDev I = inst[w.x];
        const int ncols = w.z * KS * n2;
        for (int col0 = 0; col0 < ncols && !fail; col0 += kUM) {
            // this thread's column of the tile (row m = tid of the MMA's A)
            const int col = col0 + tid;
            const bool valid = col < ncols;
            long long base = 0;
            if (valid) {
                const int blk = col / n2, j = col % n2;
                const int c = w.y + blk / KS, k = w.w * KS + blk % KS;
                base = I.f_off + (long long)c * Np + (long long)k * nR * n2 + j;
            }
            for (int kc = 0; kc < nk; ++kc, ++g) {
                const int b = g & 1;
                const uint32_t use = (uint32_t)(g >> 1);
                // 1. the buffer is free once the MMAs of two chunks back have completed
                if (g >= 2 && !mbar_wait_bounded(&mdone[b], (use - 1u) & 1u)) fail = true;
                if (__syncthreads_or(fail)) {
                    fail = true;
                    break;
                }
                // 2. the chunk's K^h pair by the bulk copy engine
                if (tid == 0) {
                    mbar_expect_tx(&bfull[b], bbytes);
                    bulk_g2s(gbase + (sB[b] - sbase), Bsplit + (size_t)kc * (bbytes / 4), bbytes, &bfull[b]);
                    pend_b = b;
                }
                // 3. this thread's row of the X chunk as TF32 pairs, four values of a at a time
                unsigned char* ah = gA[b] + (tid >> 3) * 1024 + (tid & 7) * 16;
#pragma unroll 2
                for (int k4 = 0; k4 < kUK / 4; ++k4) {
                    float v[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int a = kc * kUK + k4 * 4 + e;
                        v[e] = (valid && a < nR) ? __ldg(f + base + (long long)a * n2) * __ldg(isw + a) : 0.f;
                    }
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        hi[e] = to_tf32(v[e]);
                        lo[e] = to_tf32(v[e] - __uint_as_float(hi[e]));
                    }
                    *reinterpret_cast<uint4*>(ah + k4 * 128) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4*>(ah + kAPart + k4 * 128) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
                // 4. the writes are visible to the tensor cores
                fence_proxy_async();
                __syncthreads();
                // 5. one thread issues the chunk's MMAs: per K-step of 8, X_hi K_hi + X_hi K_lo + X_lo K_hi
                if (tid == 0) {
                    if (mbar_wait_bounded(&bfull[b], use & 1u))
                        pend_b = -1;
                    else
                        fail = true;  // the copy may still be in flight: drained at the exit
                    tc_fence_after();
                    if (!fail) {
                        const int ksteps = min(kUK / 8, (Kp8 - kc * kUK) / 8);
                        for (int s = 0; s < ksteps; ++s) {
                            const uint64_t a_hi = umma_desc(sA[b] + 256u * s), a_lo = umma_desc(sA[b] + kAPart + 256u * s);
                            const uint64_t b_hi = umma_desc(sB[b] + 256u * s), b_lo = umma_desc(sB[b] + bpart + 256u * s);
                            umma_tf32(tmem, a_hi, b_hi, idesc, (kc > 0 || s > 0) ? 1u : 0u);
                            umma_tf32(tmem, a_hi, b_lo, idesc, 1u);
                            umma_tf32(tmem, a_lo, b_hi, idesc, 1u);
                        }
                    }
                    umma_commit(&mdone[b]);
                }
            }
            // epilogue: the tile's accumulator, once its last chunk's MMAs have completed (a failure
            // of thread 0's copy wait in the last chunk is voted on below, with every thread)
            const int gl = g - 1;
            if (!mbar_wait_bounded(&mdone[gl & 1], ((uint32_t)(gl >> 1)) & 1u)) fail = true;
            if (__syncthreads_or(fail)) {
                fail = true;
                break;
            }
            tc_fence_after();
            const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
            for (int n0 = 0; n0 < Npad; n0 += 16) {
                float v[16];
                tmem_ld16(trow + (uint32_t)n0, v);
                if (valid) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int n = n0 + q;
                        if (n < nR) out[base + (long long)n * n2] = __ldg(sw + n) * v[q];
                    }
                }
            }
            tc_fence_before();  // the next tile's first MMA overwrites the accumulator
        }
    }
    // drain what this block issued, then free the tensor memory
    if (fail && tid == 0) atomicOr(err, 1);
    if (tid == 0) {
        if (pend_b >= 0) mbar_wait_bounded(&bfull[pend_b], ((uint32_t)((g - 1) >> 1)) & 1u);
        umma_commit(&drain);
        mbar_wait_bounded(&drain, 0u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

template <typename T>
cudaError_t launch_kr_contract(const T* f, T* out, const int4* items, const int* n_items, const InstDev* inst,
                               const T* KR, const T* isw, const T* sw, const MomSet& M, int grid, cudaStream_t s) {
    kr_cuda_core_kernel<T><<<grid, 256, 0, s>>>(f, out, items, n_items, inst, KR, isw, sw, M);
    return cudaPeekAtLastError();
}

// ------------------------------------------------------------------------------ K_3 (sphere)
// The third axis's derivative matrix of the sphere's curvature force (Sec. III.B, full range) as
// its own pass: out[c][k][i][j] = sum_b K_3[k][b] f[c][b][i][j], b in increasing order as the fused
// stage sums it (the same values).  Taken out of the stage so that the stage can slice the momenta
// along p_3 (the sphere's force otherwise couples every axis and one slice must hold all of a
// cell's momenta).  A block per work item of slice 0 (each cell once), a thread per (i, j) column:
// the n3 inputs of a column are read coalesced across the threads, its n3 outputs written so.
// N3: the compile-time axis size, 0 for any size up to kMaxQ3.
constexpr int kMaxQ3 = 24;

template <typename T, int N3>
__global__ void __launch_bounds__(256) k3_contract_kernel(const T* __restrict__ f, T* __restrict__ out,
                                                          const int4* __restrict__ items, const int* __restrict__ n_items,
                                                          const InstDev* __restrict__ inst, const T* __restrict__ K3,
                                                          MomSet M) {
    constexpr int NB = N3 ? N3 : kMaxQ3;
    __shared__ T sK[NB * NB];
    const int n3 = N3 ? N3 : M.n3;
    for (int e = threadIdx.x; e < n3 * n3; e += blockDim.x) sK[(e / n3) * NB + e % n3] = K3[e];
    __syncthreads();
    const int cols = M.nR * M.n2;
    const int nit = *n_items;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = items[it];
        if (w.w != 0) continue;  // slice 0 covers the item's cells once
        const InstDev& I = inst[w.x];
        for (int cl = 0; cl < w.z; ++cl) {
            const long long base = I.f_off + (long long)(w.y + cl) * M.Np;
            for (int col = threadIdx.x; col < cols; col += blockDim.x) {
                T v[NB];
#pragma unroll
                for (int b = 0; b < NB; ++b) v[b] = b < n3 ? f[base + (long long)b * cols + col] : T(0);
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    if (k >= n3) break;
                    T acc = T(0);
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        if (b < n3) acc += sK[k * NB + b] * v[b];
                    out[base + (long long)k * cols + col] = acc;
                }
            }
        }
    }
}

template <typename T>
cudaError_t launch_k3_contract(const T* f, T* out, const int4* items, const int* n_items, const InstDev* inst,
                               const T* K3, const MomSet& M, int grid, cudaStream_t s) {
    if (M.n3 > kMaxQ3) return cudaErrorInvalidValue;
    if (M.n3 == 12)
        k3_contract_kernel<T, 12><<<grid, 256, 0, s>>>(f, out, items, n_items, inst, K3, M);
    else
        k3_contract_kernel<T, 0><<<grid, 256, 0, s>>>(f, out, items, n_items, inst, K3, M);
    return cudaPeekAtLastError();
}

template cudaError_t launch_k3_contract<float>(const float*, float*, const int4*, const int*, const InstDev*,
                                               const float*, const MomSet&, int, cudaStream_t);
template cudaError_t launch_k3_contract<double>(const double*, double*, const int4*, const int*, const InstDev*,
                                                const double*, const MomSet&, int, cudaStream_t);

size_t kr_tc_smem_bytes(int Npad) { return 1024 + 4 * (size_t)kAPart + 4 * (size_t)Npad * 128; }

cudaError_t launch_kr_contract_tc(const float* f, float* out, const int4* items, const int* n_items, const InstDev* inst,
                                  const float* Bsplit, const float* isw, const float* sw, const MomSet& M, int Npad,
                                  int* err, int grid, cudaStream_t s) {
    const size_t smem = kr_tc_smem_bytes(Npad);
    cudaError_t e = cudaFuncSetAttribute(kr_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kr_tc_kernel<<<grid, 128, smem, s>>>(f, out, items, n_items, inst, Bsplit, isw, sw, M, Npad, err);
    return cudaPeekAtLastError();
}

template cudaError_t launch_kr_contract<float>(const float*, float*, const int4*, const int*, const InstDev*,
                                               const float*, const float*, const float*, const MomSet&, int,
                                               cudaStream_t);
template cudaError_t launch_kr_contract<double>(const double*, double*, const int4*, const int*, const InstDev*,
                                                const double*, const double*, const double*, const MomSet&, int,
                                                cudaStream_t);

}  // namespace fdlb
