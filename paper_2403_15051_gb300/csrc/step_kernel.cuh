// The persistent step kernel: whole SSP-RK3 steps (Sec. III) in one cooperative launch.
//
// Each block owns work items (tiles of cells; the whole momentum set) for the whole launch and
// keeps the stage's and the closure's tables in shared memory.  Per stage and item:
//   1. the bulk engine copies the rows of cells c0-3 .. c0+Be+2 of the stage input into shared
//      memory while
//   2. the closure of the tile's own cells (closure_cells, the code of the closure kernel) writes
//      their collision records straight into the shared record array; on a tile near a wall,
//      the warps beyond the closure's four sum the outgoing wall flux meanwhile, in the closure
//      kernel's order of the sums;
//   3. the stage's populations and raw sums (stream_compute, the code of the stage kernel).
// Between stages a grid barrier: the next closure reads the raw sums and slice densities of the
// cells of other blocks.  The records, wall densities and results are those of the closure and
// stage kernels, bit for bit; what goes away is two launches and two table loads per stage.
//
// The grid is co-resident (cooperative launch) and the barrier counter is zero at launch; every
// wait on it is bounded in time, after which the block sets an error flag and leaves.
#pragma once

#include "closure_item.cuh"
#include "stream_kernel.cuh"

namespace fdlb {

constexpr unsigned long long kBarrierLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Generic-proxy global stores of this thread become visible to the bulk-copy engine's reads.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Every block of the grid arrives once; `target` = (barrier index) x (grid size).  True on every
// thread of the block when all arrived, false when they did not within kBarrierLimitNs.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target) {
    fence_proxy_async_global();
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned long long t0 = global_ns();
        for (unsigned it = 0;; ++it) {
            if (ld_acquire_gpu(bar) >= target) break;
            if (it >= (1u << 26) || global_ns() - t0 > kBarrierLimitNs) {
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        fence_proxy_async_global();
    }
    return __syncthreads_and(ok) != 0;
}

template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
__global__ void __launch_bounds__(512, 1) step_kernel(StepArgs S, MomSet M) {
    __shared__ T wred[2][kWallParts][kClosureWarps];  // wall flux: warp sums per side and part
    __shared__ __align__(8) uint64_t cbar;            // completion of the band-row copy
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31;
    const int nR = NR_ ? NR_ : M.nR, n2 = N2_ ? N2_ : M.n2, n3 = N3_ ? N3_ : M.n3;
    const int KS = M.KS;  // the sphere runs here with one slice (KS = n3)
    const StreamSmem P = stream_smem_plan(S.st.B, nR * n2 * KS, nR, n2, n3, (int)(blockDim.x >> 5), (int)sizeof(T),
                                          (sizeof(T) == 4 && S.st.mma) ? 1 : 0);
    T* cellT = reinterpret_cast<T*>(smem_raw + P.rec);
    T* fs = reinterpret_cast<T*>(smem_raw + P.fs);
    uint64_t* sbar = reinterpret_cast<uint64_t*>(smem_raw);  // the stage's copy barrier
    const int Ms = nR * n2 * KS;
    // closure region: [staged band rows | tables | band-union densities]
    T* wst = reinterpret_cast<T*>(smem_raw + S.clo_off);
    T* ctab = wst + S.cl.wst_elems;
    stream_tables<T, GEOM, VW, NV, NR_, N2_, N3_>(S.st, M);
    const ClosureTabs<T> tb = closure_tables<T>(ctab, S.cl.tabT, M, tid, blockDim.x);
    T* nbuf = ctab + closure_tab_elems(M.nR, M.n2, M.n3);
    if (tid == 0) {
        mbar_init(&cbar, 1);
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t sphase = 0, cphase = 0;
    unsigned nbar = 0;
    const int nit = *S.st.n_items;
    for (int step = 0; step < S.n_steps; ++step) {
        for (int stage = 0; stage < 3; ++stage) {
            // f1 = f + dt L(f); f2 = 3/4 f + 1/4 (f1 + dt L(f1)); f^{n+1} = 1/3 f + 2/3 (f2 + dt L(f2))
            const int in = stage, out = stage == 2 ? 0 : stage + 1;
            const double a = stage == 0 ? 0.0 : (stage == 1 ? 0.75 : 1.0 / 3.0);
            const double b = stage == 0 ? 1.0 : (stage == 1 ? 0.25 : 2.0 / 3.0);
            StageArgs A = S.st;
            ClosureArgs C = S.cl;
            A.f_in = S.f[in];
            A.f_n = S.f[0];
            A.f_out = S.f[out];
            A.sums_out = S.sums[out];
            A.sumsw_out = S.sumsw[out];
            A.dens_out = S.dens[out];
            A.a = a;
            A.b = b;
            A.fa = (float)a;
            A.fb = (float)b;
            C.sums = S.sums[in];
            C.sumsw = S.sumsw[in];
            C.dens = S.dens[in];
            C.f_in = S.f[in];
            if (step > 0 || stage > 0) {
                ++nbar;
                if (!grid_barrier(S.bar, nbar * gridDim.x + (unsigned)S.bar_extra)) {
                    if (tid == 0) atomicOr(A.err, 4);
                    return;
                }
            }
            for (int it = blockIdx.x; it < nit; it += gridDim.x) {
                const int4 wi = A.items[it];
                const InstDev I = A.inst[wi.x];
                const int N = I.n_cells;
                // tiles whose stencils reach a wall's ghost cells need that wall's density
                const bool wl = wi.y < 3, wr = wi.y + wi.z + 2 >= N;
                // 2. the closure of the own cells; the extra warps sum the wall fluxes for a tile
                // near a wall: virtual warp (side, part, w) of the closure kernel's block
                // the four cells next to a wall are among the tile's staged rows (row = cell - c0 + 3):
                // the extra warps wait for the staged copy (bounded) and read them there
                auto walls = [&](int w, int nw) {
                    if (!mbar_wait_bounded(sbar, sphase)) {
                        if (lane == 0) atomicOr(A.err, 1);  // the stage's own wait reports it too
                        return;
                    }
                    const int nv = ((wl ? 1 : 0) + (wr ? 1 : 0)) * kWallParts * kClosureWarps;
                    // four virtual warps at a time: independent chains in flight together
                    for (int v0 = w; v0 < nv; v0 += 4 * nw) {
                        T acc[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int v = v0 + u * nw;
                            acc[u] = T(0);
                            if (v < nv) {
                                const int side = (wl && v < kWallParts * kClosureWarps) ? 0 : 1;
                                const int r = v % (kWallParts * kClosureWarps), part = r / kClosureWarps;
                                const T* wall = fs + (long long)((side == 0 ? 0 : N - 1) - wi.y + 3) * Ms;
                                acc[u] = wall_flux_partial<T>(wall, side == 0 ? (long long)Ms : -(long long)Ms, M, tb, side,
                                                              part, kWallParts, (r % kClosureWarps) * 32 + lane);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int v = v0 + u * nw;
                            if (v < nv) {  // warp-uniform
                                const int side = (wl && v < kWallParts * kClosureWarps) ? 0 : 1;
                                const int r = v % (kWallParts * kClosureWarps);
                                const T a = warp_sum(acc[u]);
                                if (lane == 0) wred[side][r / kClosureWarps][r % kClosureWarps] = a;
                            }
                        }
                    }
                };
                // 1. the rows of the stage input, requested after the closure's loads (the
                // records come from the closure)
                auto rows = [&]() { stream_issue<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, wi, I, false); };
                if (!closure_cells<T>(C, M, tb, I, wi.y, wi.z, cellT, wst, nbuf, &cbar, cphase, walls, rows)) {
                    stream_wait<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, sphase);  // the rows still in flight
                    return;
                }
                stream_statics<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, wi, I);
                // the wall densities as the stage kernel forms them from the parts
                T nw[2] = {T(0), T(0)};
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (side == 0 ? !wl : !wr) continue;
                    T sum = T(0);
                    for (int p = 0; p < kWallParts; ++p) sum += wall_part_sum(wred[side][p]);
                    const T iden = sizeof(T) == 4 ? (T)I.f_nw_iden[side] : (T)I.nw_iden[side];
                    nw[side] = sum * iden;
                }
                // (the wait ends with a block-wide vote: the barrier after the copy and the statics)
                if (!stream_wait<T, GEOM, VW, NV, NR_, N2_, N3_>(A, M, sphase)) return;
                // 3. the stage
                stream_compute<T, GEOM, VW, NV, NR_, N2_, N3_, true>(A, M, wi, I, nw[0], nw[1]);
            }
        }
    }
}

template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
cudaError_t launch_step_t(const StepArgs& S, const MomSet& M, int grid, int threads, size_t smem, cudaStream_t s) {
    auto kern = step_kernel<T, GEOM, VW, NV, NR_, N2_, N3_>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, S, M);
}

template <typename T, int GEOM, int VW, int NV, int NR_, int N2_, int N3_>
cudaError_t step_occupancy_t(int threads, size_t smem, int* blocks_per_sm) {
    auto kern = step_kernel<T, GEOM, VW, NV, NR_, N2_, N3_>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, threads, smem);
}

// The compile-time shapes (cylinder 16 x 8 x 8, sphere 24 x 12 x 12) with the vectors per thread
// of the stage kernel's instantiations; other configurations take the closure + stage kernels.
// With blocks_per_sm: the occupancy query instead of the launch.
template <typename T, int G>
cudaError_t step_dispatch(const StreamCfg& cfg, const StepArgs* S, const MomSet& M, int grid, int threads, size_t smem,
                          cudaStream_t s, int* blocks_per_sm) {
    constexpr int VS = sizeof(T) == 4 ? 4 : 2;
    constexpr int SR = G == 0 ? 16 : 24, S2 = G == 0 ? 8 : 12, S3 = G == 0 ? 8 : 12;
    constexpr int NA = G == 0 ? 1 : 2, NB = 2 * NA;
    if (!cfg.spec || cfg.vw != VS) return cudaErrorInvalidValue;
    if (cfg.nv == NA) {
        if (blocks_per_sm) return step_occupancy_t<T, G, VS, NA, SR, S2, S3>(threads, smem, blocks_per_sm);
        return launch_step_t<T, G, VS, NA, SR, S2, S3>(*S, M, grid, threads, smem, s);
    }
    if (cfg.nv == NB) {
        if (blocks_per_sm) return step_occupancy_t<T, G, VS, NB, SR, S2, S3>(threads, smem, blocks_per_sm);
        return launch_step_t<T, G, VS, NB, SR, S2, S3>(*S, M, grid, threads, smem, s);
    }
    return cudaErrorInvalidValue;
}

#define FDLB_STEP_INSTANCE(T, G)                                                                                  \
    cudaError_t launch_step_##T##_##G(const StreamCfg& cfg, const StepArgs* S, const MomSet& M, int grid,         \
                                      int threads, size_t smem, cudaStream_t s, int* blocks_per_sm) {             \
        return step_dispatch<T, G>(cfg, S, M, grid, threads, smem, s, blocks_per_sm);                             \
    }

}  // namespace fdlb
