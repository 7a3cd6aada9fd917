// Auxiliary kernels of the FDLB step (raw sums, closure, residual); the fused stage kernel is
// in stream_kernel.cuh.  See kernels.cuh for the data layout and the launch plan.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"
#include "kernels_decl.h"
#include "closure_item.cuh"
#include "fm_volumes.h"

namespace fdlb {

// ------------------------------------------------------------------------------ moments
// Raw quadrature sums (Eq. mom_quad) of the populations of whole cells; written into slice 0
// of the partial-sum array, the other slices are cleared; for FP32 populations also the
// double-float pairs of the sums (sumsw, the closure's input).
template <typename T>
__global__ void moments_kernel(const T* __restrict__ f, double* __restrict__ sums, T* __restrict__ dens,
                               float2* __restrict__ sumsw, const int4* __restrict__ items,
                               const int* __restrict__ n_items, const InstDev* __restrict__ inst,
                               const double* __restrict__ tab, MomSet M) {
    __shared__ double red[kMaxRed][kSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nit = *n_items;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = items[it];
        if (w.w != 0) continue;  // wall items of the closure list
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
                if (M.reduced && k == 1) {
                    // chi = int p_z^2 f: S2_zz and the p_z^2 p_a part of S3_a
                    acc[6] += v;
                    acc[10] += v * p0;
                    acc[11] += v * p1;
                    continue;
                }
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
                const long long base = ((long long)(I.cell_off + c) * M.slices) * kSums;
                double* dst = sums + base;
                dst[threadIdx.x] = s;
                for (int sl = 1; sl < M.slices; ++sl) dst[sl * kSums + threadIdx.x] = 0.0;
                if (sumsw) {  // the double-float pairs of the FP32 closure
                    const float hi = __double2float_rn(s);
                    sumsw[base + threadIdx.x] = make_float2(hi, __double2float_rn(s - (double)hi));
                    for (int sl = 1; sl < M.slices; ++sl) sumsw[base + sl * kSums + threadIdx.x] = make_float2(0.f, 0.f);
                }
                if (threadIdx.x == 0) {
                    T* dd = dens + (long long)(I.cell_off + c) * M.slices;
                    dd[0] = (T)s;
                    for (int sl = 1; sl < M.slices; ++sl) dd[sl] = T(0);
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------------ closure
// The closure kernel: items of own cells (closure_cells in closure_item.cuh) and wall items
// (kind 1 + side, part): the block sums the outgoing flux of one part of the momenta at one
// wall; the stage kernel forms n_w from the parts (diffuse walls, zero net mass flux).
template <typename T>
__global__ void __launch_bounds__(kClosureThreads) closure_kernel(ClosureArgs A, MomSet M) {
    __shared__ T red[kClosureWarps];
    __shared__ __align__(8) uint64_t cbar;  // completion of the band-row copy
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // staged band rows, then the tables in the populations' precision, then the band-union
    // densities of an item
    T* wst = reinterpret_cast<T*>(smem_raw);
    T* tabs = wst + A.wst_elems;
    const ClosureTabs<T> tb = closure_tables<T>(tabs, A.tabT, M, tid, blockDim.x);
    T* nbuf = tabs + closure_tab_elems(M.nR, M.n2, M.n3);
    if (tid == 0) {
        mbar_init(&cbar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();  // everything below reads what the previous kernels wrote
    // the successor (the stage kernel) may start now: it requests the rows of the stage input,
    // written by the kernel this one has just waited for
    pdl_trigger();
    const T* fin_all = reinterpret_cast<const T*>(A.f_in);
    T* rec_all = reinterpret_cast<T*>(A.rec);
    T* nwp = reinterpret_cast<T*>(A.nwp);
    uint32_t phase = 0;
    const int nit = *A.n_items;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = A.items[it];
        const InstDev I = A.inst[w.x];
        if (w.w != 0) {
            // ---- one part of the outgoing flux through a wall
            const int side = w.w - 1, part = w.z, P = A.wall_parts;
            const T* wall = fin_all + I.f_off + (side == 0 ? 0LL : (long long)(I.n_cells - 1) * M.Np);
            T acc = wall_flux_partial<T>(wall, side == 0 ? (long long)M.Np : -(long long)M.Np, M, tb, side, part, P, tid);
            acc = warp_sum(acc);
            if (lane == 0) red[warp] = acc;
            __syncthreads();
            if (tid == 0) nwp[((long long)w.x * 2 + side) * P + part] = wall_part_sum(red);
            __syncthreads();
            continue;
        }
        T* recb = rec_all + (long long)(I.cell_off + w.y) * A.rec_stride;
        if (!closure_cells<T>(A, M, tb, I, w.y, w.z, recb, wst, nbuf, &cbar, phase, NoExtra{}, NoAfterLoads{})) return;
    }
}

// ------------------------------------------------------------------------------ queries
// The FP64 closure record of every cell of the active instances (moments and closure queries,
// not the stage): n, u, T, q, P_12 (Eq. macro_def) from the raw sums in FP64, chi and nbar from
// the closure's side buffer.
template <typename T>
__global__ void ca_kernel(const double* __restrict__ sums, const void* cwv, double* __restrict__ ca, int slices,
                          int total_cells) {
    const T* cw = reinterpret_cast<const T*>(cwv);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < total_cells; c += gridDim.x * blockDim.x) {
        double s[kSums];
        for (int q = 0; q < kSums; ++q) s[q] = 0.0;
        for (int sl = 0; sl < slices; ++sl)
            for (int q = 0; q < kSums; ++q) s[q] += sums[((long long)c * slices + sl) * kSums + q];
        const double n = s[0], in = 1.0 / n;
        const double u0 = s[1] * in, u1 = s[2] * in, u2 = s[3] * in;
        const double tr = s[4] + s[5] + s[6];
        const double uu = u0 * u0 + u1 * u1 + u2 * u2;
        const double Tc = (tr - n * uu) * in * (1.0 / 3.0);
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
        r[9] = (double)cw[2 * (long long)c];
        r[10] = (double)cw[2 * (long long)c + 1];
        r[11] = 0.0;
    }
}

template <typename T>
void launch_ca(const double* sums, const void* cw, double* ca, int slices, int total_cells, cudaStream_t s) {
    const int g = (total_cells + 255) / 256;
    ca_kernel<T><<<g < 2048 ? (g > 0 ? g : 1) : 2048, 256, 0, s>>>(sums, cw, ca, slices, total_cells);
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
void launch_moments(const T* f, double* sums, T* dens, void* sumsw, const int4* items, const int* n_items, int grid,
                    const InstDev* inst, const double* tab, const MomSet& M, cudaStream_t s) {
    moments_kernel<T><<<grid, 256, 0, s>>>(f, sums, dens, reinterpret_cast<float2*>(sumsw), items, n_items, inst, tab, M);
}

// Slice densities from restored raw sums.
template <typename T>
__global__ void dens_kernel(const double* __restrict__ sums, T* __restrict__ dens, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dens[i] = (T)sums[i * kSums];
}

// Double-float pairs (hi = fl(s), lo = fl(s - hi)) of FP64 raw sums: the closure's input for
// FP32 populations, where the stage kernel does not write them (set-up, restored checkpoints).
__global__ void sums_pairs_kernel(const double* __restrict__ sums, float2* __restrict__ sw, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = sums[i];
        const float hi = __double2float_rn(v);
        sw[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

void launch_sums_pairs(const double* sums, void* sw, long long n, cudaStream_t s) {
    const long long g = (n + 255) / 256;
    sums_pairs_kernel<<<(int)(g < 4096 ? (g > 0 ? g : 1) : 4096), 256, 0, s>>>(sums, reinterpret_cast<float2*>(sw), n);
}

template <typename T>
void launch_dens_from_sums(const double* sums, T* dens, long long n, cudaStream_t s) {
    const long long g = (n + 255) / 256;
    dens_kernel<T><<<(int)(g < 4096 ? (g > 0 ? g : 1) : 4096), 256, 0, s>>>(sums, dens, n);
}

template <typename T>
void launch_closure(const ClosureArgs& A, const MomSet& M, int grid, int threads, size_t smem, cudaStream_t s) {
    if (smem > 32 * 1024) cudaFuncSetAttribute(closure_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    launch_maybe_programmatic(closure_kernel<T>, grid, threads, smem, s, A.programmatic, A, M);
}

int closure_blocks_per_sm(int tsize, size_t smem) {
    int n = 0;
    const cudaError_t e = tsize == 4 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, closure_kernel<float>, kClosureThreads, smem)
                                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, closure_kernel<double>, kClosureThreads, smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 8;
    }
    return n > 0 ? n : 1;
}

// ------------------------------------------------------------------------------ FM weights
// The Fischer-Methfessel band of one instance (Eq. fm, App. A), in FP64, stored in the
// populations' precision: a block per cell, the volumes U_i(R_f[j]) of the cell's ball inside the
// faces of its band into shared memory, then W_ij = norm (U_i(R_f[j+1]) - U_i(R_f[j])) over the
// stored extent (zero beyond the domain), the rest of the row zero.  Rc: cell centres (stride
// rc_stride), Rf: the N + 1 faces, blo: (first column, stored extent) per cell.
template <typename T>
__global__ void fm_band_kernel(const double* __restrict__ Rc, int rc_stride, const double* __restrict__ Rf, int N,
                               int sphere, double sigma, int width, const int2* __restrict__ blo, T* __restrict__ W,
                               FmRule rule) {
    extern __shared__ double U[];  // width + 1 values
    const double norm = 3.0 / (4.0 * kFmPi * sigma * sigma * sigma);
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
        const int lo = blo[i].x, cnt = blo[i].y;
        const double d = Rc[(long long)i * rc_stride];
        for (int t = threadIdx.x; t <= cnt; t += blockDim.x) {
            const int j = min(lo + t, N);
            U[t] = fm_volume_inside(sphere, sigma, d, Rf[j], rule);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < width; t += blockDim.x) {
            const double w = (t < cnt && lo + t < N) ? norm * (U[t + 1] - U[t]) : 0.0;
            W[(long long)i * width + t] = (T)w;
        }
        __syncthreads();
    }
}

cudaError_t launch_fm_band(int tsize, const double* Rc, int rc_stride, const double* Rf, int N, int sphere, double sigma,
                           int width, const int2* blo, void* W, const FmRule& rule, int grid, cudaStream_t s) {
    const size_t smem = (size_t)(width + 1) * sizeof(double);
    if (tsize == 4) {
        cudaFuncSetAttribute(fm_band_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fm_band_kernel<float><<<grid, 128, smem, s>>>(Rc, rc_stride, Rf, N, sphere, sigma, width, blo, (float*)W, rule);
    } else {
        cudaFuncSetAttribute(fm_band_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fm_band_kernel<double><<<grid, 128, smem, s>>>(Rc, rc_stride, Rf, N, sphere, sigma, width, blo, (double*)W, rule);
    }
    return cudaPeekAtLastError();
}

size_t closure_smem(int nR, int n2, int n3, int max_union, int wst_elems, int tsize) {
    return closure_smem_bytes(nR, n2, n3, max_union, wst_elems, tsize);
}

void launch_residual(const double* sums, int slices, const InstDev* inst, const double* geo, double* prev, double* out,
                     int n_inst, int save, cudaStream_t s) {
    residual_kernel<<<n_inst < 1024 ? n_inst : 1024, 256, 0, s>>>(sums, slices, inst, geo, prev, out, n_inst, save);
}

// Populations of one precision copied into the other (rounding to nearest for FP64 -> FP32).
template <typename A, typename B>
__global__ void convert_kernel(const A* __restrict__ src, B* __restrict__ dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (B)src[i];
}

void launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, long long n, cudaStream_t s) {
    const long long g = (n + 255) / 256;
    const int grid = (int)(g < 8192 ? (g > 0 ? g : 1) : 8192);
    if (src_fp32 && !dst_fp32)
        convert_kernel<float, double><<<grid, 256, 0, s>>>((const float*)src, (double*)dst, n);
    else if (!src_fp32 && dst_fp32)
        convert_kernel<double, float><<<grid, 256, 0, s>>>((const double*)src, (float*)dst, n);
    else if (src_fp32)
        convert_kernel<float, float><<<grid, 256, 0, s>>>((const float*)src, (float*)dst, n);
    else
        convert_kernel<double, double><<<grid, 256, 0, s>>>((const double*)src, (double*)dst, n);
}

template void launch_ca<float>(const double*, const void*, double*, int, int, cudaStream_t);
template void launch_ca<double>(const double*, const void*, double*, int, int, cudaStream_t);
template void launch_dens_from_sums<float>(const double*, float*, long long, cudaStream_t);
template void launch_dens_from_sums<double>(const double*, double*, long long, cudaStream_t);
template void launch_moments<float>(const float*, double*, float*, void*, const int4*, const int*, int, const InstDev*,
                                    const double*, const MomSet&, cudaStream_t);
template void launch_moments<double>(const double*, double*, double*, void*, const int4*, const int*, int, const InstDev*,
                                     const double*, const MomSet&, cudaStream_t);
template void launch_closure<float>(const ClosureArgs&, const MomSet&, int, int, size_t, cudaStream_t);
template void launch_closure<double>(const ClosureArgs&, const MomSet&, int, int, size_t, cudaStream_t);

}  // namespace fdlb
