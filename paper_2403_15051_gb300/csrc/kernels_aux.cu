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
            double acc[kSums];
#pragma unroll
            for (int q = 0; q < kSums; ++q) acc[q] = 0.0;
            for (int m = threadIdx.x; m < M.Np; m += blockDim.x) {
                const int k = m / (M.nR * M.n2), rem = m % (M.nR * M.n2), i = rem / M.n2, j = rem % M.n2;
                const double p0 = tab[M.o_pR + i], p1 = tab[M.o_p2 + j], p2 = tab[M.o_p3 + k];
                const double v = (double)fc[m], ps = p0 * p0 + p1 * p1 + p2 * p2;
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
#pragma unroll
            for (int q = 0; q < kSums; ++q) {
                double s = warp_sum(acc[q]);
                if (lane == 0) red[warp][q] = s;
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
// Per cell: n, u, T, q from the raw sums (Eq. macro_def); nbar over the stored FM band
// (Eq. fm, n = 0 outside the domain); chi = chi_SET(pi sigma^3 nbar / 6) (Eqs. chi, chi_ret).
template <typename T>
__global__ void closure_kernel(ClosureArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* nbuf = reinterpret_cast<T*>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nit = *A.n_items;
    const T* band = reinterpret_cast<const T*>(A.band);
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = A.items[it];
        const InstDev I = A.inst[w.x];
        const int c0 = w.y, cnt = w.z, N = I.n_cells;
        const double* S = A.sums + (long long)I.cell_off * A.slices * kSums;
        double* ca = A.ca + (long long)I.cell_off * kCA;
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
            const int c = c0 + t;
            double s[kSums];
#pragma unroll
            for (int q = 0; q < kSums; ++q) s[q] = 0.0;
            for (int sl = 0; sl < A.slices; ++sl)
#pragma unroll
                for (int q = 0; q < kSums; ++q) s[q] += S[((long long)c * A.slices + sl) * kSums + q];
            const double n = s[0];
            const double u0 = s[1] / n, u1 = s[2] / n, u2 = s[3] / n;
            const double tr = s[4] + s[5] + s[6];
            const double uu = u0 * u0 + u1 * u1 + u2 * u2;
            const double Tc = (tr - n * uu) / (3.0 * n);
            // M2 u (rows of the symmetric second-moment matrix)
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
            if (I.chi_local) {
                r[9] = chi_cs(I.etafac * n);
                r[10] = n;
            }
            r[11] = 0.0;
        }
        if (!I.chi_local) {
            const int jlo = A.band_lo[I.cell_off + c0];
            const int jhi = min(N - 1, A.band_lo[I.cell_off + c0 + cnt - 1] + I.band_w - 1);
            const int nu = jhi - jlo + 1;
            for (int j = threadIdx.x; j < nu && j < A.max_union; j += blockDim.x) {
                double nj = 0.0;
                for (int sl = 0; sl < A.slices; ++sl) nj += S[((long long)(jlo + j) * A.slices + sl) * kSums];
                nbuf[j] = (T)nj;
            }
            __syncthreads();
            for (int t = warp; t < cnt; t += nwarps) {
                const int c = c0 + t;
                const int lo = A.band_lo[I.cell_off + c];
                const T* Wr = band + I.band_off + (long long)c * I.band_w;
                T acc = T(0);
                for (int k = lane; k < I.band_w; k += 32) {
                    const int j = lo + k;
                    if (j <= jhi) acc += Wr[k] * nbuf[j - jlo];
                }
                acc = warp_sum(acc);
                if (lane == 0) {
                    const double nbar = (double)acc;
                    ca[(long long)c * kCA + 9] = chi_cs(I.etafac * nbar);
                    ca[(long long)c * kCA + 10] = nbar;
                }
            }
            __syncthreads();
        }
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
void launch_closure(const ClosureArgs& A, int grid, int threads, size_t smem, cudaStream_t s) {
    closure_kernel<T><<<grid, threads, smem, s>>>(A);
}

void launch_residual(const double* sums, int slices, const InstDev* inst, const double* geo, double* prev, double* out,
                     int n_inst, int save, cudaStream_t s) {
    residual_kernel<<<n_inst < 1024 ? n_inst : 1024, 256, 0, s>>>(sums, slices, inst, geo, prev, out, n_inst, save);
}

template void launch_moments<float>(const float*, double*, const int4*, const int*, int, const InstDev*,
                                    const double*, const MomSet&, cudaStream_t);
template void launch_moments<double>(const double*, double*, const int4*, const int*, int, const InstDev*,
                                     const double*, const MomSet&, cudaStream_t);
template void launch_closure<float>(const ClosureArgs&, int, int, size_t, cudaStream_t);
template void launch_closure<double>(const ClosureArgs&, int, int, size_t, cudaStream_t);

}  // namespace fdlb
