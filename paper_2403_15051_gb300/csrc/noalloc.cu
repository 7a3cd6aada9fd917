// Per-cell moments of a population array with no device allocation.
//
// Some callers cannot allocate device memory: plugins embedded in an application that owns the
// whole device-memory budget and forbids allocations of its own, and latency-critical loops in
// which cudaMalloc's implicit device synchronisation is not acceptable.  For them this entry
// point reduces populations they already hold to per-cell moments using only the caller's
// input and output buffers plus a fixed scratch array that lives in this library's module
// (allocated when the library is loaded, held by every GPU that loads it until exit).
//
// It is the moment-reduction kernel of the solver (13 raw quadrature sums per cell, Eq. mom_quad,
// then n, u, T, q and the shear stress, Eq. macro_def) with its partial-sum buffer moved into
// that scratch array.
#include <cuda_runtime.h>

#include <mutex>

#include "device_common.cuh"
#include "internal.h"
#include "kernels.cuh"

namespace fdlb {
namespace {

constexpr int kNoAllocMaxCells = 32768;         // largest n_cells per call (3.4 MB of scratch)
constexpr int kNoAllocNodes = 2 * kMaxQ + 2 * kMaxQ;  // radial (2Q) + two full-range axes (Q each)

// Scratch shared by every call on a device: the raw sums of each cell, then the momentum nodes.
__device__ __align__(256) double g_noalloc_scratch[(size_t)kNoAllocMaxCells * kSums + kNoAllocNodes];

// Device address of the scratch array, looked up once per device on the first call; the lookup is
// serialised across host threads.
void* g_scratch_addr[256] = {};
std::mutex g_scratch_mutex;

// Raw sums of every cell: a block per cell (grid-stride), per-thread partials and warp tree in
// the populations' precision, FP64 across warps.  Every call overwrites the sums of its cells.
template <typename T>
__global__ void noalloc_sums_kernel(const T* __restrict__ f, int n_cells, int nR, int n2, int n3,
                                    double* __restrict__ scratch) {
    __shared__ double red[kMaxRed][kSums];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int Np = nR * n2 * n3;
    const double* nodes = scratch + (size_t)kNoAllocMaxCells * kSums;
    for (int c = blockIdx.x; c < n_cells; c += gridDim.x) {
        const T* fc = f + (long long)c * Np;
        T acc[kSums];
#pragma unroll
        for (int q = 0; q < kSums; ++q) acc[q] = T(0);
        for (int m = threadIdx.x; m < Np; m += blockDim.x) {
            // library layout inside a cell: [k][i][j]
            const int k = m / (nR * n2), rem = m % (nR * n2), i = rem / n2, j = rem % n2;
            const T p0 = (T)nodes[i], p1 = (T)nodes[nR + j], p2 = (T)nodes[nR + n2 + k];
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
#pragma unroll
        for (int q = 0; q < kSums; ++q) {
            const T s = warp_sum(acc[q]);
            if (lane == 0) red[warp][q] = (double)s;
        }
        __syncthreads();
        if (threadIdx.x < kSums) {
            double s = 0.0;
            for (int ww = 0; ww < nw; ++ww) s += red[ww][threadIdx.x];
            scratch[(size_t)c * kSums + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// n, u_1..3, T, q_1..3, P_12 of every cell from its raw sums.
__global__ void noalloc_moments_kernel(const double* __restrict__ scratch, int n_cells, double* __restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n_cells; c += gridDim.x * blockDim.x) {
        const double* s = scratch + (size_t)c * kSums;
        const double n = s[0];
        const double u0 = s[1] / n, u1 = s[2] / n, u2 = s[3] / n;
        const double tr = s[4] + s[5] + s[6];
        const double uu = u0 * u0 + u1 * u1 + u2 * u2;
        const double m0 = s[4] * u0 + s[7] * u1 + s[8] * u2;
        const double m1 = s[7] * u0 + s[5] * u1 + s[9] * u2;
        const double m2 = s[8] * u0 + s[9] * u1 + s[6] * u2;
        double* o = out + (size_t)c * FDLB_NMOM;
        o[0] = n;
        o[1] = u0;
        o[2] = u1;
        o[3] = u2;
        o[4] = (tr - n * uu) / (3.0 * n);
        o[5] = 0.5 * (s[10] - 2.0 * m0 - u0 * tr + 2.0 * n * uu * u0);
        o[6] = 0.5 * (s[11] - 2.0 * m1 - u1 * tr + 2.0 * n * uu * u1);
        o[7] = 0.5 * (s[12] - 2.0 * m2 - u2 * tr + 2.0 * n * uu * u2);
        o[8] = s[7] - n * u0 * u1;
    }
}

}  // namespace
}  // namespace fdlb

extern "C" int fdlb_moments_noalloc(int precision, int Q_R, int Q_2, int Q_3, const double* nodes_host, int n_cells,
                                    const void* f_dev, double* moments_dev, void* cuda_stream) {
    using namespace fdlb;
    if (precision != FDLB_FP32 && precision != FDLB_FP64) return FDLB_EINVAL;
    if (Q_R < 1 || Q_R > kMaxQ || Q_2 < 1 || Q_2 > kMaxQ || Q_3 < 1 || Q_3 > kMaxQ) return FDLB_EINVAL;
    if (n_cells < 1 || n_cells > kNoAllocMaxCells || !nodes_host || !f_dev || !moments_dev) return FDLB_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return FDLB_ENOGPU;
    void* sp = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            // one-time set-up on this device: the device address of the scratch array
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return FDLB_ECUDA;
            g_scratch_addr[dev] = p;
        }
        sp = g_scratch_addr[dev];
    }
    double* scratch = static_cast<double*>(sp);
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the momentum nodes go to the tail of the scratch array, in stream order
    const int n_nodes = 2 * Q_R + Q_2 + Q_3;
    if (cudaMemcpyAsync(scratch + (size_t)kNoAllocMaxCells * kSums, nodes_host, n_nodes * sizeof(double),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FDLB_ECUDA;
    // launches through cudaLaunchKernel return this call's own launch error, so an error left by
    // earlier work on the thread is neither reported here nor cleared
    int nR = 2 * Q_R, n2 = Q_2, n3 = Q_3, nc = n_cells;
    const int grid = n_cells < 4096 ? n_cells : 4096;
    cudaError_t e;
    if (precision == FDLB_FP32) {
        const float* fp = static_cast<const float*>(f_dev);
        void* args[] = {&fp, &nc, &nR, &n2, &n3, &scratch};
        e = cudaLaunchKernel((const void*)noalloc_sums_kernel<float>, dim3(grid), dim3(256), args, 0, s);
    } else {
        const double* fp = static_cast<const double*>(f_dev);
        void* args[] = {&fp, &nc, &nR, &n2, &n3, &scratch};
        e = cudaLaunchKernel((const void*)noalloc_sums_kernel<double>, dim3(grid), dim3(256), args, 0, s);
    }
    if (e != cudaSuccess) return FDLB_ECUDA;
    const double* sc = scratch;
    void* margs[] = {&sc, &nc, &moments_dev};
    e = cudaLaunchKernel((const void*)noalloc_moments_kernel, dim3((n_cells + 255) / 256), dim3(256), margs, 0, s);
    return e == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
}
