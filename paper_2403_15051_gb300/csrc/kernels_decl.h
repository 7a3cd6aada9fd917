// Launch interface between the host solver (fdlb.cu) and the kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fdlb {

constexpr int kCellScalars = 20;   // per-cell collision scalars kept in shared memory

struct StreamSmem {
    int fs, tabs, cell, geo, red, ecoef, misc, total;
};

// Shared-memory plan of the stream kernel (byte offsets), shared with the host.
__host__ __device__ inline StreamSmem stream_smem_plan(int B, int Ms, int nR, int n2, int n3, int nwarps, int tsize) {
    auto al = [](long long x) { return (int)((x + 15) & ~15LL); };
    StreamSmem s;
    int off = 16;  // mbarrier
    s.fs = off;
    off += al((long long)(B + 6) * Ms * tsize);  // rows of cells c0-3 .. c0+B+2
    s.tabs = off;
    off += al((long long)(2 * (nR + n2 + n3) + nR * nR + n2 * n2 + n3 * n3 + 2 * (nR + n2 + n3)) * tsize);
    s.cell = off;
    off += al((long long)B * (kCellScalars + nR + n2 + n3) * tsize);
    s.geo = off;
    off += al((long long)B * 3 * tsize);
    s.red = off;
    off += al((long long)2 * nwarps * kSums * 8);
    s.ecoef = off;
    s.misc = off;
    s.total = off;
    return s;
}


template <typename T>
void launch_moments(const T* f, double* sums, const int4* items, const int* n_items, int grid, const InstDev* inst,
                    const double* tab, const MomSet& M, cudaStream_t s);

template <typename T>
void launch_closure(const ClosureArgs& A, const MomSet& M, int grid, int threads, size_t smem, cudaStream_t s);

size_t closure_smem(int max_cells, int max_union, int tsize);

// Per-cell collision record: kCellScalars scalars then g_R, g_2, g_3; padded to 4 entries.
inline int record_stride(int nR, int n2, int n3) { return (kCellScalars + nR + n2 + n3 + 3) / 4 * 4; }

#define FDLB_STREAM_DECL(T, G)                                                                             \
    cudaError_t launch_stream_##T##_##G(int mpt, const StageArgs& A, const MomSet& M, int grid, int threads, \
                                        size_t smem, cudaStream_t s);
FDLB_STREAM_DECL(float, 0)
FDLB_STREAM_DECL(float, 1)
FDLB_STREAM_DECL(double, 0)
FDLB_STREAM_DECL(double, 1)
#undef FDLB_STREAM_DECL

void launch_residual(const double* sums, int slices, const InstDev* inst, const double* geo, double* prev, double* out,
                     int n_inst, int save, cudaStream_t s);

}  // namespace fdlb
