// Launch interface between the host solver (fdlb.cu) and the kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "fm_volumes.h"

namespace fdlb {

constexpr int kCellScalars = 20;   // per-cell collision scalars kept in shared memory

// Per-cell collision record (populations' precision): kCellScalars scalars, then g_2, g_R, g_3
// (g_2 first so that a vector of consecutive j starts on a vector boundary); padded to 4 entries.
inline __host__ __device__ int record_stride(int nR, int n2, int n3) { return (kCellScalars + nR + n2 + n3 + 3) / 4 * 4; }
inline __host__ __device__ int rec_off_g2() { return kCellScalars; }
inline __host__ __device__ int rec_off_gR(int n2) { return kCellScalars + n2; }
inline __host__ __device__ int rec_off_g3(int nR, int n2) { return kCellScalars + n2 + nR; }

// Launch with programmatic stream serialization when `programmatic` (see pdl_wait), else the
// ordinary way.
template <typename... Args>
inline cudaError_t launch_maybe_programmatic(void (*kern)(Args...), int grid, int threads, size_t smem, cudaStream_t s,
                                             int programmatic, Args... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = programmatic ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Row stride of K^h in the stage kernel's shared memory: a multiple of four elements (16-byte
// vector loads of a row) whose rows fall on distinct banks for the rows a quarter warp reads.
inline __host__ __device__ int kr_stride(int nR) { return (nR + 3) / 4 * 4 + 4; }
// Elements of the p_2 nodes at the start of the tables, padded to 16 bytes (four elements).
inline __host__ __device__ int p2_span(int n2) { return (n2 + 3) / 4 * 4; }
// Elements from K_2 to K^h: K_2, padded to 16 bytes.
inline __host__ __device__ int kr_offset(int n2, int tsize) { return (n2 * n2 * tsize + 15) / 16 * 16 / tsize; }

struct StreamSmem {
    int fs, rec, tabs, geo, red, kr, total;
};

// Shared-memory plan of the stream kernel (byte offsets), shared with the host: the staged rows
// of cells c0-3 .. c0+B+2, the tile's collision records, the tables (the p_2 nodes, K_2
// transposed, then K^h with row stride kr_stride(nR), K_3 with row stride n3+1, the other nodes
// and the weights, the wall Maxwellians), the cell geometry and the per-warp partial sums.
__host__ __device__ inline StreamSmem stream_smem_plan(int B, int Ms, int nR, int n2, int n3, int nwarps, int tsize,
                                                       int mma = 0, int krg = 0) {
    auto al = [](long long x) { return (int)((x + 15) & ~15LL); };
    StreamSmem s;
    int off = 16;  // mbarrier
    s.fs = off;
    off += al((long long)(B + 6) * Ms * tsize);
    s.rec = off;
    off += al((long long)B * record_stride(nR, n2, n3) * tsize);
    s.tabs = off;
    // (no K^h table when K^h f comes from the contraction kernel: krg)
    off += al((long long)(p2_span(n2) + 2 * (nR + n3) + n2 + (krg ? 0 : nR) * kr_stride(nR) + kr_offset(n2, tsize) +
                          n3 * (n3 + 1) + 2 * (nR + n2 + n3)) * tsize);
    s.geo = off;
    off += al((long long)B * 3 * tsize);
    s.red = off;
    off += al((long long)B * nwarps * 16 * tsize);
    s.kr = off;  // K^h f of the tile's own cells (tensor-core path)
    if (mma) off += al((long long)B * Ms * tsize);
    s.total = off;
    return s;
}

// Launch shape of the stream kernel: VW consecutive j momenta per vector, at most NV vectors
// per thread, and whether the compile-time shape (cylinder 16 x 8 x 8, sphere 24 x 12 x 12)
// is used.
struct StreamCfg {
    int vw, nv, spec;
    int minb = 1;  // register bound of the stage kernel: 1 or 3 blocks per SM (cylinder FP32 shape)
};

// Raw sums (FP64, slice 0), double-float pairs (FP32 populations) and densities of every cell of a
// state of total_cells cells.
template <typename T>
void launch_moments(const T* f, double* sums, T* dens, void* sumsw, long long total_cells, int grid, const double* tab,
                    const MomSet& M, cudaStream_t s);

template <typename T>
// The FP64 closure record of every cell (kCA columns); with `packed`, also the moments query's rows
// (the first kNmom columns) contiguous, [cell][kNmom].
void launch_ca(const double* sums, const void* cw, double* ca, int slices, int total_cells, cudaStream_t s,
               double* packed = nullptr);

void launch_sums_pairs(const double* sums, void* sw, long long n, cudaStream_t s);

template <typename T>
void launch_dens_from_sums(const double* sums, T* dens, long long n, cudaStream_t s);

template <typename T>
void launch_closure(const ClosureArgs& A, const MomSet& M, int grid, int threads, size_t smem, cudaStream_t s);

size_t closure_smem(int nR, int n2, int n3, int max_union, int wst_elems, int tsize);
// Blocks of the closure kernel that fit on an SM with `smem` bytes of dynamic shared memory each.
int closure_blocks_per_sm(int tsize, size_t smem);
// The batch form of the closure (closure_band_kernel, then closure_records_kernel; items of at
// most kClosureCells cells), and the blocks of either that reside on one SM.
template <typename T>
void launch_closure_batch(const ClosureArgs& A, const MomSet& M, int grid, size_t smem, cudaStream_t s);
int closure_batch_blocks_per_sm(int tsize, size_t smem);


#define FDLB_STREAM_DECL(T, G)                                                                             \
    cudaError_t launch_stream_##T##_##G(const StreamCfg& cfg, const StageArgs& A, const MomSet& M, int grid, \
                                        int threads, size_t smem, cudaStream_t s);
FDLB_STREAM_DECL(float, 0)
FDLB_STREAM_DECL(float, 1)
FDLB_STREAM_DECL(double, 0)
FDLB_STREAM_DECL(double, 1)
#undef FDLB_STREAM_DECL

#define FDLB_STEP_DECL(T, G)                                                                                   \
    cudaError_t launch_step_##T##_##G(const StreamCfg& cfg, const StepArgs* S, const MomSet& M, int grid,     \
                                      int threads, size_t smem, cudaStream_t s, int* blocks_per_sm);
FDLB_STEP_DECL(float, 0)
FDLB_STEP_DECL(float, 1)
FDLB_STEP_DECL(double, 0)
FDLB_STEP_DECL(double, 1)
#undef FDLB_STEP_DECL

// K^h f of the populations of the stage items' cells (Sec. III.B half-range derivative matrix
// applied along the radial momentum axis), written in the layout of f: the CUDA-core kernel
// (any precision) or, for FP32 populations where available, the tensor-core kernel.
template <typename T>
cudaError_t launch_kr_contract(const T* f, T* out, const int4* items, const int* n_items, const InstDev* inst,
                               const T* KR, const T* isw, const T* sw, const MomSet& M, int grid, cudaStream_t s);

// The tensor-core form (FP32): Bsplit holds the weight-scaled K^h (kr_contract.cu) as TF32 pairs in
// the kernel's shared-memory layout (kr_split_table), isw / sw the scales, Npad = 2Q_R rounded up to
// 16; err is set when a bounded wait runs out.
// Sphere: out = K_3 f along the third momentum axis, per cell (each cell once: the items of slice 0
// of the stream work list), in the order the stage kernel contracts it (the same values).
template <typename T>
cudaError_t launch_k3_contract(const T* f, T* out, const int4* items, const int* n_items, const InstDev* inst,
                               const T* K3, const MomSet& M, int grid, cudaStream_t s);
cudaError_t launch_kr_contract_tc(const float* f, float* out, const int4* items, const int* n_items, const InstDev* inst,
                                  const float* Bsplit, const float* isw, const float* sw, const MomSet& M, int Npad,
                                  int* err, int grid, cudaStream_t s);
size_t kr_tc_smem_bytes(int Npad);

// The Fischer-Methfessel weights of one instance's band, computed on the device in FP64 (the host
// set-up's arithmetic, fm_volumes.h) and stored in the populations' precision (tsize 4 or 8).
cudaError_t launch_fm_band(int tsize, const double* Rc, int rc_stride, const double* Rf, int N, int sphere, double sigma,
                           int width, const int2* blo, void* W, const FmRule& rule, int grid, cudaStream_t s);

// dst = src x scale, the product formed in FP64 and rounded once to the destination's precision.
void launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, long long n, cudaStream_t s,
                    double scale = 1.0);

void launch_residual(const double* sums, int slices, const InstDev* inst, const double* geo, double* prev, double* out,
                     int n_inst, int save, cudaStream_t s);

}  // namespace fdlb
