// Learned warm start: a one-dimensional Fourier neural operator trained on the solver's own
// steady states (the paper has no network; this is the library's warm-start service).
//
// Network (sizes chosen at creation): 5 instance parameters -> 6 input channels on P points of the
// normalised radius (5 normalised parameters + x) -> lift to width W -> L Fourier layers
// v <- GELU(v W_l + b_l + G R_l F v) (F: the 2m real DFT rows of the m lowest modes, R_l per-mode
// complex W x W mixing, G the truncated inverse) -> GELU(v P1 + c1) (hidden H) -> P2 + c2 ->
// 4 output channels (normalised n, u_2, T, q_R profiles).
//
// Precision: FP32 master weights (Adam), BF16 copies of every weight matrix used as GEMM
// operands, FP32 activations and FP32 accumulation in every product.  The products with a BF16
// weight operand run on the tensor cores (mma.sync BF16, the activations as two BF16 parts); the
// products of two FP32 operands (the DFT pair, the weight gradients) on the FP32 pipe.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <utility>
#include <vector>

#include "internal.h"

namespace fdlb {
namespace {

constexpr int kCin = 6, kCout = 4;

// --------------------------------------------------------------------------- kernels
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

// C[z] = alpha op(A[z]) op(B[z]) + beta C[z], row-major, batch z = blockIdx.z.  64 x 64 tiles,
// 256 threads, 4 x 4 outputs per thread, K in slices of 16 staged in shared memory, FP32 FMA.
template <typename TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda, int tA,
                                                   long long sA, const TB* __restrict__ Bm, int ldb, int tB,
                                                   long long sB, float* __restrict__ C, int ldc, long long sC,
                                                   float alpha, float beta) {
    __shared__ float As[16][64 + 4];
    __shared__ float Bs[16][64 + 4];
    const int z = blockIdx.z;
    A += z * sA;
    Bm += z * sB;
    C += z * sC;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e >> 6, mm = e & 63;
            const int gm = m0 + mm, gk = k0 + kk;
            float va = 0.f;
            if (gm < M && gk < K) va = tA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[kk][mm] = va;
            const int gn = n0 + mm;
            float vb = 0.f;
            if (gn < N && gk < K) vb = to_f(tB ? Bm[(long long)gn * ldb + gk] : Bm[(long long)gk * ldb + gn]);
            Bs[kk][mm] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < M && gn < N) {
                float* c = C + (long long)gm * ldc + gn;
                *c = alpha * acc[i][j] + (beta != 0.f ? beta * *c : 0.f);
            }
        }
}

// The products with a BF16 weight operand on the tensor cores: C[z] = alpha A[z] op(B[z]) + beta C[z]
// with mma.sync m16n8k16 (BF16 operands, FP32 accumulation).  The FP32 activations A are split into
// two BF16 parts, a = a_hi + a_lo (a_hi = bf16(a), a_lo = bf16(a - a_hi)), and both parts multiply the
// (exactly BF16) weights: the product keeps ~2^-17 of a's relative accuracy, as the FP32 FMA form does
// to within that.  64 x 64 output tiles, 128 threads (four warps of 32 x 32: 2 x 4 MMA tiles of
// 16 x 8), K in slices of 16 staged in shared memory as [row][k] BF16.
// Fragment ownership of m16n8k16 (g = lane / 4, t = lane % 4; pairs of BF16 per 32-bit register, the
// lower index in the low half): A a0 (g, 2t..2t+1), a1 (g+8, 2t..), a2 (g, 2t+8..), a3 (g+8, 2t+8..);
// B b0 (k 2t..2t+1, n g), b1 (k 2t+8..2t+9, n g); D d0 (g, 2t), d1 (g, 2t+1), d2 (g+8, 2t), d3 (g+8, 2t+1).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(int M, int N, int K, const float* __restrict__ A, int lda, int tA,
                                                        long long sA, const __nv_bfloat16* __restrict__ Bm, int ldb, int tB,
                                                        long long sB, float* __restrict__ C, int ldc, long long sC,
                                                        float alpha, float beta) {
    constexpr int KP = 16 + 8;  // padded row: 48 bytes, pairs stay 4-byte aligned
    __shared__ __align__(16) __nv_bfloat16 Ah[64][KP], Al[64][KP], Bs[64][KP];
    const int z = blockIdx.z;
    A += z * sA;
    Bm += z * sB;
    C += z * sC;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 128) {
            const int r = e >> 4, kk = e & 15, gk = k0 + kk;
            const int gm = m0 + r;
            float va = 0.f;
            if (gm < M && gk < K) va = tA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            const __nv_bfloat16 hi = __float2bfloat16_rn(va);
            Ah[r][kk] = hi;
            Al[r][kk] = __float2bfloat16_rn(va - __bfloat162float(hi));
            const int gn = n0 + r;
            __nv_bfloat16 vb = __float2bfloat16_rn(0.f);
            if (gn < N && gk < K) vb = tB ? Bm[(long long)gn * ldb + gk] : Bm[(long long)gk * ldb + gn];
            Bs[r][kk] = vb;
        }
        __syncthreads();
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r = wm + mt * 16 + g;
            ah[mt][0] = *reinterpret_cast<const uint32_t*>(&Ah[r][2 * t]);
            ah[mt][1] = *reinterpret_cast<const uint32_t*>(&Ah[r + 8][2 * t]);
            ah[mt][2] = *reinterpret_cast<const uint32_t*>(&Ah[r][2 * t + 8]);
            ah[mt][3] = *reinterpret_cast<const uint32_t*>(&Ah[r + 8][2 * t + 8]);
            al[mt][0] = *reinterpret_cast<const uint32_t*>(&Al[r][2 * t]);
            al[mt][1] = *reinterpret_cast<const uint32_t*>(&Al[r + 8][2 * t]);
            al[mt][2] = *reinterpret_cast<const uint32_t*>(&Al[r][2 * t + 8]);
            al[mt][3] = *reinterpret_cast<const uint32_t*>(&Al[r + 8][2 * t + 8]);
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = wn + nt * 8 + g;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * t]);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Bs[c][2 * t + 8]);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma_bf16(acc[mt][nt], al[mt], b0, b1);
                mma_bf16(acc[mt][nt], ah[mt], b0, b1);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gm = m0 + wm + mt * 16 + g + ((q & 2) ? 8 : 0), gn = n0 + wn + nt * 8 + 2 * t + (q & 1);
                if (gm < M && gn < N) {
                    float* c = C + (long long)gm * ldc + gn;
                    *c = alpha * acc[mt][nt][q] + (beta != 0.f ? beta * *c : 0.f);
                }
            }
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143267794f;
}

// u <- u + bias (per column); v = GELU(u) when v != nullptr.
__global__ void bias_act_kernel(float* __restrict__ u, const float* __restrict__ bias, float* __restrict__ v,
                                long long rows, int cols) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < rows * cols;
         e += (long long)gridDim.x * blockDim.x) {
        const float x = u[e] + bias[e % cols];
        u[e] = x;
        if (v) v[e] = gelu_f(x);
    }
}

// d <- d * GELU'(u)
__global__ void gelu_back_kernel(float* __restrict__ d, const float* __restrict__ u, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        d[e] *= gelu_grad_f(u[e]);
}

// column sums of a [rows][cols] array into out[cols] (one block per column, fixed order)
__global__ void colsum_kernel(const float* __restrict__ x, long long rows, int cols, float* __restrict__ out) {
    __shared__ float red[32];
    const int c = blockIdx.x;
    float s = 0.f;
    for (long long r = threadIdx.x; r < rows; r += blockDim.x) s += x[r * cols + c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[c] = t;
    }
}

// Input channels: the five parameters, normalised, broadcast over x, then x / (P - 1).
// Normalisation: (log10 Kn + 1), (eta0 - 0.155)/0.145, (ratio - 3.1)/1.9, (u_w - 0.15)/0.15,
// (T_ratio - 1.15)/0.15 (the ranges of the parameter sweep mapped to about [-1, 1]).
__global__ void features_kernel(const float* __restrict__ raw, int B, int P, float* __restrict__ a) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * P; e += gridDim.x * blockDim.x) {
        const int b = e / P, x = e % P;
        const float* r = raw + b * 5;
        float* o = a + (long long)e * kCin;
        o[0] = log10f(r[0]) + 1.f;
        o[1] = (r[1] - 0.155f) / 0.145f;
        o[2] = (r[2] - 3.1f) / 1.9f;
        o[3] = (r[3] - 0.15f) / 0.15f;
        o[4] = (r[4] - 1.15f) / 0.15f;
        o[5] = (float)x / (float)(P - 1);
    }
}

// MSE loss and its gradient: loss = mean (out - t)^2, dout = 2 (out - t) / count.  One block,
// fixed-order reduction.
__global__ void mse_kernel(const float* __restrict__ out, const float* __restrict__ t, long long n,
                           float* __restrict__ dout, float* __restrict__ loss) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const float d = out[e] - t[e];
        dout[e] = 2.f * d / (float)n;
        s += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        *loss = (float)(tot / (double)n);
    }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the FP32 master weights, then the BF16 copy.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, __nv_bfloat16* __restrict__ wb, long long n, float lr, float c1,
                            float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float a = 0.9f * m1[e] + 0.1f * gg;
        const float b = 0.999f * m2[e] + 0.001f * gg * gg;
        m1[e] = a;
        m2[e] = b;
        const float x = w[e] - lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
        w[e] = x;
        wb[e] = __float2bfloat16_rn(x);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        wb[e] = __float2bfloat16_rn(w[e]);
}

}  // namespace

// --------------------------------------------------------------------------- network object
struct NNet {
    int W, m, L, H, P, Bmax;
    long long n_params = 0;
    // parameter offsets (same order as the FP64 reference layout)
    long long o_lw, o_lb, o_p1w, o_p1b, o_p2w, o_p2b;
    std::vector<long long> o_rre, o_rim, o_w, o_b;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    unsigned char* ws = nullptr;
    float *w = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16* wb = nullptr;
    float *F = nullptr, *G = nullptr;
    float *raw = nullptr, *a = nullptr, *vs = nullptr, *us = nullptr, *vh = nullptr, *yh = nullptr, *s = nullptr;
    float *z1 = nullptr, *h = nullptr, *out = nullptr, *tgt = nullptr, *dout = nullptr, *dh = nullptr;
    float *dv = nullptr, *dv2 = nullptr, *du = nullptr, *dyh = nullptr, *dvh = nullptr, *loss = nullptr;
    int step = 0;
};

namespace {

template <typename TB>
cudaError_t gemm(NNet& n, int M, int N, int K, const float* A, int lda, int tA, long long sA, const TB* B, int ldb,
                 int tB, long long sB, float* C, int ldc, long long sC, int batch, float alpha, float beta) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
    if constexpr (std::is_same<TB, __nv_bfloat16>::value)
        gemm_bf16_kernel<<<grid, 128, 0, n.stream>>>(M, N, K, A, lda, tA, sA, B, ldb, tB, sB, C, ldc, sC, alpha, beta);
    else
        gemm_kernel<TB><<<grid, 256, 0, n.stream>>>(M, N, K, A, lda, tA, sA, B, ldb, tB, sB, C, ldc, sC, alpha, beta);
    return cudaGetLastError();
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

// Forward pass for B samples whose raw parameters are in n.raw; leaves every activation the
// backward pass needs.
int forward(NNet& n, int B) {
    const int W = n.W, m = n.m, P = n.P, H = n.H;
    const long long rows = (long long)B * P;
    features_kernel<<<grid_for(rows), 256, 0, n.stream>>>(n.raw, B, P, n.a);
    float* v0 = n.vs;
    gemm(n, (int)rows, W, kCin, n.a, kCin, 0, 0, n.wb + n.o_lw, W, 0, 0, v0, W, 0, 1, 1.f, 0.f);
    bias_act_kernel<<<grid_for(rows * W), 256, 0, n.stream>>>(v0, n.w + n.o_lb, nullptr, rows, W);
    for (int l = 0; l < n.L; ++l) {
        float* v = n.vs + (long long)l * rows * W;
        float* vn = n.vs + (long long)(l + 1) * rows * W;
        float* u = n.us + (long long)l * rows * W;
        float* vh = n.vh + (long long)l * B * 2 * m * W;
        // spectral path: vh[b] = F v[b]; per mode k: yre = re Rre - im Rim, yim = re Rim + im Rre;
        // s[b] = G yh[b]
        gemm(n, 2 * m, W, P, n.F, P, 0, 0, v, W, 0, (long long)P * W, vh, W, (long long)2 * m * W, B, 1.f, 0.f);
        const __nv_bfloat16* rre = n.wb + n.o_rre[l];
        const __nv_bfloat16* rim = n.wb + n.o_rim[l];
        const int ld = 2 * m * W;
        gemm(n, B, W, W, vh, ld, 0, W, rre, W, 0, (long long)W * W, n.yh, ld, W, m, 1.f, 0.f);
        gemm(n, B, W, W, vh + m * W, ld, 0, W, rim, W, 0, (long long)W * W, n.yh, ld, W, m, -1.f, 1.f);
        gemm(n, B, W, W, vh, ld, 0, W, rim, W, 0, (long long)W * W, n.yh + m * W, ld, W, m, 1.f, 0.f);
        gemm(n, B, W, W, vh + m * W, ld, 0, W, rre, W, 0, (long long)W * W, n.yh + m * W, ld, W, m, 1.f, 1.f);
        gemm(n, P, W, 2 * m, n.G, 2 * m, 0, 0, n.yh, W, 0, (long long)2 * m * W, u, W, (long long)P * W, B, 1.f, 0.f);
        // pointwise path and activation: u = s + v W_l + b_l, v' = GELU(u)
        gemm(n, (int)rows, W, W, v, W, 0, 0, n.wb + n.o_w[l], W, 0, 0, u, W, 0, 1, 1.f, 1.f);
        bias_act_kernel<<<grid_for(rows * W), 256, 0, n.stream>>>(u, n.w + n.o_b[l], vn, rows, W);
    }
    const float* vL = n.vs + (long long)n.L * rows * W;
    gemm(n, (int)rows, H, W, vL, W, 0, 0, n.wb + n.o_p1w, H, 0, 0, n.z1, H, 0, 1, 1.f, 0.f);
    bias_act_kernel<<<grid_for(rows * H), 256, 0, n.stream>>>(n.z1, n.w + n.o_p1b, n.h, rows, H);
    gemm(n, (int)rows, kCout, H, n.h, H, 0, 0, n.wb + n.o_p2w, kCout, 0, 0, n.out, kCout, 0, 1, 1.f, 0.f);
    bias_act_kernel<<<grid_for(rows * kCout), 256, 0, n.stream>>>(n.out, n.w + n.o_p2b, nullptr, rows, kCout);
    return cudaGetLastError() == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
}

// Backward pass from n.dout into n.g (reverse order of `forward`).
int backward(NNet& n, int B) {
    const int W = n.W, m = n.m, P = n.P, H = n.H;
    const long long rows = (long long)B * P;
    float* g = n.g;
    gemm(n, H, kCout, (int)rows, n.h, H, 1, 0, n.dout, kCout, 0, 0, g + n.o_p2w, kCout, 0, 1, 1.f, 0.f);
    colsum_kernel<<<kCout, 256, 0, n.stream>>>(n.dout, rows, kCout, g + n.o_p2b);
    gemm(n, (int)rows, H, kCout, n.dout, kCout, 0, 0, n.wb + n.o_p2w, kCout, 1, 0, n.dh, H, 0, 1, 1.f, 0.f);
    gelu_back_kernel<<<grid_for(rows * H), 256, 0, n.stream>>>(n.dh, n.z1, rows * H);
    const float* vL = n.vs + (long long)n.L * rows * W;
    gemm(n, W, H, (int)rows, vL, W, 1, 0, n.dh, H, 0, 0, g + n.o_p1w, H, 0, 1, 1.f, 0.f);
    colsum_kernel<<<H, 256, 0, n.stream>>>(n.dh, rows, H, g + n.o_p1b);
    gemm(n, (int)rows, W, H, n.dh, H, 0, 0, n.wb + n.o_p1w, H, 1, 0, n.dv, W, 0, 1, 1.f, 0.f);
    const int ld = 2 * m * W;
    for (int l = n.L - 1; l >= 0; --l) {
        const float* v = n.vs + (long long)l * rows * W;
        const float* u = n.us + (long long)l * rows * W;
        const float* vh = n.vh + (long long)l * B * 2 * m * W;
        const __nv_bfloat16* rre = n.wb + n.o_rre[l];
        const __nv_bfloat16* rim = n.wb + n.o_rim[l];
        // du = dv GELU'(u) (in place in dv)
        gelu_back_kernel<<<grid_for(rows * W), 256, 0, n.stream>>>(n.dv, u, rows * W);
        float* du = n.dv;
        gemm(n, W, W, (int)rows, v, W, 1, 0, du, W, 0, 0, g + n.o_w[l], W, 0, 1, 1.f, 0.f);
        colsum_kernel<<<W, 256, 0, n.stream>>>(du, rows, W, g + n.o_b[l]);
        gemm(n, (int)rows, W, W, du, W, 0, 0, n.wb + n.o_w[l], W, 1, 0, n.dv2, W, 0, 1, 1.f, 0.f);
        // spectral path: dyh[b] = G^T du[b]
        gemm(n, 2 * m, W, P, n.G, 2 * m, 1, 0, du, W, 0, (long long)P * W, n.dyh, W, (long long)2 * m * W, B, 1.f,
             0.f);
        // dRre[k] = re^T dyre + im^T dyim ; dRim[k] = re^T dyim - im^T dyre
        gemm(n, W, W, B, vh, ld, 1, W, n.dyh, ld, 0, W, g + n.o_rre[l], W, (long long)W * W, m, 1.f, 0.f);
        gemm(n, W, W, B, vh + m * W, ld, 1, W, n.dyh + m * W, ld, 0, W, g + n.o_rre[l], W, (long long)W * W, m, 1.f,
             1.f);
        gemm(n, W, W, B, vh, ld, 1, W, n.dyh + m * W, ld, 0, W, g + n.o_rim[l], W, (long long)W * W, m, 1.f, 0.f);
        gemm(n, W, W, B, vh + m * W, ld, 1, W, n.dyh, ld, 0, W, g + n.o_rim[l], W, (long long)W * W, m, -1.f, 1.f);
        // dre = dyre Rre^T + dyim Rim^T ; dim = -dyre Rim^T + dyim Rre^T
        gemm(n, B, W, W, n.dyh, ld, 0, W, rre, W, 1, (long long)W * W, n.dvh, ld, W, m, 1.f, 0.f);
        gemm(n, B, W, W, n.dyh + m * W, ld, 0, W, rim, W, 1, (long long)W * W, n.dvh, ld, W, m, 1.f, 1.f);
        gemm(n, B, W, W, n.dyh, ld, 0, W, rim, W, 1, (long long)W * W, n.dvh + m * W, ld, W, m, -1.f, 0.f);
        gemm(n, B, W, W, n.dyh + m * W, ld, 0, W, rre, W, 1, (long long)W * W, n.dvh + m * W, ld, W, m, 1.f, 1.f);
        // dv = du W^T + F^T dvh[b]
        gemm(n, P, W, 2 * m, n.F, P, 1, 0, n.dvh, W, 0, (long long)2 * m * W, n.dv2, W, (long long)P * W, B, 1.f,
             1.f);
        std::swap(n.dv, n.dv2);
    }
    gemm(n, kCin, W, (int)rows, n.a, kCin, 1, 0, n.dv, W, 0, 0, g + n.o_lw, W, 0, 1, 1.f, 0.f);
    colsum_kernel<<<W, 256, 0, n.stream>>>(n.dv, rows, W, g + n.o_lb);
    return cudaGetLastError() == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
}

int upload_inputs(NNet& n, const float* raw, const float* tgt, int B) {
    if (cudaMemcpyAsync(n.raw, raw, (size_t)B * 5 * 4, cudaMemcpyHostToDevice, n.stream) != cudaSuccess)
        return FDLB_ECUDA;
    if (tgt && cudaMemcpyAsync(n.tgt, tgt, (size_t)B * n.P * kCout * 4, cudaMemcpyHostToDevice, n.stream) != cudaSuccess)
        return FDLB_ECUDA;
    return FDLB_OK;
}

}  // namespace
}  // namespace fdlb

using fdlb::NNet;

extern "C" {

int fdlb_nn_create(int width, int modes, int layers, int hidden, int n_points, int max_batch, void* cuda_stream,
                   fdlb_nn_handle* out) try {
    if (!out || width < 1 || width > 512 || modes < 1 || 2 * modes > n_points || layers < 1 || layers > 16 ||
        hidden < 1 || n_points < 8 || n_points > 4096 || max_batch < 1 || max_batch > 4096)
        return FDLB_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return FDLB_ENOGPU;
    auto* n = new NNet();
    n->W = width;
    n->m = modes;
    n->L = layers;
    n->H = hidden;
    n->P = n_points;
    n->Bmax = max_batch;
    long long off = 0;
    auto take = [&](long long sz) {
        const long long o = off;
        off += sz;
        return o;
    };
    const int W = width;
    n->o_lw = take((long long)fdlb::kCin * W);
    n->o_lb = take(W);
    for (int l = 0; l < layers; ++l) {
        n->o_rre.push_back(take((long long)modes * W * W));
        n->o_rim.push_back(take((long long)modes * W * W));
        n->o_w.push_back(take((long long)W * W));
        n->o_b.push_back(take(W));
    }
    n->o_p1w = take((long long)W * hidden);
    n->o_p1b = take(hidden);
    n->o_p2w = take((long long)hidden * fdlb::kCout);
    n->o_p2b = take(fdlb::kCout);
    n->n_params = off;
    // workspace
    const long long rows = (long long)max_batch * n_points;
    const long long np = n->n_params;
    std::vector<std::pair<void**, size_t>> bufs = {
        {(void**)&n->w, np * 4},  {(void**)&n->g, np * 4},  {(void**)&n->m1, np * 4}, {(void**)&n->m2, np * 4},
        {(void**)&n->wb, np * 2}, {(void**)&n->F, (size_t)2 * modes * n_points * 4},
        {(void**)&n->G, (size_t)2 * modes * n_points * 4}, {(void**)&n->raw, (size_t)max_batch * 5 * 4},
        {(void**)&n->a, rows * fdlb::kCin * 4}, {(void**)&n->vs, (size_t)(layers + 1) * rows * W * 4},
        {(void**)&n->us, (size_t)layers * rows * W * 4}, {(void**)&n->vh, (size_t)layers * max_batch * 2 * modes * W * 4},
        {(void**)&n->yh, (size_t)max_batch * 2 * modes * W * 4}, {(void**)&n->z1, rows * hidden * 4},
        {(void**)&n->h, rows * hidden * 4}, {(void**)&n->out, rows * fdlb::kCout * 4},
        {(void**)&n->tgt, rows * fdlb::kCout * 4}, {(void**)&n->dout, rows * fdlb::kCout * 4},
        {(void**)&n->dh, rows * hidden * 4}, {(void**)&n->dv, rows * W * 4}, {(void**)&n->dv2, rows * W * 4},
        {(void**)&n->dyh, (size_t)max_batch * 2 * modes * W * 4}, {(void**)&n->dvh, (size_t)max_batch * 2 * modes * W * 4},
        {(void**)&n->loss, 256}};
    size_t total = 0;
    for (auto& b : bufs) total += (b.second + 255) / 256 * 256;
    if (cudaMalloc(&n->ws, total) != cudaSuccess) {
        delete n;
        return FDLB_ENOMEM;
    }
    size_t o = 0;
    for (auto& b : bufs) {
        *b.first = n->ws + o;
        o += (b.second + 255) / 256 * 256;
    }
    n->stream = (cudaStream_t)cuda_stream;
    if (!n->stream) {
        cudaStreamCreate(&n->stream);
        n->own_stream = true;
    }
    cudaMemsetAsync(n->ws, 0, total, n->stream);
    // DFT rows F [2m][P] (cos, -sin) and the truncated inverse G [P][2m]
    std::vector<float> F((size_t)2 * modes * n_points), G((size_t)2 * modes * n_points);
    const double pi2 = 6.283185307179586477;
    for (int k = 0; k < modes; ++k)
        for (int x = 0; x < n_points; ++x) {
            const double ang = pi2 * k * x / n_points, c = k == 0 ? 1.0 : 2.0;
            F[(size_t)k * n_points + x] = (float)std::cos(ang);
            F[(size_t)(modes + k) * n_points + x] = (float)-std::sin(ang);
            G[(size_t)x * 2 * modes + k] = (float)(c * std::cos(ang) / n_points);
            G[(size_t)x * 2 * modes + modes + k] = (float)(-c * std::sin(ang) / n_points);
        }
    cudaMemcpyAsync(n->F, F.data(), F.size() * 4, cudaMemcpyHostToDevice, n->stream);
    cudaMemcpyAsync(n->G, G.data(), G.size() * 4, cudaMemcpyHostToDevice, n->stream);
    if (cudaStreamSynchronize(n->stream) != cudaSuccess) {
        cudaFree(n->ws);
        delete n;
        return FDLB_ECUDA;
    }
    *out = reinterpret_cast<fdlb_nn_handle>(n);
    return FDLB_OK;
} FDLB_HOST_CATCH

void fdlb_nn_destroy(fdlb_nn_handle h) {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    cudaFree(n->ws);
    if (n->own_stream) cudaStreamDestroy(n->stream);
    delete n;
}

int fdlb_nn_num_params(fdlb_nn_handle h, int64_t* count) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n || !count) return FDLB_EINVAL;
    *count = n->n_params;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_nn_set_params(fdlb_nn_handle h, const float* theta) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n || !theta) return FDLB_EINVAL;
    if (cudaMemcpyAsync(n->w, theta, n->n_params * 4, cudaMemcpyHostToDevice, n->stream) != cudaSuccess)
        return FDLB_ECUDA;
    cudaMemsetAsync(n->m1, 0, n->n_params * 4, n->stream);
    cudaMemsetAsync(n->m2, 0, n->n_params * 4, n->stream);
    fdlb::to_bf16_kernel<<<fdlb::grid_for(n->n_params), 256, 0, n->stream>>>(n->w, n->wb, n->n_params);
    n->step = 0;
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
} FDLB_HOST_CATCH

int fdlb_nn_init_params(fdlb_nn_handle h, uint64_t seed) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n) return FDLB_EINVAL;
    // seeded initialisation (splitmix64 uniforms): weight matrices U(-1, 1)/sqrt(fan_in), spectral
    // weights U(0, 1)/width^2, biases 0
    std::vector<float> t(n->n_params, 0.f);
    uint64_t st = seed;
    auto uni = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](long long off, long long cnt, double lo, double hi) {
        for (long long e = 0; e < cnt; ++e) t[off + e] = (float)(lo + (hi - lo) * uni());
    };
    const int W = n->W;
    fill(n->o_lw, (long long)fdlb::kCin * W, -1.0 / std::sqrt((double)fdlb::kCin), 1.0 / std::sqrt((double)fdlb::kCin));
    for (int l = 0; l < n->L; ++l) {
        fill(n->o_rre[l], (long long)n->m * W * W, 0.0, 1.0 / ((double)W * W));
        fill(n->o_rim[l], (long long)n->m * W * W, 0.0, 1.0 / ((double)W * W));
        fill(n->o_w[l], (long long)W * W, -1.0 / std::sqrt((double)W), 1.0 / std::sqrt((double)W));
    }
    fill(n->o_p1w, (long long)W * n->H, -1.0 / std::sqrt((double)W), 1.0 / std::sqrt((double)W));
    fill(n->o_p2w, (long long)n->H * fdlb::kCout, -1.0 / std::sqrt((double)n->H), 1.0 / std::sqrt((double)n->H));
    return fdlb_nn_set_params(h, t.data());
} FDLB_HOST_CATCH

int fdlb_nn_get_params(fdlb_nn_handle h, float* theta) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n || !theta) return FDLB_EINVAL;
    if (cudaMemcpyAsync(theta, n->w, n->n_params * 4, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess)
        return FDLB_ECUDA;
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
} FDLB_HOST_CATCH

int fdlb_nn_forward(fdlb_nn_handle h, const float* raw_params, int batch, float* out_host) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n || !raw_params || !out_host || batch < 1 || batch > n->Bmax) return FDLB_EINVAL;
    int rc = fdlb::upload_inputs(*n, raw_params, nullptr, batch);
    if (!rc) rc = fdlb::forward(*n, batch);
    if (rc) return rc;
    if (cudaMemcpyAsync(out_host, n->out, (size_t)batch * n->P * fdlb::kCout * 4, cudaMemcpyDeviceToHost, n->stream) !=
        cudaSuccess)
        return FDLB_ECUDA;
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
} FDLB_HOST_CATCH

int fdlb_nn_loss_grad(fdlb_nn_handle h, const float* raw_params, const float* targets, int batch, float* loss,
                      float* grad_host) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n || !raw_params || !targets || batch < 1 || batch > n->Bmax) return FDLB_EINVAL;
    int rc = fdlb::upload_inputs(*n, raw_params, targets, batch);
    if (!rc) rc = fdlb::forward(*n, batch);
    if (rc) return rc;
    const long long cnt = (long long)batch * n->P * fdlb::kCout;
    fdlb::mse_kernel<<<1, 1024, 0, n->stream>>>(n->out, n->tgt, cnt, n->dout, n->loss);
    rc = fdlb::backward(*n, batch);
    if (rc) return rc;
    if (loss && cudaMemcpyAsync(loss, n->loss, 4, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess) return FDLB_ECUDA;
    if (grad_host &&
        cudaMemcpyAsync(grad_host, n->g, n->n_params * 4, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess)
        return FDLB_ECUDA;
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
} FDLB_HOST_CATCH

int fdlb_nn_train_step(fdlb_nn_handle h, const float* raw_params, const float* targets, int batch, float lr,
                       float* loss) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n || !(lr > 0.f)) return FDLB_EINVAL;
    int rc = fdlb_nn_loss_grad(h, raw_params, targets, batch, loss, nullptr);
    if (rc) return rc;
    n->step++;
    const float c1 = 1.f - std::pow(0.9f, (float)n->step), c2 = 1.f - std::pow(0.999f, (float)n->step);
    fdlb::adam_kernel<<<fdlb::grid_for(n->n_params), 256, 0, n->stream>>>(n->w, n->g, n->m1, n->m2, n->wb, n->n_params,
                                                                         lr, c1, c2);
    return cudaStreamSynchronize(n->stream) == cudaSuccess ? FDLB_OK : FDLB_ECUDA;
} FDLB_HOST_CATCH

int fdlb_nn_warm_start(fdlb_nn_handle h, fdlb_handle solver, int instance, const float* raw_params) try {
    NNet* n = reinterpret_cast<NNet*>(h);
    if (!n || !solver || !raw_params) return FDLB_EINVAL;
    fdlb_info info;
    int rc = fdlb_get_info(solver, instance, &info);
    if (rc) return rc;
    std::vector<float> out((size_t)n->P * fdlb::kCout);
    rc = fdlb_nn_forward(h, raw_params, 1, out.data());
    if (rc) return rc;
    // decode: n = n0 (1 + o0), u_2 = 0.1 o1, T = T_in (1 + 0.1 o2), q_R = 0.01 n0 T_in^1.5 o3, with
    // T_in = 1 (the parameter sweep fixes the inner wall at T = 1; T_out = T_in * ratio)
    const double Tin = 1.0;
    std::vector<double> nn(n->P), u2(n->P), T(n->P), qR(n->P);
    for (int x = 0; x < n->P; ++x) {
        const float* o = &out[(size_t)x * fdlb::kCout];
        nn[x] = info.n0 * std::max(0.05, 1.0 + (double)o[0]);
        u2[x] = 0.1 * (double)o[1];
        T[x] = Tin * std::max(0.05, 1.0 + 0.1 * (double)o[2]);
        qR[x] = 0.01 * info.n0 * Tin * std::sqrt(Tin) * (double)o[3];
    }
    // The walls conserve mass, so the steady state depends on the total mass: the seed must carry
    // the instance's own mass (that of its uniform start).  The seeded populations are linear in
    // (n, q_R) at fixed u_2 and T, so scaling both profiles scales the mass exactly.
    double m_uniform = 0.0, m_seed = 0.0;
    rc = fdlb_init_uniform(solver, instance, 0.0, 0.0);
    if (!rc) rc = fdlb_get_diagnostics(solver, instance, &m_uniform, nullptr, nullptr);
    if (!rc) rc = fdlb_init_from_moments(solver, instance, nn.data(), u2.data(), T.data(), qR.data(), n->P);
    if (!rc) rc = fdlb_get_diagnostics(solver, instance, &m_seed, nullptr, nullptr);
    if (rc) return rc;
    if (!(m_seed > 0.0) || !(m_uniform > 0.0)) return FDLB_ENAN;
    const double lam = m_uniform / m_seed;
    for (int x = 0; x < n->P; ++x) {
        nn[x] *= lam;
        qR[x] *= lam;
    }
    return fdlb_init_from_moments(solver, instance, nn.data(), u2.data(), T.data(), qR.data(), n->P);
} FDLB_HOST_CATCH

}  // extern "C"
