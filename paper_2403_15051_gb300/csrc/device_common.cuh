// Device helpers shared by the kernel translation units: PTX wrappers for the bulk-copy
// engine and mbarriers, the WENO5 reconstruction, the Carnahan-Starling contact value and
// warp reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdlb {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// One-dimensional bulk copy global -> shared by the TMA engine; completion is counted in
// bytes on `bar`.  Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Asks the bulk-copy engine to bring `bytes` at `src` into L2 (a hint: no completion, no effect on
// results).  Address 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after 1 s of global time (a copy completes in microseconds), or after
// 2^22 tries (each suspends for a hardware-chosen interval) whichever comes first.  Returns false
// if the phase never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = global_ns();
    for (int it = 1; it < (1 << 22); ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((it & 63) == 0 && global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization may
// start while its predecessor in the stream is still running: it does only work that reads
// nothing the predecessor writes (constant tables into shared memory), then pdl_wait(), which
// returns once the predecessor grid has completed and its memory is visible.  pdl_trigger() lets
// the successor be scheduled as soon as every block of this grid has started.  Both are no-ops
// for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// TF32 tensor-core helpers: round to TF32 (ties away), and the warp-wide m16n8k8 product with
// FP32 accumulation.  Fragment ownership (g = lane / 4, t = lane % 4): A (16 x 8, row major)
// a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4); B (8 x 8) b0 (t, g), b1 (t + 4, g);
// C, D (16 x 8) c0 (g, 2t), c1 (g, 2t + 1), c2 (g + 8, 2t), c3 (g + 8, 2t + 1).
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <typename T>
__device__ __forceinline__ T ldg_t(const T* p) {
    return __ldg(p);
}

__device__ __forceinline__ float ratio_fast(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double ratio_fast(double a, double b) { return a / b; }

// Fifth-order WENO reconstruction (Jiang & Shu 1996; epsilon 1e-6, power 2) at the right face
// of the cell holding c, upwind from the left; reversing the five arguments gives the value at
// the left face of the cell holding c, upwind from the right.  The nonlinear weights
// d_k / (eps + beta_k)^2 are scaled by the square of the smallest (eps + beta_k), which leaves
// the normalised weights unchanged and keeps every intermediate in [0, 1] (no FP32 overflow for
// large populations).
template <typename T>
__device__ __forceinline__ T weno5(T a, T b, T c, T d, T e) {
    const T eps = T(1e-6);
    const T k13 = T(13.0 / 12.0), q = T(0.25);
    const T t0 = a - T(2) * b + c, t1 = a - T(4) * b + T(3) * c;
    const T t2 = b - T(2) * c + d, t3 = b - d;
    const T t4 = c - T(2) * d + e, t5 = T(3) * c - T(4) * d + e;
    const T e0 = eps + k13 * t0 * t0 + q * t1 * t1;
    const T e1 = eps + k13 * t2 * t2 + q * t3 * t3;
    const T e2 = eps + k13 * t4 * t4 + q * t5 * t5;
    const T m = fmin(e0, fmin(e1, e2));
    const T s0 = ratio_fast(m, e0), s1 = ratio_fast(m, e1), s2 = ratio_fast(m, e2);
    const T a0 = T(0.1) * s0 * s0, a1 = T(0.6) * s1 * s1, a2 = T(0.3) * s2 * s2;
    const T r0 = T(2) * a - T(7) * b + T(11) * c;
    const T r1 = -b + T(5) * c + T(2) * d;
    const T r2 = T(2) * c + T(5) * d - e;
    return ratio_fast(a0 * r0 + a1 * r1 + a2 * r2, T(6) * (a0 + a1 + a2));
}

// ---- pairs of lanes: two momenta of a vector per instruction.  FP32 pairs use the packed FP32x2
// operations of the sm_100 family (__ffma2_rn, __fadd2_rn, __fmul2_rn: one issue slot for two
// FP32 operations, each lane rounded like the scalar operation); FP64 pairs are two scalar
// operations.  Every operation is written out (nothing is left to the compiler's contraction),
// so a lane's result is the same whichever pair it travels in.
template <typename T>
struct PairT;
template <>
struct PairT<float> {
    using type = float2;
};
template <>
struct PairT<double> {
    using type = double2;
};
template <typename T>
using Pair = typename PairT<T>::type;

__device__ __forceinline__ float2 p_make(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 p_make(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 p_splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ double2 p_splat(double a) { return make_double2(a, a); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 p_fma(double2 a, double2 b, double2 c) {
    return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 p_add(double2 a, double2 b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 p_mul(double2 a, double2 b) { return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)); }
// a - b: b times -1 is exact, so the fused form rounds once, like a subtraction
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double2 p_sub(double2 a, double2 b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
__device__ __forceinline__ float2 p_min(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }
__device__ __forceinline__ double2 p_min(double2 a, double2 b) { return make_double2(fmin(a.x, b.x), fmin(a.y, b.y)); }
// Approximate FP32 reciprocal (the PTX rcp.approx instruction: at most one unit in the last place
// off, subnormals flushed to zero).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// a / b lane by lane: for FP32 the product with the approximate reciprocal (the operands here are
// normal numbers well inside the range); for FP64 the correctly rounded quotient.
__device__ __forceinline__ float2 p_ratio(float2 a, float2 b) {
    return __fmul2_rn(a, make_float2(rcp_approx(b.x), rcp_approx(b.y)));
}
__device__ __forceinline__ double2 p_ratio(double2 a, double2 b) { return make_double2(a.x / b.x, a.y / b.y); }

// The same reconstruction written on the window in ascending cell order, w0..w4, for either
// upwind direction: sigma = +1 gives weno5(w0, .., w4) (value at the right face of w2's cell,
// from the left), sigma = -1 gives weno5(w4, .., w0) (left face, from the right).  The three
// smoothness indicators belong to the left, centre and right stencils whatever the direction,
// and every candidate value is (D_k + 12 w2 -+ 3 sigma t_k) / 2 with D_k the stencil's second
// difference and t_k the first-difference part of its indicator, so the value is
// w2 + sum_k a_k X_k / (12 sum_k a_k), X_k = D_k +- 3 sigma t_k.  The linear weights follow the
// direction: (dL, dC, dR) = (0.1, 0.6, 0.3) or (0.3, 0.6, 0.1); s3 = 3 sigma.  Indicators are
// taken four times over (e4 + 13/3 D^2 + t^2, e4 = 4 eps): the normalised weights are unchanged.
// The reconstruction is homogeneous of degree one in the window once eps scales with its square:
// the value for c w0..c w4 with c^2 e4 is c times the value for w0..w4 with e4.
// Written for a pair of momenta (one packed operation per step for FP32 pairs).  The window's
// first difference enters negated (w0 - w1), and so does the centre stencil's first-difference
// part (-tC = d1 + d2), which the indicators square and the candidate values take with the
// opposite sign: no negation is ever formed.  s3, ns3 = 3 sigma and its negative; dL, dR the
// linear weights of the outer stencils; e4 = 4 eps (w^2 for the reconstruction of f, below).
template <typename T>
__device__ __forceinline__ Pair<T> weno5_pair(Pair<T> w0, Pair<T> w1, Pair<T> w2, Pair<T> w3, Pair<T> w4, Pair<T> s3,
                                              Pair<T> ns3, Pair<T> dL, Pair<T> dR, Pair<T> e4) {
    using P = Pair<T>;
    const P nd0 = p_sub(w0, w1), d1 = p_sub(w2, w1), d2 = p_sub(w3, w2), d3 = p_sub(w4, w3);
    const P D1 = p_add(d1, nd0), D2 = p_sub(d2, d1), D3 = p_sub(d3, d2);
    const P tL = p_fma(p_splat(T(3)), d1, nd0);    // 3 d1 - d0
    const P ntC = p_add(d1, d2);                    // -tC
    const P tR = p_fma(p_splat(T(-3)), d2, d3);     // d3 - 3 d2
    const P c = p_splat(T(13.0 / 3.0));
    const P EL = p_fma(tL, tL, p_fma(p_mul(c, D1), D1, e4));
    const P EC = p_fma(ntC, ntC, p_fma(p_mul(c, D2), D2, e4));
    const P ER = p_fma(tR, tR, p_fma(p_mul(c, D3), D3, e4));
    const P m = p_min(EL, p_min(EC, ER));
    const P sL = p_ratio(m, EL), sC = p_ratio(m, EC), sR = p_ratio(m, ER);
    const P aL = p_mul(dL, p_mul(sL, sL)), aC = p_mul(p_splat(T(0.6)), p_mul(sC, sC)), aR = p_mul(dR, p_mul(sR, sR));
    const P XL = p_fma(s3, tL, D1), XC = p_fma(s3, ntC, D2), XR = p_fma(ns3, tR, D3);
    const P num = p_fma(aR, XR, p_fma(aC, XC, p_mul(aL, XL)));
    const P den = p_mul(p_splat(T(12)), p_add(p_add(aL, aC), aR));
    return p_add(w2, p_ratio(num, den));
}

// ---- wide accumulators: plain FP64 for FP64 populations; for FP32 populations a double-float
// (hi + lo, about 44 significant bits) on the FP32 pipe, because FP64 arithmetic on GB300 costs
// 64 cycles per dependent operation and about 440 per division.  The error-free transformations
// are Knuth's TwoSum and the fused-multiply-add TwoProduct (Dekker 1971; the double-double
// algorithms of Hida, Li and Bailey 2001, restated for float pairs).
template <typename T>
struct Wide;
template <>
struct Wide<double> {
    double v;
};
template <>
struct Wide<float> {
    float hi, lo;
};

__device__ __forceinline__ Wide<double> w_from(double s, double*) { return {s}; }
__device__ __forceinline__ Wide<float> w_from(double s, float*) {
    const float hi = __double2float_rn(s);
    return {hi, __double2float_rn(s - (double)hi)};
}
__device__ __forceinline__ Wide<double> w_from_t(double x) { return {x}; }
__device__ __forceinline__ Wide<float> w_from_t(float x) { return {x, 0.f}; }
__device__ __forceinline__ double w_hi(Wide<double> a) { return a.v; }
__device__ __forceinline__ float w_hi(Wide<float> a) { return a.hi; }
__device__ __forceinline__ Wide<double> w_add(Wide<double> a, Wide<double> b) { return {a.v + b.v}; }
__device__ __forceinline__ Wide<double> w_sub(Wide<double> a, Wide<double> b) { return {a.v - b.v}; }
__device__ __forceinline__ Wide<double> w_mul(Wide<double> a, Wide<double> b) { return {a.v * b.v}; }
__device__ __forceinline__ Wide<double> w_div(Wide<double> a, Wide<double> b) { return {a.v / b.v}; }
__device__ __forceinline__ Wide<double> w_scale(Wide<double> a, double c) { return {a.v * c}; }

__device__ __forceinline__ Wide<float> w_norm(float s, float e) {  // |s| >= |e|
    const float hi = s + e;
    return {hi, e - (hi - s)};
}
__device__ __forceinline__ Wide<float> w_add(Wide<float> a, Wide<float> b) {
    const float s = a.hi + b.hi, v = s - a.hi;
    float e = (a.hi - (s - v)) + (b.hi - v);
    e += a.lo + b.lo;
    return w_norm(s, e);
}
__device__ __forceinline__ Wide<float> w_sub(Wide<float> a, Wide<float> b) { return w_add(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ Wide<float> w_mul(Wide<float> a, Wide<float> b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return w_norm(p, e);
}
__device__ __forceinline__ Wide<float> w_scale(Wide<float> a, float c) {
    const float p = a.hi * c;
    const float e = fmaf(a.lo, c, fmaf(a.hi, c, -p));
    return w_norm(p, e);
}
// a / b: a first quotient, the remainder a - q1 b in double-float, a correction.  The two
// quotients need only single-precision accuracy (the remainder is exact to the double-float
// level), so they are the fast ones.
__device__ __forceinline__ Wide<float> w_div(Wide<float> a, Wide<float> b) {
    const float q1 = __fdividef(a.hi, b.hi);
    const Wide<float> r = w_sub(a, w_scale(b, q1));
    return w_norm(q1, __fdividef(r.hi, b.hi));
}
__device__ __forceinline__ Wide<double> w_shfl_xor(Wide<double> a, int o) { return {__shfl_xor_sync(0xffffffffu, a.v, o)}; }
__device__ __forceinline__ Wide<float> w_shfl_xor(Wide<float> a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

template <typename T>
__device__ __forceinline__ T chi_cs_t(T eta) {
    const T om = T(1) - eta;
    return (T(2) - eta) / (T(2) * om * om * om);
}

__device__ __forceinline__ double chi_cs(double eta) {
    const double om = 1.0 - eta;
    return (2.0 - eta) / (2.0 * om * om * om);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of 16 values over the 32 lanes of a warp, transposed: at every level of the butterfly a
// lane keeps half of its values and sends the other half, so the warp needs 16 shuffles instead
// of 16 x 5.  Lane L returns the sum of value (L >> 1).  Fixed order: deterministic.
template <typename T>
__device__ __forceinline__ T warp_sum16_transposed(const T (&v)[16], int lane) {
    T w8[8], w4[4], w2[2];
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const T send = b4 ? v[t] : v[t + 8], keep = b4 ? v[t + 8] : v[t];
        w8[t] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const T send = b3 ? w8[t] : w8[t + 4], keep = b3 ? w8[t + 4] : w8[t];
        w4[t] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const T send = b2 ? w4[t] : w4[t + 2], keep = b2 ? w4[t + 2] : w4[t];
        w2[t] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    const T send = b1 ? w2[0] : w2[1], keep = b1 ? w2[1] : w2[0];
    const T w1 = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    return w1 + __shfl_xor_sync(0xffffffffu, w1, 1);
}

// Five-point derivative stencil in the mapped coordinate (gradients of Eq. j1): fourth-order
// central in the interior, one-sided fourth-order at the two cells next to each wall.
template <typename R>
__device__ __forceinline__ void stencil5(int c, int N, int* idx, R* w) {
    const R k = R(1) / R(12);
    if (c >= 2 && c <= N - 3) {
        idx[0] = c - 2; idx[1] = c - 1; idx[2] = c; idx[3] = c + 1; idx[4] = c + 2;
        w[0] = k; w[1] = -8 * k; w[2] = 0; w[3] = 8 * k; w[4] = -k;
    } else if (c == 0) {
        for (int q = 0; q < 5; ++q) idx[q] = q;
        w[0] = -25 * k; w[1] = 48 * k; w[2] = -36 * k; w[3] = 16 * k; w[4] = -3 * k;
    } else if (c == 1) {
        for (int q = 0; q < 5; ++q) idx[q] = q;
        w[0] = -3 * k; w[1] = -10 * k; w[2] = 18 * k; w[3] = -6 * k; w[4] = k;
    } else if (c == N - 2) {
        for (int q = 0; q < 5; ++q) idx[q] = N - 1 - q;
        w[0] = 3 * k; w[1] = 10 * k; w[2] = -18 * k; w[3] = 6 * k; w[4] = -k;
    } else {
        for (int q = 0; q < 5; ++q) idx[q] = N - 1 - q;
        w[0] = 25 * k; w[1] = -48 * k; w[2] = 36 * k; w[3] = -16 * k; w[4] = 3 * k;
    }
}

}  // namespace fdlb
