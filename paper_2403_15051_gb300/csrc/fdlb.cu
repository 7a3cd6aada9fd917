// Host side of the FDLB library: device state, launch sequencing, CUDA graphs, steady-state
// driver, checkpoints and the C ABI declared in include/fdlb.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "internal.h"
#include "kernels_decl.h"

namespace fdlb {

namespace {

constexpr double kPiH = 3.14159265358979323846;
constexpr size_t kAlign = 256;
// Radial node counts from which the K^h contraction runs as its own kernel (the fused stage then
// reads K^h f; below, the stage contracts from a K^h table in shared memory).
constexpr int kKrKernelMinNodes = 32;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte layout of all device state, computed identically for sizing and carving.
struct Layout {
    size_t f[3], sums[3], sumsw[3], dens[3], ca, cw, rec, tab, tabT, inst, geo, geoT, gw, gwT, band, band_lo, sitems, n_sitems, citems,
        n_citems, nwp, err, gbar,
        rprev, rout, krf, krB, mpk, bpairs, n_bpairs, k3f, total;
};

}  // namespace

struct Solver {
    int n_inst = 0, geometry = 0, precision = 0;
    int reduced = 0;  // FDLB_CYL_Z: the cylinder's kernels on the pair (phi, chi) as the third index
    size_t tsize = 8;
    AxisRule aR, a2, a3;
    int NR = 0, N2 = 0, N3 = 0, nR = 0, n2 = 0, n3 = 0, Np = 0;
    std::vector<InstanceSetup> setup;
    std::vector<InstDev> inst_h;
    std::vector<long long> f_off;
    std::vector<int> cell_off;
    int total_cells = 0;
    size_t f_elems = 0, band_elems = 0;
    int max_sitems = 0, max_citems = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, n_sm = 0;
    size_t smem_optin = 0, smem_per_sm = 0;
    // device memory
    unsigned char* ws = nullptr;
    bool own_ws = false;
    Layout lay{};
    void* f[3] = {nullptr, nullptr, nullptr};
    double* sums[3] = {nullptr, nullptr, nullptr};
    void* sumsw[3] = {nullptr, nullptr, nullptr};
    void* dens[3] = {nullptr, nullptr, nullptr};
    void *geoT = nullptr, *gwT = nullptr, *nwp = nullptr, *cw = nullptr;
    void* rec = nullptr;
    void* tabT = nullptr;
    BandPair* bpairs = nullptr;  // the batch closure's band jobs (per work list)
    int* n_bpairs = nullptr;
    double *ca = nullptr, *mpk = nullptr, *tab = nullptr, *geo = nullptr, *gw = nullptr, *rprev = nullptr,
           *rout = nullptr;
    InstDev* inst_d = nullptr;
    void* band = nullptr;
    int* band_lo = nullptr;
    int4 *sitems = nullptr, *citems = nullptr;
    int *n_sitems = nullptr, *n_citems = nullptr, *err = nullptr;
    unsigned* gbar = nullptr;
    std::vector<double> tab_h;
    MomSet M{};
    // tiling of the stream kernel
    int B = 16, KS = 1, threads = 0;
    StreamCfg scfg{1, 4, 0};
    size_t smem_stream = 0;
    int use_bulk = 0;
    int closure_cells = 4, closure_threads = 128;  // own cells per closure item (<= kClosureCells)
    int closure_batch = 0;  // the closure as two launches over all items (items of kClosureCells cells)
    int grid_cbatch = 1;
    size_t cbatch_smem = 0;
    int autotune_mode = 1;  // 0 off; 1 tune on the first step of a batch; 2 also of a single instance
    int stall_checks = 0;   // run_to_steady: checks without halving the best residual before an instance stops
    int stage_minb = 1;     // register bound of the stage kernel (1; 3, 2 or 5 blocks per SM where built)
    bool tuned = false;     // the tuner has run (or its cached choice was applied) for this handle
    int closure_wst = 0;                           // staged band-row elements per closure block
    int grid_stream = 1, grid_closure = 1;
    size_t closure_smem = 0;
    int max_union = 1;
    std::vector<char> active;
    std::vector<int64_t> inst_steps;
    std::vector<double> last_res;
    cudaGraphExec_t gexec = nullptr;
    int64_t launches = 0, last_launches = 0;
    bool prev_valid = false;
    int graph_steps = 20;
    // per-kernel timing (events around each launch, direct launches)
    bool timing = false;
    int programmatic = 1;  // closure and stage kernels overlap their prologues with the predecessor
    int tensor = 0;        // K^h contraction on the tensor cores where available
    void* krf = nullptr;   // K^h f of the stage input (contraction kernel), when allocated
    int krg_on = 0;        // the contraction kernel is in use
    void* k3f = nullptr;   // sphere: K_3 f of the stage input, when the momenta are sliced along p_3
    int k3_on = 0;         // ... and in use (slices narrower than the p_3 axis)
    float* krB = nullptr;  // K^h as TF32 pairs in the tensor-core kernel's layout (FP32 populations)
    int kr_tc = 0;         // the contraction kernel runs on the tensor cores
    int mma_on = 0;        // ... and in use for the current tiling
    // persistent step kernel (closure + stage per tile, grid barriers between stages)
    int fused = 0;         // use it where the configuration allows (off by default: slower on GB300)
    int test_tx_extra = 0, test_bar_extra = 0;  // test hooks of the bounded waits (0 in use)
    int fused_on = 0;      // ... and in use for the current tiling
    int grid_step = 0, step_wst = 0, step_clo_off = 0, max_tile = 0;
    size_t smem_step = 0;
    cudaEvent_t tev[3] = {nullptr, nullptr, nullptr};
    double t_stream_ms = 0.0, t_closure_ms = 0.0, t_step_ms = 0.0;
    int64_t n_step_t = 0, n_step_steps = 0;
    int64_t n_stream_t = 0, n_closure_t = 0;
};

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return FDLB_OK;
    if (e == cudaErrorMemoryAllocation) return FDLB_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return FDLB_ENOGPU;
    return FDLB_ECUDA;
}

namespace {

#define FDLB_CUDA(call)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return ::fdlb::cuda_status(e_); \
    } while (0)

// Table buffer (FP64) shared by all instances: nodes, weights, K matrices, equilibrium
// tables of Sec. III.C and the half-range recurrence.
void build_tables(Solver& S) {
    auto& t = S.tab_h;
    t.clear();
    auto put = [&](const std::vector<double>& v) {
        int o = (int)t.size();
        t.insert(t.end(), v.begin(), v.end());
        return o;
    };
    MomSet& M = S.M;
    M.o_pR = put(S.aR.p);
    M.o_wR = put(S.aR.w);
    M.o_p2 = put(S.a2.p);
    M.o_w2 = put(S.a2.w);
    M.o_p3 = put(S.a3.p);
    M.o_w3 = put(S.a3.w);
    std::vector<double> K;
    k_half_matrix(S.aR, K);
    M.o_KR = put(K);
    k2_full_matrix(S.a2, K);
    M.o_K2 = put(K);
    k2_full_matrix(S.a3, K);
    M.o_K3 = put(K);
    // GR[k][l] = w_k h_l(|p_k|);  G2[j][l] = w_j He_l(p_j) / l!
    const int QR = S.aR.Q;
    std::vector<double> GR((size_t)S.nR * kMaxE, 0.0), G2((size_t)S.n2 * kMaxE, 0.0), G3((size_t)S.n3 * kMaxE, 0.0);
    for (int k = 0; k < S.nR; ++k) {
        const double x = std::fabs(S.aR.p[k]);
        double h[kMaxE + 2];
        h[0] = 1.0 / std::sqrt(S.aR.beta[0]);
        if (S.NR >= 1) h[1] = (x - S.aR.alpha[0]) * h[0] / std::sqrt(S.aR.beta[1]);
        for (int l = 1; l < S.NR; ++l)
            h[l + 1] = ((x - S.aR.alpha[l]) * h[l] - std::sqrt(S.aR.beta[l]) * h[l - 1]) / std::sqrt(S.aR.beta[l + 1]);
        for (int l = 0; l <= S.NR; ++l) GR[(size_t)k * kMaxE + l] = S.aR.w[k] * h[l];
    }
    auto fill_full = [&](const AxisRule& ax, int N, std::vector<double>& G) {
        for (int j = 0; j < ax.Q; ++j) {
            double h0 = 1.0, h1 = ax.p[j], fact = 1.0;
            for (int l = 0; l <= N; ++l) {
                double He = l == 0 ? 1.0 : (l == 1 ? ax.p[j] : 0.0);
                if (l >= 2) {
                    He = ax.p[j] * h1 - (l - 1) * h0;
                    h0 = h1;
                    h1 = He;
                }
                if (l > 0) fact *= l;
                G[(size_t)j * kMaxE + l] = ax.w[j] * He / fact;
            }
        }
    };
    fill_full(S.a2, S.N2, G2);
    fill_full(S.a3, S.N3, G3);
    M.o_GR = put(GR);
    M.o_G2 = put(G2);
    M.o_G3 = put(G3);
    std::vector<double> ha(kMaxE, 0.0), hb(kMaxE + 1, 0.0), h0(kMaxE, 0.0);
    for (int l = 0; l < kMaxE && l < (int)S.aR.alpha.size(); ++l) ha[l] = S.aR.alpha[l];
    for (int l = 0; l <= kMaxE && l < (int)S.aR.beta.size(); ++l) hb[l] = std::sqrt(S.aR.beta[l]);
    {
        double h[kMaxE + 2];
        h[0] = 1.0 / std::sqrt(S.aR.beta[0]);
        if (kMaxE > 1 && (int)S.aR.beta.size() > 1) h[1] = (0.0 - S.aR.alpha[0]) * h[0] / std::sqrt(S.aR.beta[1]);
        for (int l = 1; l + 1 < kMaxE && l + 1 < (int)S.aR.beta.size(); ++l)
            h[l + 1] = ((0.0 - S.aR.alpha[l]) * h[l] - std::sqrt(S.aR.beta[l]) * h[l - 1]) / std::sqrt(S.aR.beta[l + 1]);
        for (int l = 0; l < kMaxE && l <= QR; ++l) h0[l] = h[l];
    }
    M.o_ha = put(ha);
    M.o_hb = put(hb);
    M.o_h0 = put(h0);
}

// The tensor-core contraction's K^h table: per chunk of 32 values of a, the TF32 high part then the
// low part of K^h[n][a] (n < Npad = 2Q_R rounded up to 16; zero beyond 2Q_R) in the kernel's
// shared-memory layout, float (n / 8) * 256 + (a % 32 / 4) * 32 + (n % 8) * 4 + a % 4.
int kr_npad(int nR) { return (nR + 15) / 16 * 16; }
size_t kr_split_floats(int nR) {
    const int nk = ((nR + 7) / 8 * 8 + 31) / 32;
    return (size_t)nk * kr_npad(nR) * 64;
}
float tf32_round(float x) {
    // round to the 10-bit TF32 mantissa, ties away from zero (the rule of cvt.rna.tf32.f32)
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}
// The FP32 contraction's tables (kr_contract.cu): the weight-scaled Khat_ia = K^h_ia sqrt(w_a / w_i)
// in FP64 from the radial weights w, then [split table | isw[nR] | sw[nR] | Khat[nR][nR] (FP32)],
// isw = 1/sqrt(w) (zero beyond the float range: those populations are zero), sw = sqrt(w).
size_t kr_table_floats(int nR) { return kr_split_floats(nR) + 2 * (size_t)nR + (size_t)nR * nR; }
std::vector<double> kr_scaled(const std::vector<double>& tab, int o_KR, int o_wR, int nR) {
    std::vector<double> K((size_t)nR * nR);
    for (int i = 0; i < nR; ++i)
        for (int a = 0; a < nR; ++a)
            K[(size_t)i * nR + a] = tab[o_KR + (size_t)i * nR + a] * std::sqrt(tab[o_wR + a] / tab[o_wR + i]);
    return K;
}
std::vector<float> kr_split_table(const std::vector<double>& tab, int o_KR, int o_wR, int nR) {
    const int Npad = kr_npad(nR), nk = ((nR + 7) / 8 * 8 + 31) / 32;
    const std::vector<double> Kh = kr_scaled(tab, o_KR, o_wR, nR);
    std::vector<float> out(kr_table_floats(nR), 0.f);
    float* isw = out.data() + kr_split_floats(nR);
    float* sw = isw + nR;
    float* kplain = sw + nR;
    for (int a = 0; a < nR; ++a) {
        const double s = std::sqrt(tab[o_wR + a]);
        sw[a] = (float)s;
        isw[a] = 1.0 / s > 3.0e38 ? 0.f : (float)(1.0 / s);
    }
    for (size_t e = 0; e < Kh.size(); ++e) kplain[e] = (float)Kh[e];
    for (int kc = 0; kc < nk; ++kc) {
        float* hi = out.data() + (size_t)kc * Npad * 64;
        float* lo = hi + (size_t)Npad * 32;
        for (int n = 0; n < nR; ++n)
            for (int kk = 0; kk < 32; ++kk) {
                const int a = kc * 32 + kk;
                if (a >= nR) continue;
                const float k32 = (float)Kh[(size_t)n * nR + a];
                const float h = tf32_round(k32);
                const size_t off = (size_t)(n / 8) * 256 + (kk / 4) * 32 + (n % 8) * 4 + kk % 4;
                hi[off] = h;
                lo[off] = tf32_round(k32 - h);
            }
    }
    return out;
}

Layout make_layout(const Solver& S) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 1), kAlign);
        return o;
    };
    for (int b = 0; b < 3; ++b) L.f[b] = take(S.f_elems * S.tsize);
    for (int b = 0; b < 3; ++b) L.sums[b] = take((size_t)S.total_cells * S.n3 * kSums * sizeof(double));
    // double-float pairs of the sums for the FP32 closure
    for (int b = 0; b < 3; ++b) L.sumsw[b] = take(S.tsize == 4 ? (size_t)S.total_cells * S.n3 * kSums * 8 : 0);
    for (int b = 0; b < 3; ++b) L.dens[b] = take((size_t)S.total_cells * S.n3 * S.tsize);
    L.ca = take((size_t)S.total_cells * kCA * sizeof(double));
    L.mpk = take((size_t)S.total_cells * kNmom * sizeof(double));  // the moments query's rows
    L.bpairs = take((size_t)S.max_citems * sizeof(BandPair));   // the batch closure's band jobs
    L.k3f = take(S.geometry == FDLB_SPH ? S.f_elems * S.tsize : 0);  // sphere: K_3 f of the stage input
    L.n_bpairs = take(sizeof(int));
    L.cw = take((size_t)S.total_cells * 2 * S.tsize);
    L.rec = take((size_t)S.total_cells * record_stride(S.nR, S.n2, S.n3) * S.tsize);
    L.tab = take(S.tab_h.size() * sizeof(double));
    L.tabT = take(S.tab_h.size() * S.tsize);
    L.inst = take(S.n_inst * sizeof(InstDev));
    L.geo = take((size_t)S.total_cells * kGeo * sizeof(double));
    L.geoT = take((size_t)S.total_cells * kGeo * S.tsize);
    L.gw = take((size_t)S.n_inst * 2 * (S.nR + S.n2 + S.n3) * sizeof(double));
    L.gwT = take((size_t)S.n_inst * 2 * (S.nR + S.n2 + S.n3) * S.tsize);
    L.band = take(S.band_elems * S.tsize);
    L.band_lo = take((size_t)S.total_cells * 2 * sizeof(int));  // (first column, extent) per cell
    L.sitems = take((size_t)S.max_sitems * sizeof(int4));
    L.n_sitems = take(sizeof(int));
    L.citems = take((size_t)S.max_citems * sizeof(int4));
    L.n_citems = take(sizeof(int));
    L.nwp = take((size_t)S.n_inst * 2 * kWallParts * S.tsize);
    L.err = take(sizeof(int));
    L.gbar = take(64);  // grid barrier counter of the persistent step kernel
    L.rprev = take((size_t)S.total_cells * 4 * sizeof(double));
    L.rout = take((size_t)S.n_inst * 10 * sizeof(double));
    // K^h f of the stage input for the contraction kernel (large radial orders only)
    L.krf = take(S.nR >= kKrKernelMinNodes ? S.f_elems * S.tsize : 0);
    // K^h as TF32 pairs for the tensor-core contraction kernel (FP32 populations)
    L.krB = take(S.nR >= kKrKernelMinNodes && S.tsize == 4 ? kr_table_floats(S.nR) * sizeof(float) : 0);
    L.total = off;
    return L;
}

// Host-side plan of one handle: validation, quadrature, per-instance set-up, sizes.
int plan_solver(const fdlb_params* ps, int n, Solver& S) try {
    if (!ps || n < 1) return FDLB_EINVAL;
    const fdlb_params& p0 = ps[0];
    for (int q = 0; q < n; ++q) {
        const fdlb_params& p = ps[q];
        if (p.geometry != p0.geometry || p.Q_R != p0.Q_R || p.Q_2 != p0.Q_2 || p.Q_3 != p0.Q_3 ||
            p.precision != p0.precision || p.N_R != p0.N_R || p.N_2 != p0.N_2 || p.N_3 != p0.N_3)
            return FDLB_EINVAL;
    }
    int rc = validate_params([&] {
        fdlb_params t = p0;
        auto order = [](int N, int Q) { return N < 0 ? std::min(Q - 1, kMaxN) : N; };
        t.N_R = order(t.N_R, t.Q_R);
        t.N_2 = order(t.N_2, t.Q_2);
        t.N_3 = order(t.N_3, t.Q_3);
        return t;
    }());
    if (rc) return rc;
    S.n_inst = n;
    S.reduced = p0.geometry == FDLB_CYL_Z ? 1 : 0;
    S.geometry = S.reduced ? FDLB_CYL : p0.geometry;
    S.precision = p0.precision;
    S.tsize = p0.precision == FDLB_FP32 ? 4 : 8;
    S.aR = make_axis(p0.Q_R, true);
    S.a2 = make_axis(p0.Q_2, false);
    if (S.reduced) {
        // the pair (phi, chi) in the place of the p_z nodes: no p_z, unit weights (WENO then works on
        // phi / (w_R w_2) and chi / (w_R w_2))
        S.a3 = AxisRule();
        S.a3.Q = 2;
        S.a3.p = {0.0, 0.0};
        S.a3.w = {1.0, 1.0};
        S.a3.alpha = {0.0, 0.0, 0.0};
        S.a3.beta = {1.0, 1.0, 2.0};
    } else {
        S.a3 = make_axis(p0.Q_3, false);
    }
    S.nR = 2 * p0.Q_R;
    S.n2 = p0.Q_2;
    S.n3 = S.reduced ? 2 : p0.Q_3;
    S.Np = S.nR * S.n2 * S.n3;
    S.setup.resize(n);
    for (int q = 0; q < n; ++q) {
        rc = build_instance(ps[q], S.aR, S.setup[q]);
        if (rc) return rc;
    }
    S.NR = S.setup[0].NR;
    S.N2 = S.setup[0].N2;
    S.N3 = S.setup[0].N3;
    build_tables(S);
    S.f_off.resize(n);
    S.cell_off.resize(n);
    S.total_cells = 0;
    S.f_elems = 0;
    S.band_elems = 0;
    S.max_sitems = 0;
    S.max_citems = 0;
    const size_t falign = kAlign / S.tsize;
    // cell indices, work-item counts and the FM band offsets are 32-bit in the device tables:
    // a batch whose totals pass 2^31 - 1 (e.g. ~5000 instances of 1024 stretched cells, whose
    // bands hold ~4.3e5 entries each) is rejected here instead of wrapping
    const long long kIntMax = 2147483647LL;
    long long cells = 0, sitems = 0, citems = 0;
    for (int q = 0; q < n; ++q) {
        const int N = S.setup[q].p.n_cells;
        S.cell_off[q] = (int)cells;
        S.f_off[q] = (long long)S.f_elems;
        cells += N;
        S.f_elems += align_up((size_t)N * S.Np, falign);
        S.band_elems += (size_t)N * S.setup[q].band.width;
        sitems += (long long)(N / 2 + 1) * S.n3;  // tiles of at least two cells, at most n3 slices
        citems += (long long)N + 2 * kWallParts;  // room for one-cell closure items, + the wall items
        if (cells > kIntMax || sitems > kIntMax || citems > kIntMax || S.band_elems > (size_t)kIntMax)
            return FDLB_EINVAL;
    }
    S.total_cells = (int)cells;
    S.max_sitems = (int)sitems;
    S.max_citems = (int)citems;
    S.active.assign(n, 1);
    S.inst_steps.assign(n, 0);
    S.last_res.assign(n, -1.0);
    return FDLB_OK;
} FDLB_HOST_CATCH


// Wall Maxwellians per axis and the incoming-flux normaliser of the diffuse wall.
void wall_tables(const Solver& S, int q, double* out, double* den) {
    const InstanceSetup& I = S.setup[q];
    const int stride = S.nR + S.n2 + S.n3;
    for (int side = 0; side < 2; ++side) {
        double* o = out + side * stride;
        const double Tw = I.p.T_wall[side], uw = I.p.u_wall[side];
        g_half_host(S.aR, S.NR, 0.0, Tw, o);
        g_full_host(S.a2, S.N2, uw, Tw, o + S.nR);
        if (S.reduced) {
            // the wall's pair (int g_z, int p_z^2 g_z) = (1, T_w)
            o[S.nR + S.n2] = 1.0;
            o[S.nR + S.n2 + 1] = Tw;
        } else {
            g_full_host(S.a3, S.N3, 0.0, Tw, o + S.nR + S.n2);
        }
        double sR = 0.0, s2 = 0.0, s3 = 0.0;
        for (int i = 0; i < S.nR; ++i)
            if (side == 0 ? S.aR.p[i] > 0 : S.aR.p[i] < 0) sR += std::fabs(S.aR.p[i]) * o[i];
        for (int j = 0; j < S.n2; ++j) s2 += o[S.nR + j];
        for (int k = 0; k < (S.reduced ? 1 : S.n3); ++k) s3 += o[S.nR + S.n2 + k];  // mass: phi alone
        den[side] = sR * s2 * s3;
    }
}

void fill_inst(Solver& S, int q) {
    const InstanceSetup& I = S.setup[q];
    InstDev& d = S.inst_h[q];
    d.n_cells = I.p.n_cells;
    d.cell_off = S.cell_off[q];
    d.f_off = S.f_off[q];
    d.band_w = I.band.width;
    d.chi_local = I.p.chi_model == FDLB_CHI_SET_LOCAL ? 1 : 0;
    d.geometry = I.p.geometry == FDLB_SPH ? 1 : 0;
    d.sigma = I.sigma;
    d.bfac = 2.0 * kPiH / 3.0 * I.sigma * I.sigma * I.sigma;
    d.etafac = kPiH * I.sigma * I.sigma * I.sigma / 6.0;
    d.dt = I.dt;
    d.ds = I.grid.ds;
    std::vector<double> tmp(2 * (S.nR + S.n2 + S.n3));
    wall_tables(S, q, tmp.data(), d.nw_den);
    for (int side = 0; side < 2; ++side) {
        d.nw_iden[side] = 1.0 / d.nw_den[side];
        d.f_nw_iden[side] = (float)d.nw_iden[side];
    }
    d.f_sigma = (float)d.sigma;
    d.f_bfac = (float)d.bfac;
    d.f_etafac = (float)d.etafac;
    d.f_ids = (float)(1.0 / d.ds);
    d.f_dt = (float)d.dt;
}

// Work lists: stream items (instance, first cell, cells, slice) over the active instances,
// tiles of 3..B cells, largest instances first; closure items (instance, first cell, cells).
cudaError_t launch_step_dispatch(const Solver& S, const StepArgs* P, int* blocks_per_sm) {
    const int g = S.geometry;
    if (S.precision == FDLB_FP32)
        return g == FDLB_CYL ? launch_step_float_0(S.scfg, P, S.M, S.grid_step, S.threads, S.smem_step, S.stream, blocks_per_sm)
                             : launch_step_float_1(S.scfg, P, S.M, S.grid_step, S.threads, S.smem_step, S.stream, blocks_per_sm);
    return g == FDLB_CYL ? launch_step_double_0(S.scfg, P, S.M, S.grid_step, S.threads, S.smem_step, S.stream, blocks_per_sm)
                         : launch_step_double_1(S.scfg, P, S.M, S.grid_step, S.threads, S.smem_step, S.stream, blocks_per_sm);
}

// Whether the persistent step kernel runs the current configuration, and its launch shape: the
// compile-time shapes, one momentum slice, the bulk staging, tiles within the closure's reach,
// at least one warp beyond the closure's four, and a co-resident grid (every block owns the
// tiles it + k grid for the whole launch).
int plan_step_kernel(Solver& S, int n_items) {
    S.fused_on = 0;
    S.grid_step = 0;
    if (!S.fused || S.krg_on || S.k3_on || !S.scfg.spec || S.M.slices != 1 || !S.use_bulk || S.threads < 5 * 32 || S.max_tile < 1 ||
        S.max_tile > kClosureCells || n_items < 1)
        return FDLB_OK;
    // shared memory: the stage's plan, then [staged band rows | closure tables | band-union
    // densities]; static shared memory of the closure (< 16 KB) stays below the opt-in limit
    const size_t clo_off = (S.smem_stream + 15) / 16 * 16;
    const size_t base = clo_off + closure_smem(S.nR, S.n2, S.n3, S.max_union, 0, (int)S.tsize);
    const size_t limit = S.smem_optin > 16384 ? S.smem_optin - 16384 : 0;
    if (base > limit) return FDLB_OK;
    int wst = 0;
    for (int q = 0; q < S.n_inst; ++q)
        wst = std::max(wst, std::min(S.setup[q].p.n_cells, S.max_tile + 4) * S.setup[q].band.width);
    wst = (int)std::min<size_t>((size_t)wst, (limit - base) / S.tsize);
    S.step_wst = wst;
    S.step_clo_off = (int)clo_off;
    S.smem_step = clo_off + closure_smem(S.nR, S.n2, S.n3, S.max_union, wst, (int)S.tsize);
    int bps = 0;
    if (launch_step_dispatch(S, nullptr, &bps) != cudaSuccess || bps < 1) {
        cudaGetLastError();
        return FDLB_OK;
    }
    S.grid_step = std::min(n_items, bps * S.n_sm);
    S.fused_on = 1;
    return FDLB_OK;
}

int upload_items(Solver& S) {
    std::vector<int> order;
    for (int q = 0; q < S.n_inst; ++q)
        if (S.active[q]) order.push_back(q);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return S.setup[a].p.n_cells > S.setup[b].p.n_cells; });
    std::vector<int4> si, ci;
    const int slices = S.n3 / S.KS;
    for (int q : order) {
        const int N = S.setup[q].p.n_cells;
        int nt = (N + S.B - 1) / S.B;
        if (S.n_inst == 1 && S.n_sm > 0) {
            // one instance: a multiple of the SM count of tiles (one or more full waves; every
            // SM gets the same number of tiles), tile sizes differing by at most one cell, the
            // larger first, as long as tiles keep at least two cells
            const int per_wave = S.n_sm;
            const int r = (nt * slices + per_wave - 1) / per_wave * per_wave / slices;
            if (r >= nt && r * slices % per_wave == 0 && N / r >= 2) nt = r;
        }
        const int base = N / nt, rem = N % nt;
        int c0 = 0;
        for (int t = 0; t < nt; ++t) {
            const int cnt = base + (t < rem ? 1 : 0);
            for (int sl = 0; sl < slices; ++sl) si.push_back(make_int4(q, c0, cnt, sl));
            c0 += cnt;
        }
        // the wall densities first (their blocks read four cells of populations), then the cells
        for (int side = 0; side < 2; ++side)
            for (int part = 0; part < kWallParts; ++part) ci.push_back(make_int4(q, side ? N - 1 : 0, part, 1 + side));
        const int cc = S.closure_batch ? kClosureCells : S.closure_cells;
        for (int c = 0; c < N; c += cc) ci.push_back(make_int4(q, c, std::min(cc, N - c), 0));
    }
    if ((int)si.size() > S.max_sitems || (int)ci.size() > S.max_citems) return FDLB_EINVAL;
    // the batch closure's band jobs: two band rows of an item at a time (instances with chi at the
    // local density have none), or a wall part; geometry only, so formed here once per work list
    std::vector<BandPair> bp;
    if (S.closure_batch) {
        for (const int4& w : ci) {
            const InstanceSetup& I = S.setup[w.x];
            const InstDev& D = S.inst_h[w.x];
            if (w.w != 0) {
                bp.push_back(BandPair{0, 0, 0, 0, -w.w, w.z, 0, w.x});
                continue;
            }
            if (D.chi_local || I.band.width == 0) continue;
            const int N = I.p.n_cells;
            for (int t = 0; t < w.z; t += 2) {
                const int a = w.y + t, b = a + 1;
                const bool hasB = t + 1 < w.z;
                BandPair p{};
                p.wA = (long long)D.band_off + (long long)a * D.band_w;
                p.wB = p.wA + D.band_w;
                p.dA = (long long)D.cell_off + I.band.lo[a];
                p.dB = hasB ? (long long)D.cell_off + I.band.lo[b] : p.dA;
                p.kmaxA = std::min(I.band.cnt[a], N - I.band.lo[a]);
                p.kmaxB = hasB ? std::min(I.band.cnt[b], N - I.band.lo[b]) : 0;
                p.gc = D.cell_off + a;
                p.q = w.x;
                bp.push_back(p);
            }
        }
        if ((int)bp.size() > S.max_citems) return FDLB_EINVAL;
    }
    const int nbp = (int)bp.size();
    if (nbp) FDLB_CUDA(cudaMemcpyAsync(S.bpairs, bp.data(), nbp * sizeof(BandPair), cudaMemcpyHostToDevice, S.stream));
    FDLB_CUDA(cudaMemcpyAsync(S.n_bpairs, &nbp, sizeof(int), cudaMemcpyHostToDevice, S.stream));
    const int ns = (int)si.size(), nc = (int)ci.size();
    if (ns) FDLB_CUDA(cudaMemcpyAsync(S.sitems, si.data(), ns * sizeof(int4), cudaMemcpyHostToDevice, S.stream));
    if (nc) FDLB_CUDA(cudaMemcpyAsync(S.citems, ci.data(), nc * sizeof(int4), cudaMemcpyHostToDevice, S.stream));
    FDLB_CUDA(cudaMemcpyAsync(S.n_sitems, &ns, sizeof(int), cudaMemcpyHostToDevice, S.stream));
    FDLB_CUDA(cudaMemcpyAsync(S.n_citems, &nc, sizeof(int), cudaMemcpyHostToDevice, S.stream));
    FDLB_CUDA(cudaStreamSynchronize(S.stream));  // host vectors go out of scope
    // closure shared memory: the tables and the union of the FM bands of one item's reach (the
    // closure kernel's items and, for the persistent step kernel, the tiles)
    int max_union = 1;
    S.max_tile = 0;
    auto reach_union = [&](const int4& w) {
        const InstanceSetup& I = S.setup[w.x];
        if (I.band.width == 0) return;
        const int N = I.p.n_cells;
        const int h0 = std::max(0, std::min(w.y - 2, N - 5)), h1 = std::min(N, std::max(w.y + w.z + 2, 5));
        const int lo = I.band.lo[h0];
        const int hi = std::min(N - 1, I.band.lo[h1 - 1] + I.band.cnt[h1 - 1] - 1 + 3);
        max_union = std::max(max_union, hi - lo + 1);
    };
    for (const int4& w : ci)
        if (w.w == 0) reach_union(w);
    for (const int4& w : si) {
        reach_union(w);
        S.max_tile = std::max(S.max_tile, w.z);
    }
    S.max_union = max_union;
    // staged band rows of one item's reach (at most closure_cells + 4 rows); instances whose rows
    // do not fit read them from global memory instead
    int wst = 0;
    for (int q = 0; q < S.n_inst; ++q)
        wst = std::max(wst, std::min(S.setup[q].p.n_cells, S.closure_cells + 4) * S.setup[q].band.width);
    const size_t base = closure_smem(S.nR, S.n2, S.n3, max_union, 0, (int)S.tsize);
    if (base > S.smem_optin) return FDLB_EINVAL;
    wst = (int)std::min<size_t>((size_t)wst, (S.smem_optin - base) / S.tsize);
    // Many more items than co-resident blocks (batches, long instances): the closure is bound by
    // how many items are in flight, not by one item's latency, so each block keeps to the share of
    // an SM's shared memory that lets as many blocks reside as its registers allow; the band rows
    // of wider bands are then read from global memory (coalesced along the row) instead of being
    // staged.
    const bool throughput = nc > S.n_sm * 8;
    int closure_bps = 8;
    if (throughput && S.smem_per_sm > 0) {
        closure_bps = std::max(1, closure_blocks_per_sm((int)S.tsize, base));
        const size_t target = S.smem_per_sm / closure_bps;
        wst = target > base + 1024 ? (int)std::min<size_t>((size_t)wst, (target - base - 1024) / S.tsize) : 0;
    }
    S.closure_wst = wst;
    S.closure_smem = closure_smem(S.nR, S.n2, S.n3, max_union, wst, (int)S.tsize);
    S.grid_closure = std::max(1, std::min(nc, S.n_sm * (throughput ? closure_bps : 8)));
    // the batch form: the tables only, as many blocks as reside
    S.cbatch_smem = closure_smem(S.nR, S.n2, S.n3, 0, 0, (int)S.tsize);
    S.grid_cbatch = std::max(1, std::min(nc, S.n_sm * closure_batch_blocks_per_sm((int)S.tsize, S.cbatch_smem)));
    S.grid_stream = std::max(1, ns);
    return plan_step_kernel(S, ns);
}

int launch_moments_all(Solver& S, int buf);

int configure_tiling(Solver& S, int B, int KS, int threads) {
    const int old_slices = S.M.slices;
    if (B > 0) S.B = std::max(2, B);
    if (KS > 0) S.KS = KS;
    // the sphere's force couples every axis: slices narrower than the p_3 axis take K_3 f from its
    // own contraction kernel
    if (S.geometry == FDLB_SPH && !S.k3f) S.KS = S.n3;
    if (S.KS < 1 || S.n3 % S.KS) S.KS = S.n3;
    S.k3_on = S.geometry == FDLB_SPH && S.KS < S.n3 ? 1 : 0;
    if (S.geometry == FDLB_CYL) {
        // a block holds at most 512 threads of at most 8 momenta: narrower slices (p_3 is passive on
        // the cylinder) where a slice of the large radial orders would exceed that
        const int vw_max = S.tsize == 4 ? 8 : 8;
        while (S.KS > 1 && S.nR * S.n2 * S.KS > 512 * vw_max) {
            int k = S.KS - 1;
            while (k > 1 && S.n3 % k) --k;
            S.KS = k;
        }
    }
    const int Ms = S.nR * S.n2 * S.KS;
    S.M.nR = S.nR;
    S.M.n2 = S.n2;
    S.M.n3 = S.n3;
    S.M.Np = S.Np;
    S.M.NR = S.NR;
    S.M.N2 = S.N2;
    S.M.N3 = S.N3;
    S.M.KS = S.KS;
    S.M.slices = S.n3 / S.KS;
    S.M.Ms = Ms;
    S.M.reduced = S.reduced;
    // vectors of VW consecutive j momenta; compile-time shapes for the benchmark workloads
    StreamCfg cfg{};
    if (S.tsize == 4)
        cfg.vw = S.n2 % 4 == 0 ? 4 : (S.n2 % 2 == 0 ? 2 : 1);
    else
        cfg.vw = S.n2 % 2 == 0 ? 2 : 1;
    cfg.spec = ((S.geometry == FDLB_CYL && S.nR == 16 && S.n2 == 8 && S.n3 == 8) ||
                (S.geometry == FDLB_SPH && S.nR == 24 && S.n2 == 12 && S.n3 == 12)) &&
               cfg.vw == (S.tsize == 4 ? 4 : 2);
    const int cap = threads > 0 ? threads : 256;
    // the cylinder's FP32 shape in blocks of at most 128 threads: a thread per whole p_2 row (8
    // momenta; per-vector and per-cell work spread over twice the momenta, half the warps per cell)
    if (cfg.spec && S.tsize == 4 && S.geometry == FDLB_CYL && cap <= 128 && Ms / 8 <= 128) cfg.vw = 8;
    const int Vs = Ms / cfg.vw;
    int nt = 0;
    if (cfg.vw == 8) {
        cfg.nv = 1;
        nt = (Vs + 31) / 32 * 32;
    } else if (cfg.spec) {
        // vectors per thread fixed by the instantiation: the smaller count whose block fits the cap
        const int na = S.geometry == FDLB_CYL ? 1 : 2, nb = 2 * na;
        cfg.nv = ((Vs + na - 1) / na + 31) / 32 * 32 <= std::max(cap, 32) ? na : nb;
        nt = ((Vs + cfg.nv - 1) / cfg.nv + 31) / 32 * 32;
    } else {
        cfg.nv = cfg.vw == 4 ? 2 : 4;  // the most a thread holds; fewer when the block has room
        nt = (std::min(Vs, cap) + 31) / 32 * 32;
        if ((long long)nt * cfg.nv < Vs) nt = ((Vs + cfg.nv - 1) / cfg.nv + 31) / 32 * 32;
    }
    if (nt > 512 || (long long)nt * cfg.nv < Vs) return FDLB_EINVAL;
    if (cfg.vw == 8)
        cfg.minb = (S.stage_minb == 2 || S.stage_minb == 3 || S.stage_minb == 5) ? S.stage_minb : 1;
    else
        cfg.minb = (S.stage_minb == 3 && cfg.spec && S.tsize == 4 && S.geometry == FDLB_CYL && nt <= 256) ? 3 : 1;
    S.scfg = cfg;
    S.threads = nt;
    S.mma_on = S.tensor && cfg.spec && cfg.vw == 4 && S.tsize == 4 && S.nR % 8 == 0 && !S.krg_on;
    // shrink the tile until it fits in shared memory
    for (;;) {
        StreamSmem P = stream_smem_plan(S.B, Ms, S.nR, S.n2, S.n3, nt / 32, (int)S.tsize, S.mma_on ? 1 : 0,
                                        S.krg_on ? 1 : 0);
        if ((size_t)P.total <= S.smem_optin || S.B <= 2) {
            S.smem_stream = P.total;
            break;
        }
        S.B = std::max(2, S.B / 2);
    }
    if (S.smem_stream > S.smem_optin) return FDLB_EINVAL;
    S.use_bulk = ((size_t)Ms * S.tsize % 16 == 0 && (size_t)S.Np * S.tsize % 16 == 0) ? 1 : 0;
    if (S.gexec) {
        cudaGraphExecDestroy(S.gexec);
        S.gexec = nullptr;
    }
    int rc = upload_items(S);
    if (rc) return rc;
    // the partial sums are stored per slice: rebuild them for a new slice count (under the same
    // slicing they stay as the last stage wrote them, so a new tile size or block size leaves the
    // state and its sums bit for bit as they were)
    if (S.M.slices != old_slices) return launch_moments_all(S, 0);
    return FDLB_OK;
}

template <typename T>
void to_device_layout(const Solver& S, const double* src, std::vector<T>& dst, int N) {
    // ABI [cell][i][j][k] -> device [cell][k][i][j]
    dst.resize((size_t)N * S.Np);
    for (int c = 0; c < N; ++c)
        for (int i = 0; i < S.nR; ++i)
            for (int j = 0; j < S.n2; ++j)
                for (int k = 0; k < S.n3; ++k)
                    dst[(size_t)c * S.Np + ((size_t)k * S.nR + i) * S.n2 + j] =
                        (T)src[(size_t)c * S.Np + ((size_t)i * S.n2 + j) * S.n3 + k];
}

template <typename T>
void from_device_layout(const Solver& S, const std::vector<T>& src, double* dst, int N) {
    for (int c = 0; c < N; ++c)
        for (int i = 0; i < S.nR; ++i)
            for (int j = 0; j < S.n2; ++j)
                for (int k = 0; k < S.n3; ++k)
                    dst[(size_t)c * S.Np + ((size_t)i * S.n2 + j) * S.n3 + k] =
                        (double)src[(size_t)c * S.Np + ((size_t)k * S.nR + i) * S.n2 + j];
}

int launch_moments_all(Solver& S, int buf) {
    // a warp per cell, every cell of the state
    const long long blocks = ((long long)S.total_cells + 7) / 8;
    const int grid = (int)std::max<long long>(1, std::min<long long>(blocks, (long long)S.n_sm * 8));
    if (S.precision == FDLB_FP32) {
        // the FP64 sums and the double-float pairs the FP32 closure reads
        launch_moments<float>((const float*)S.f[buf], S.sums[buf], (float*)S.dens[buf], S.sumsw[buf], S.total_cells,
                              grid, S.tab, S.M, S.stream);
    } else {
        launch_moments<double>((const double*)S.f[buf], S.sums[buf], (double*)S.dens[buf], nullptr, S.total_cells, grid,
                               S.tab, S.M, S.stream);
    }
    S.launches++;
    return cuda_status(cudaGetLastError());
}

int launch_closure_buf(Solver& S, int buf, int write_ca) {
    ClosureArgs A{};
    A.sums = S.sums[buf];
    A.sumsw = S.sumsw[buf];
    A.dens = S.dens[buf];
    A.f_in = S.f[buf];
    A.cw = S.cw;
    A.rec = S.rec;
    A.rec_stride = record_stride(S.nR, S.n2, S.n3);
    A.nwp = S.nwp;
    A.items = S.citems;
    A.n_items = S.n_citems;
    A.inst = S.inst_d;
    A.band = S.band;
    A.band_lo = S.band_lo;
    A.tabT = S.tabT;
    A.geoT = S.geoT;
    A.slices = S.M.slices;
    A.max_union = S.max_union;
    A.wall_parts = kWallParts;
    A.wst_elems = S.closure_wst;
    A.err = S.err;
    A.programmatic = S.programmatic;
    A.pairs = S.bpairs;
    A.n_pairs = S.n_bpairs;
    if (S.closure_batch) {
        if (S.precision == FDLB_FP32)
            launch_closure_batch<float>(A, S.M, S.grid_cbatch, S.cbatch_smem, S.stream);
        else
            launch_closure_batch<double>(A, S.M, S.grid_cbatch, S.cbatch_smem, S.stream);
        S.launches += 2;
    } else {
        if (S.precision == FDLB_FP32)
            launch_closure<float>(A, S.M, S.grid_closure, S.closure_threads, S.closure_smem, S.stream);
        else
            launch_closure<double>(A, S.M, S.grid_closure, S.closure_threads, S.closure_smem, S.stream);
        S.launches++;
    }
    if (write_ca) {
        // the FP64 closure record for the queries (not part of the stage)
        if (S.precision == FDLB_FP32)
            launch_ca<float>(S.sums[buf], S.cw, S.ca, S.M.slices, S.total_cells, S.stream);
        else
            launch_ca<double>(S.sums[buf], S.cw, S.ca, S.M.slices, S.total_cells, S.stream);
        S.launches++;
    }
    return cuda_status(cudaGetLastError());
}

int launch_stream_only(Solver& S, int in, int fn, int out, double a, double b, int mode);

// K^h f of buffer `in` by the contraction kernel (large radial orders).
int launch_kr_buf(Solver& S, int in) {
    const int grid = std::max(1, std::min(S.grid_stream, S.n_sm * 8));
    cudaError_t e;
    const float* isw = S.krB ? S.krB + kr_split_floats(S.nR) : nullptr;
    const float* sw = isw ? isw + S.nR : nullptr;
    if (S.kr_tc)
        e = launch_kr_contract_tc((const float*)S.f[in], (float*)S.krf, S.sitems, S.n_sitems, S.inst_d, S.krB, isw, sw,
                                  S.M, kr_npad(S.nR), S.err, std::max(1, std::min(S.grid_stream, S.n_sm)), S.stream);
    else if (S.precision == FDLB_FP32)  // the weight-scaled form, as the tensor-core kernel
        e = launch_kr_contract<float>((const float*)S.f[in], (float*)S.krf, S.sitems, S.n_sitems, S.inst_d, sw + S.nR,
                                      isw, sw, S.M, grid, S.stream);
    else
        e = launch_kr_contract<double>((const double*)S.f[in], (double*)S.krf, S.sitems, S.n_sitems, S.inst_d,
                                       (const double*)S.tabT + S.M.o_KR, nullptr, nullptr, S.M, grid, S.stream);
    S.launches++;
    return cuda_status(e);
}

// Sphere with momenta sliced along p_3: K_3 f of buffer `in` by its contraction kernel.
int launch_k3_buf(Solver& S, int in) {
    const int grid = std::max(1, std::min(S.grid_stream, S.n_sm * 8));
    cudaError_t e;
    if (S.precision == FDLB_FP32)
        e = launch_k3_contract<float>((const float*)S.f[in], (float*)S.k3f, S.sitems, S.n_sitems, S.inst_d,
                                      (const float*)S.tabT + S.M.o_K3, S.M, grid, S.stream);
    else
        e = launch_k3_contract<double>((const double*)S.f[in], (double*)S.k3f, S.sitems, S.n_sitems, S.inst_d,
                                       (const double*)S.tabT + S.M.o_K3, S.M, grid, S.stream);
    S.launches++;
    return cuda_status(e);
}

// One right-hand-side evaluation and RK combination: closure launch, then the fused stage.
// In timing mode each launch is bracketed by events and its duration accumulated.
int launch_stage(Solver& S, int in, int fn, int out, double a, double b, int mode, int write_ca = 0) {
    if (S.krg_on) {
        const int rc = launch_kr_buf(S, in);
        if (rc) return rc;
    }
    if (S.k3_on) {
        const int rc = launch_k3_buf(S, in);
        if (rc) return rc;
    }
    if (S.timing) {
        FDLB_CUDA(cudaEventRecord(S.tev[0], S.stream));
        int rc = launch_closure_buf(S, in, write_ca);
        if (rc) return rc;
        FDLB_CUDA(cudaEventRecord(S.tev[1], S.stream));
        rc = launch_stream_only(S, in, fn, out, a, b, mode);
        if (rc) return rc;
        FDLB_CUDA(cudaEventRecord(S.tev[2], S.stream));
        FDLB_CUDA(cudaEventSynchronize(S.tev[2]));
        float m1 = 0.f, m2 = 0.f;
        FDLB_CUDA(cudaEventElapsedTime(&m1, S.tev[0], S.tev[1]));
        FDLB_CUDA(cudaEventElapsedTime(&m2, S.tev[1], S.tev[2]));
        S.t_closure_ms += m1;
        S.t_stream_ms += m2;
        S.n_closure_t++;
        S.n_stream_t++;
        return FDLB_OK;
    }
    int rc = launch_closure_buf(S, in, write_ca);
    if (rc) return rc;
    return launch_stream_only(S, in, fn, out, a, b, mode);
}

int launch_stream_only(Solver& S, int in, int fn, int out, double a, double b, int mode) {
    StageArgs A{};
    A.f_in = S.f[in];
    A.f_n = S.f[fn];
    A.f_out = S.f[out];
    A.rec = S.rec;
    A.rec_stride = record_stride(S.nR, S.n2, S.n3);
    A.nwp = S.nwp;
    A.wall_parts = kWallParts;
    A.sums_out = S.sums[out];
    A.sumsw_out = S.sumsw[out];
    A.dens_out = S.dens[out];
    A.items = S.sitems;
    A.n_items = S.n_sitems;
    A.inst = S.inst_d;
    A.tab = S.tab;
    A.tabT = S.tabT;
    A.geoT = S.geoT;
    A.gwT = S.gwT;
    A.err = S.err;
    A.a = a;
    A.b = b;
    A.fa = (float)a;
    A.fb = (float)b;
    A.mode = mode;
    A.B = S.B;
    A.use_bulk = S.use_bulk;
    A.programmatic = S.programmatic;
    A.mma = S.mma_on;
    A.tx_extra = S.test_tx_extra;
    A.krf = S.krg_on ? S.krf : nullptr;
    A.k3f = S.k3_on ? S.k3f : nullptr;
    cudaError_t e;
    const int g = S.geometry;
    if (S.precision == FDLB_FP32)
        e = g == FDLB_CYL ? launch_stream_float_0(S.scfg, A, S.M, S.grid_stream, S.threads, S.smem_stream, S.stream)
                          : launch_stream_float_1(S.scfg, A, S.M, S.grid_stream, S.threads, S.smem_stream, S.stream);
    else
        e = g == FDLB_CYL ? launch_stream_double_0(S.scfg, A, S.M, S.grid_stream, S.threads, S.smem_stream, S.stream)
                          : launch_stream_double_1(S.scfg, A, S.M, S.grid_stream, S.threads, S.smem_stream, S.stream);
    S.launches++;
    return cuda_status(e);
}

// One SSP-RK3 step (Sec. III): f1 = f + dt L(f); f2 = 3/4 f + 1/4 (f1 + dt L(f1));
// f^{n+1} = 1/3 f + 2/3 (f2 + dt L(f2)).  Buffers: 0 = f^n (and f^{n+1}), 1 = f1, 2 = f2.
int launch_step(Solver& S) {
    int rc = launch_stage(S, 0, 0, 1, 0.0, 1.0, 0);
    if (!rc) rc = launch_stage(S, 1, 0, 2, 0.75, 0.25, 0);
    if (!rc) rc = launch_stage(S, 2, 0, 0, 1.0 / 3.0, 2.0 / 3.0, 0);
    return rc;
}

int upload_state(Solver& S, int q, const double* f_host) {
    const int N = S.setup[q].p.n_cells;
    if (S.precision == FDLB_FP32) {
        std::vector<float> t;
        to_device_layout(S, f_host, t, N);
        FDLB_CUDA(cudaMemcpyAsync((float*)S.f[0] + S.f_off[q], t.data(), t.size() * 4, cudaMemcpyHostToDevice, S.stream));
        FDLB_CUDA(cudaStreamSynchronize(S.stream));
    } else {
        std::vector<double> t;
        to_device_layout(S, f_host, t, N);
        FDLB_CUDA(cudaMemcpyAsync((double*)S.f[0] + S.f_off[q], t.data(), t.size() * 8, cudaMemcpyHostToDevice, S.stream));
        FDLB_CUDA(cudaStreamSynchronize(S.stream));
    }
    S.inst_steps[q] = 0;
    S.prev_valid = false;
    return launch_moments_all(S, 0);
}

int download_buf(Solver& S, int q, int buf, double* out) {
    const int N = S.setup[q].p.n_cells;
    if (S.precision == FDLB_FP32) {
        std::vector<float> t((size_t)N * S.Np);
        FDLB_CUDA(cudaMemcpyAsync(t.data(), (const float*)S.f[buf] + S.f_off[q], t.size() * 4, cudaMemcpyDeviceToHost,
                                  S.stream));
        FDLB_CUDA(cudaStreamSynchronize(S.stream));
        from_device_layout(S, t, out, N);
    } else {
        std::vector<double> t((size_t)N * S.Np);
        FDLB_CUDA(cudaMemcpyAsync(t.data(), (const double*)S.f[buf] + S.f_off[q], t.size() * 8, cudaMemcpyDeviceToHost,
                                  S.stream));
        FDLB_CUDA(cudaStreamSynchronize(S.stream));
        from_device_layout(S, t, out, N);
    }
    return FDLB_OK;
}

// Host evaluation of the uniform equilibrium or the Shakhov-type seed of one instance.
void seed_state(const Solver& S, int q, const std::vector<double>& n, const std::vector<double>& u2,
                const std::vector<double>& T, const std::vector<double>& qR, std::vector<double>& f) {
    const int N = S.setup[q].p.n_cells;
    f.assign((size_t)N * S.Np, 0.0);
    std::vector<double> gR(S.nR), g2(S.n2), g3(S.n3);
    for (int c = 0; c < N; ++c) {
        g_half_host(S.aR, S.NR, 0.0, T[c], gR.data());
        g_full_host(S.a2, S.N2, u2[c], T[c], g2.data());
        if (S.reduced) {
            // the p_z-integrals of the seed against 1 (phi) and p_z^2 (chi): xi^2 carries p_z^2 as
            // T or 3T, and chi's part is weighted by T
            for (int i = 0; i < S.nR; ++i)
                for (int j = 0; j < S.n2; ++j) {
                    const double pR = S.aR.p[i], x1 = S.a2.p[j] - u2[c];
                    const double xs = pR * pR + x1 * x1, qf = pR * qR[c] / (n[c] * T[c] * T[c]);
                    const double base = n[c] * gR[i] * g2[j];
                    const size_t o = (size_t)c * S.Np + ((size_t)i * S.n2 + j) * S.n3;
                    f[o] = base * (1.0 + ((xs + T[c]) / (5.0 * T[c]) - 1.0) * qf);
                    f[o + 1] = T[c] * base * (1.0 + ((xs + 3.0 * T[c]) / (5.0 * T[c]) - 1.0) * qf);
                }
            continue;
        }
        g_full_host(S.a3, S.N3, 0.0, T[c], g3.data());
        for (int i = 0; i < S.nR; ++i)
            for (int j = 0; j < S.n2; ++j)
                for (int k = 0; k < S.n3; ++k) {
                    const double pR = S.aR.p[i], x1 = S.a2.p[j] - u2[c], x2 = S.a3.p[k];
                    const double xs = pR * pR + x1 * x1 + x2 * x2;
                    const double fac = 1.0 + (xs / (5.0 * T[c]) - 1.0) * pR * qR[c] / (n[c] * T[c] * T[c]);
                    f[(size_t)c * S.Np + ((size_t)i * S.n2 + j) * S.n3 + k] = n[c] * gR[i] * g2[j] * g3[k] * fac;
                }
    }
}

int ensure_graph(Solver& S) {
    if (S.gexec) return FDLB_OK;
    cudaGraph_t graph = nullptr;
    const int64_t before = S.launches;
    FDLB_CUDA(cudaStreamBeginCapture(S.stream, cudaStreamCaptureModeThreadLocal));
    int rc = FDLB_OK;
    for (int s = 0; s < S.graph_steps && !rc; ++s) rc = launch_step(S);
    cudaError_t e = cudaStreamEndCapture(S.stream, &graph);
    S.launches = before;
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    FDLB_CUDA(e);
    e = cudaGraphInstantiate(&S.gexec, graph, 0);
    cudaGraphDestroy(graph);
    return cuda_status(e);
}

// n whole steps in one launch of the persistent step kernel (barrier counter cleared first).
int launch_steps_fused(Solver& S, int64_t n) {
    StepArgs P{};
    StageArgs& A = P.st;
    A.rec = S.rec;
    A.rec_stride = record_stride(S.nR, S.n2, S.n3);
    A.nwp = S.nwp;
    A.wall_parts = kWallParts;
    A.items = S.sitems;
    A.n_items = S.n_sitems;
    A.inst = S.inst_d;
    A.tab = S.tab;
    A.tabT = S.tabT;
    A.geoT = S.geoT;
    A.gwT = S.gwT;
    A.err = S.err;
    A.mode = 0;
    A.B = S.B;
    A.use_bulk = S.use_bulk;
    A.mma = S.mma_on;
    ClosureArgs& C = P.cl;
    C.cw = S.cw;
    C.rec = S.rec;
    C.rec_stride = A.rec_stride;
    C.nwp = S.nwp;
    C.items = S.sitems;
    C.n_items = S.n_sitems;
    C.inst = S.inst_d;
    C.band = S.band;
    C.band_lo = S.band_lo;
    C.tabT = S.tabT;
    C.geoT = S.geoT;
    C.slices = S.M.slices;
    C.max_union = S.max_union;
    C.wall_parts = kWallParts;
    C.wst_elems = S.step_wst;
    C.err = S.err;
    for (int b = 0; b < 3; ++b) {
        P.f[b] = S.f[b];
        P.sums[b] = S.sums[b];
        P.sumsw[b] = S.sumsw[b];
        P.dens[b] = S.dens[b];
    }
    P.bar = S.gbar;
    P.n_steps = (int)n;
    P.clo_off = S.step_clo_off;
    P.bar_extra = S.test_bar_extra;
    A.tx_extra = S.test_tx_extra;
    FDLB_CUDA(cudaMemsetAsync(S.gbar, 0, sizeof(unsigned), S.stream));
    S.launches++;
    if (!S.timing) return cuda_status(launch_step_dispatch(S, &P, nullptr));
    FDLB_CUDA(cudaEventRecord(S.tev[0], S.stream));
    const int rc = cuda_status(launch_step_dispatch(S, &P, nullptr));
    if (rc) return rc;
    FDLB_CUDA(cudaEventRecord(S.tev[1], S.stream));
    FDLB_CUDA(cudaEventSynchronize(S.tev[1]));
    float m = 0.f;
    FDLB_CUDA(cudaEventElapsedTime(&m, S.tev[0], S.tev[1]));
    S.t_step_ms += m;
    S.n_step_t++;
    S.n_step_steps += n;
    return FDLB_OK;
}

// ------------------------------------------------------------------ autotuner
// Tile shapes chosen by timing: cells per stream tile B and own cells per closure item, the two
// knobs that regroup cells without changing any cell's arithmetic (the per-cell results and the
// order of every sum stay those of the default, so tuning changes no result bit); the block size
// and the momentum slicing, which do reorder the sums, stay as configured.  Each candidate is
// timed over three stages (closure + fused stage, the second RK stage's form, written to the
// stage-1 buffers, which every step overwrites before reading) after one warm-up stage; B is
// tuned first at the current closure grouping, then the closure grouping at the best B.  The
// choice is cached per process for the momentum set, precision, block size, slicing and the
// size class of the handle (log2 of its cells and of its instances).
struct TuneKey {
    int geometry, precision, nR, n2, n3, KS, threads, cells_log2, inst_log2;
    bool operator<(const TuneKey& o) const {
        const int a[9] = {geometry, precision, nR, n2, n3, KS, threads, cells_log2, inst_log2};
        const int b[9] = {o.geometry, o.precision, o.nR, o.n2, o.n3, o.KS, o.threads, o.cells_log2, o.inst_log2};
        return std::lexicographical_compare(a, a + 9, b, b + 9);
    }
};
struct TuneVal {
    int B, closure_cells, minb, batch;
};
std::map<TuneKey, TuneVal> g_tune_cache;
std::mutex g_tune_mutex;

int ilog2(long long x) {
    int r = 0;
    while (x > 1) {
        x >>= 1;
        ++r;
    }
    return r;
}

TuneKey tune_key(const Solver& S) {
    return TuneKey{S.geometry, S.precision, S.nR, S.n2, S.n3, S.KS, S.threads, ilog2(S.total_cells), ilog2(S.n_inst)};
}

int set_closure_grouping(Solver& S, int cells, int batch = -1) {
    S.closure_cells = cells;
    if (batch >= 0) S.closure_batch = batch;
    if (S.gexec) {
        cudaGraphExecDestroy(S.gexec);
        S.gexec = nullptr;
    }
    return upload_items(S);
}

// Time of three stages of the current tiling (ms), or a negative value if a launch failed.
float time_stages(Solver& S, cudaEvent_t e0, cudaEvent_t e1) {
    if (launch_stage(S, 0, 0, 1, 0.75, 0.25, 0) != FDLB_OK) return -1.f;
    cudaEventRecord(e0, S.stream);
    for (int r = 0; r < 3; ++r)
        if (launch_stage(S, 0, 0, 1, 0.75, 0.25, 0) != FDLB_OK) return -1.f;
    cudaEventRecord(e1, S.stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

int run_autotune(Solver& S, bool use_cache) {
    S.tuned = true;
    const TuneKey key = tune_key(S);
    if (use_cache) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            S.stage_minb = it->second.minb;
            int rc = configure_tiling(S, it->second.B, S.KS, S.threads);
            return rc ? rc : set_closure_grouping(S, it->second.closure_cells, it->second.batch);
        }
    }
    const bool timing = S.timing;
    S.timing = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FDLB_CUDA(cudaEventCreate(&e0));
    FDLB_CUDA(cudaEventCreate(&e1));
    const int KS = S.KS, threads = S.threads;
    int bestB = S.B, bestC = S.closure_cells, bestM = S.stage_minb, bestBatch = S.closure_batch;
    float best = time_stages(S, e0, e1);
    if (best < 0.f) best = 1e30f;
    const int Bs[] = {2, 3, 4, 6, 8, 12, 16, 24, 32};
    // the register bound of the stage kernel: three blocks per SM where that variant is built, and
    // for the row kernel also two and five
    const bool minb_choice = S.scfg.spec && S.tsize == 4 && S.geometry == FDLB_CYL && S.threads <= 256;
    const bool rows = S.scfg.vw == 8;
    int rc = FDLB_OK;
    for (int mb : {1, 3, 2, 5}) {
        if (mb == 3 && !minb_choice) continue;
        if ((mb == 2 || mb == 5) && !rows) continue;
        S.stage_minb = mb;
        for (int B : Bs) {
            if (B == bestB && mb == bestM) continue;
            if (configure_tiling(S, B, KS, threads) != FDLB_OK || S.B != B) continue;
            const float ms = time_stages(S, e0, e1);
            if (ms >= 0.f && ms < best) {
                best = ms;
                bestB = B;
                bestM = mb;
            }
        }
    }
    S.stage_minb = bestM;
    rc = configure_tiling(S, bestB, KS, threads);
    // the closure: the chain form with items of C cells, or the batch form (two launches)
    const int Cs[] = {2, 4, 8, 16};
    for (int C : Cs) {
        if (rc || (C == bestC && !bestBatch)) continue;
        if (set_closure_grouping(S, C, 0) != FDLB_OK) continue;
        const float ms = time_stages(S, e0, e1);
        if (ms >= 0.f && ms < best) {
            best = ms;
            bestC = C;
            bestBatch = 0;
        }
    }
    if (!rc && !bestBatch && set_closure_grouping(S, bestC, 1) == FDLB_OK) {
        const float ms = time_stages(S, e0, e1);
        if (ms >= 0.f && ms < best) {
            best = ms;
            bestBatch = 1;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    S.timing = timing;
    if (!rc) rc = set_closure_grouping(S, bestC, bestBatch);
    if (!rc) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = {bestB, bestC, bestM, bestBatch};
    }
    return rc;
}

int maybe_autotune(Solver& S) {
    if (S.tuned || S.autotune_mode == 0 || (S.autotune_mode == 1 && S.n_inst < 2)) return FDLB_OK;
    return run_autotune(S, true);
}

int do_steps(Solver& S, int64_t n) {
    if (n > 0) {
        const int rc = maybe_autotune(S);
        if (rc) return rc;
    }
    const int64_t before = S.launches;
    int64_t done = 0;
    if (S.fused_on) {
        constexpr int64_t kMaxStepsPerLaunch = 1 << 12;
        while (done < n) {
            const int64_t k = std::min(n - done, kMaxStepsPerLaunch);
            const int rc = launch_steps_fused(S, k);
            if (rc) return rc;
            done += k;
        }
    }
    if (n >= S.graph_steps && !S.timing) {
        int rc = ensure_graph(S);
        if (rc) return rc;
        while (n - done >= S.graph_steps) {
            FDLB_CUDA(cudaGraphLaunch(S.gexec, S.stream));
            S.launches += (int64_t)S.graph_steps * 3 * ((S.krg_on ? 1 : 0) + (S.k3_on ? 1 : 0) + (S.closure_batch ? 2 : 1) + 1);
            done += S.graph_steps;
        }
    }
    for (; done < n; ++done) {
        int rc = launch_step(S);
        if (rc) return rc;
    }
    for (int q = 0; q < S.n_inst; ++q)
        if (S.active[q]) S.inst_steps[q] += n;
    S.last_launches = S.launches - before;
    return FDLB_OK;
}

int solver_create(const fdlb_params* ps, int n, void* stream, void* workspace, size_t ws_bytes, fdlb_handle* out) {
    if (!out) return FDLB_EINVAL;
    *out = nullptr;
    auto S = std::make_unique<Solver>();
    int rc = plan_solver(ps, n, *S);
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return FDLB_ENOGPU;
    FDLB_CUDA(cudaGetDevice(&S->device));
    FDLB_CUDA(cudaDeviceGetAttribute(&S->n_sm, cudaDevAttrMultiProcessorCount, S->device));
    int optin = 0;
    FDLB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, S->device));
    S->smem_optin = (size_t)optin;
    int per_sm = 0;
    FDLB_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, S->device));
    S->smem_per_sm = (size_t)per_sm;
    S->stream = (cudaStream_t)stream;
    if (!S->stream) {
        // the legacy default stream cannot be captured into a graph: use a private blocking
        // stream (it still orders itself with the legacy stream)
        FDLB_CUDA(cudaStreamCreate(&S->stream));
        S->own_stream = true;
    }
    S->lay = make_layout(*S);
    if (workspace) {
        if (ws_bytes < S->lay.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return FDLB_ENOMEM;
        S->ws = (unsigned char*)workspace;
    } else {
        FDLB_CUDA(cudaMalloc(&S->ws, S->lay.total));
        S->own_ws = true;
    }
    Solver& R = *S;
    const Layout& L = R.lay;
    for (int b = 0; b < 3; ++b) {
        R.f[b] = R.ws + L.f[b];
        R.sums[b] = (double*)(R.ws + L.sums[b]);
        R.sumsw[b] = (void*)(R.ws + L.sumsw[b]);
        R.dens[b] = (void*)(R.ws + L.dens[b]);
    }
    R.ca = (double*)(R.ws + L.ca);
    R.mpk = (double*)(R.ws + L.mpk);
    R.bpairs = (BandPair*)(R.ws + L.bpairs);
    R.k3f = R.geometry == FDLB_SPH ? (void*)(R.ws + L.k3f) : nullptr;
    R.n_bpairs = (int*)(R.ws + L.n_bpairs);
    R.rec = R.ws + L.rec;
    R.tabT = R.ws + L.tabT;
    R.tab = (double*)(R.ws + L.tab);
    R.inst_d = (InstDev*)(R.ws + L.inst);
    R.geo = (double*)(R.ws + L.geo);
    R.gw = (double*)(R.ws + L.gw);
    R.band = R.ws + L.band;
    R.band_lo = (int*)(R.ws + L.band_lo);
    R.sitems = (int4*)(R.ws + L.sitems);
    R.n_sitems = (int*)(R.ws + L.n_sitems);
    R.citems = (int4*)(R.ws + L.citems);
    R.n_citems = (int*)(R.ws + L.n_citems);
    R.nwp = (void*)(R.ws + L.nwp);
    R.cw = (void*)(R.ws + L.cw);
    R.geoT = (void*)(R.ws + L.geoT);
    R.gwT = (void*)(R.ws + L.gwT);
    R.err = (int*)(R.ws + L.err);
    R.gbar = (unsigned*)(R.ws + L.gbar);
    R.rprev = (double*)(R.ws + L.rprev);
    R.rout = (double*)(R.ws + L.rout);
    R.krf = R.nR >= kKrKernelMinNodes ? (void*)(R.ws + L.krf) : nullptr;
    R.krg_on = R.krf != nullptr;
    FDLB_CUDA(cudaMemsetAsync(R.ws, 0, L.total, R.stream));
    if (R.krg_on && R.precision == FDLB_FP32) {
        // K^h as TF32 pairs for the tensor-core contraction (after the workspace is cleared)
        R.krB = (float*)(R.ws + L.krB);
        const std::vector<float> kb = kr_split_table(R.tab_h, R.M.o_KR, R.M.o_wR, R.nR);
        FDLB_CUDA(cudaMemcpyAsync(R.krB, kb.data(), kb.size() * sizeof(float), cudaMemcpyHostToDevice, R.stream));
        FDLB_CUDA(cudaStreamSynchronize(R.stream));
        R.tensor = 1;  // the tensor-core contraction by default
        R.kr_tc = 1;
    }
    // tables, instances, geometry, walls, FM band
    FDLB_CUDA(cudaMemcpyAsync(R.tab, R.tab_h.data(), R.tab_h.size() * 8, cudaMemcpyHostToDevice, R.stream));
    std::vector<float> tabf(R.tab_h.begin(), R.tab_h.end());
    if (R.precision == FDLB_FP32)
        FDLB_CUDA(cudaMemcpyAsync(R.tabT, tabf.data(), tabf.size() * 4, cudaMemcpyHostToDevice, R.stream));
    else
        FDLB_CUDA(cudaMemcpyAsync(R.tabT, R.tab_h.data(), R.tab_h.size() * 8, cudaMemcpyHostToDevice, R.stream));
    R.inst_h.resize(n);
    std::vector<double> geo((size_t)R.total_cells * kGeo), gw((size_t)n * 2 * (R.nR + R.n2 + R.n3));
    std::vector<int> blo((size_t)R.total_cells * 2, 0);
    size_t boff = 0;
    for (int q = 0; q < n; ++q) {
        fill_inst(R, q);
        R.inst_h[q].band_off = (int)boff;
        const InstanceSetup& I = R.setup[q];
        const Grid& g = I.grid;
        for (int c = 0; c < g.N; ++c) {
            double* o = &geo[(size_t)(R.cell_off[q] + c) * kGeo];
            o[0] = g.R_c[c];
            o[1] = 1.0 / g.dRds_c[c];
            o[2] = g.A_f[c + 1] / g.V_c[c];
            o[3] = g.A_f[c] / g.V_c[c];
            o[4] = I.p.geometry == FDLB_SPH ? 0.5 * g.kappa[c] : g.kappa[c];
            o[5] = g.V_c[c];
            if (I.band.width) {
                blo[(size_t)(R.cell_off[q] + c) * 2] = I.band.lo[c];
                blo[(size_t)(R.cell_off[q] + c) * 2 + 1] = I.band.cnt[c];
            }
        }
        double den[2];
        wall_tables(R, q, &gw[(size_t)q * 2 * (R.nR + R.n2 + R.n3)], den);
        boff += (size_t)I.p.n_cells * I.band.width;
    }
    FDLB_CUDA(cudaMemcpyAsync(R.inst_d, R.inst_h.data(), n * sizeof(InstDev), cudaMemcpyHostToDevice, R.stream));
    FDLB_CUDA(cudaMemcpyAsync(R.geo, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice, R.stream));
    FDLB_CUDA(cudaMemcpyAsync(R.gw, gw.data(), gw.size() * 8, cudaMemcpyHostToDevice, R.stream));
    std::vector<float> geof(geo.begin(), geo.end()), gwf(gw.begin(), gw.end());
    if (R.precision == FDLB_FP32) {
        FDLB_CUDA(cudaMemcpyAsync(R.geoT, geof.data(), geof.size() * 4, cudaMemcpyHostToDevice, R.stream));
        FDLB_CUDA(cudaMemcpyAsync(R.gwT, gwf.data(), gwf.size() * 4, cudaMemcpyHostToDevice, R.stream));
    } else {
        FDLB_CUDA(cudaMemcpyAsync(R.geoT, geo.data(), geo.size() * 8, cudaMemcpyHostToDevice, R.stream));
        FDLB_CUDA(cudaMemcpyAsync(R.gwT, gw.data(), gw.size() * 8, cudaMemcpyHostToDevice, R.stream));
    }
    FDLB_CUDA(cudaMemcpyAsync(R.band_lo, blo.data(), blo.size() * sizeof(int), cudaMemcpyHostToDevice, R.stream));
    // the Fischer-Methfessel weights, computed on the device (the faces of every instance staged in
    // the stage-1 population buffer, unused until the first step)
    {
        std::vector<double> faces;
        std::vector<size_t> face_off(n);
        for (int q = 0; q < n; ++q) {
            face_off[q] = faces.size();
            faces.insert(faces.end(), R.setup[q].grid.R_f.begin(), R.setup[q].grid.R_f.end());
        }
        if (faces.size() * sizeof(double) > L.f[2] - L.f[1]) return FDLB_ENOMEM;
        double* dfaces = reinterpret_cast<double*>(R.f[1]);
        FDLB_CUDA(cudaMemcpyAsync(dfaces, faces.data(), faces.size() * sizeof(double), cudaMemcpyHostToDevice, R.stream));
        const FmRule rule = fm_rule();
        for (int q = 0; q < n; ++q) {
            const InstanceSetup& I = R.setup[q];
            if (I.band.width == 0) continue;
            const int N = I.p.n_cells;
            FDLB_CUDA(launch_fm_band((int)R.tsize, R.geo + (size_t)R.cell_off[q] * kGeo, kGeo, dfaces + face_off[q], N,
                                     I.p.geometry == FDLB_SPH ? 1 : 0, I.sigma, I.band.width,
                                     reinterpret_cast<const int2*>(R.band_lo) + R.cell_off[q],
                                     (unsigned char*)R.band + (size_t)R.inst_h[q].band_off * R.tsize, rule,
                                     std::max(1, std::min(N, R.n_sm * 4)), R.stream));
        }
    }
    FDLB_CUDA(cudaStreamSynchronize(R.stream));
    // default tiling: a slice per p_3 value on the cylinder (p_3 is passive there)
    // default tiling (the fastest of a sweep on GB300; fdlb_autotune refines it per workload):
    // whole cells per block, 4 cells per tile (cylinder, 256 threads) or 8 (sphere, 512 threads).
    // The cylinder's 16 x 8 x 8 FP32 shape over many cells (batches) in blocks of 128 threads of
    // whole p_2 rows: 12% less time per stage on the 512-instance sweep, 30% more on one
    // 1024-cell instance, whose few tiles are bound by latency
    const bool cyl_rows = R.tsize == 4 && R.nR == 16 && R.n2 == 8 && R.n3 == 8 && R.total_cells > R.n_sm * 64;
    rc = R.geometry == FDLB_CYL ? configure_tiling(R, 4, R.n3, cyl_rows ? 128 : 256) : configure_tiling(R, 8, R.n3, 512);
    // closure items: few cells each where the whole closure is one short latency-bound launch (2 on
    // the cylinder, 4 on the sphere, with overlapped launches), 8 where items outnumber the blocks
    // that fit on the device several times over (batches, long instances: throughput-bound); with
    // items of the batch form (kClosureCells cells) several times the SM count, the batch form
    R.closure_cells = R.geometry == FDLB_CYL ? 2 : 4;
    if (R.total_cells / R.closure_cells > R.n_sm * 8) R.closure_cells = 8;
    R.closure_batch = R.total_cells / kClosureCells > R.n_sm * 4 ? 1 : 0;
    if (!rc) rc = upload_items(R);
    for (int q = 0; q < n && !rc; ++q) rc = fdlb_init_uniform(reinterpret_cast<fdlb_handle>(S.get()), q, 0.0, 0.0);
    if (rc) {
        if (R.own_ws) cudaFree(R.ws);
        if (R.own_stream) cudaStreamDestroy(R.stream);
        return rc;
    }
    *out = reinterpret_cast<fdlb_handle>(S.release());
    return FDLB_OK;
}

}  // namespace
}  // namespace fdlb

using fdlb::Solver;

static Solver* SOL(fdlb_handle h) { return reinterpret_cast<Solver*>(h); }

namespace fdlb {
// Per instance and chunk of C elements, the FP64 sums of (a - b)^2 and b^2 over populations (tsize 4
// or 8) at offsets off[q], counts cnt[q] (device arrays); part: n_inst * chunks * 2 doubles
// (kernels_aux.cu).
cudaError_t launch_change_sums(int tsize, const void* a, const void* b, const long long* off, const long long* cnt,
                               int n_inst, int chunks, long long C, double* part, cudaStream_t s);
}  // namespace fdlb

extern "C" {

int fdlb_create(const fdlb_params* p, void* cuda_stream, fdlb_handle* out) try {
    return fdlb::solver_create(p, 1, cuda_stream, nullptr, 0, out);
} FDLB_HOST_CATCH

int fdlb_batch_create(const fdlb_params* ps, int n_instances, void* cuda_stream, fdlb_handle* out) try {
    return fdlb::solver_create(ps, n_instances, cuda_stream, nullptr, 0, out);
} FDLB_HOST_CATCH

int fdlb_workspace_bytes(const fdlb_params* ps, int n_instances, size_t* bytes) {
    if (!bytes) return FDLB_EINVAL;
    Solver S;
    int rc = fdlb::plan_solver(ps, n_instances, S);
    if (rc) return rc;
    *bytes = fdlb::make_layout(S).total;
    return FDLB_OK;
}

int fdlb_create_in(const fdlb_params* ps, int n_instances, void* cuda_stream, void* workspace, size_t workspace_bytes,
                   fdlb_handle* out) try {
    if (!workspace) return FDLB_EINVAL;
    return fdlb::solver_create(ps, n_instances, cuda_stream, workspace, workspace_bytes, out);
} FDLB_HOST_CATCH

void fdlb_destroy(fdlb_handle h) {
    Solver* S = SOL(h);
    if (!S) return;
    if (S->stream) cudaStreamSynchronize(S->stream);
    else cudaDeviceSynchronize();
    if (S->gexec) cudaGraphExecDestroy(S->gexec);
    if (S->own_ws && S->ws) cudaFree(S->ws);
    for (cudaEvent_t e : S->tev)
        if (e) cudaEventDestroy(e);
    if (S->own_stream) cudaStreamDestroy(S->stream);
    delete S;
}

int fdlb_set_wall(fdlb_handle h, int instance, int side, double T_w, double u_tangential) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst || (side != 0 && side != 1)) return FDLB_EINVAL;
    if (!(T_w > 0.0) || !std::isfinite(u_tangential)) return FDLB_EINVAL;
    if (S->geometry == FDLB_SPH && u_tangential != 0.0) return FDLB_EINVAL;
    S->setup[instance].p.T_wall[side] = T_w;
    S->setup[instance].p.u_wall[side] = u_tangential;
    fdlb::fill_inst(*S, instance);
    const int stride = S->nR + S->n2 + S->n3;
    std::vector<double> gw(2 * stride);
    double den[2];
    fdlb::wall_tables(*S, instance, gw.data(), den);
    FDLB_CUDA(cudaMemcpyAsync(S->gw + (size_t)instance * 2 * stride, gw.data(), gw.size() * 8, cudaMemcpyHostToDevice,
                              S->stream));
    FDLB_CUDA(cudaMemcpyAsync(S->inst_d + instance, &S->inst_h[instance], sizeof(fdlb::InstDev),
                              cudaMemcpyHostToDevice, S->stream));
    FDLB_CUDA(cudaStreamSynchronize(S->stream));
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_init_uniform(fdlb_handle h, int instance, double n0, double T0) try {
    Solver* S = SOL(h);
    if (!S || instance >= S->n_inst) return FDLB_EINVAL;
    if (instance < 0) {
        for (int q = 0; q < S->n_inst; ++q) {
            int rc = fdlb_init_uniform(h, q, n0, T0);
            if (rc) return rc;
        }
        return FDLB_OK;
    }
    const fdlb::InstanceSetup& I = S->setup[instance];
    const int N = I.p.n_cells;
    const double nn = n0 > 0.0 ? n0 : I.n0;
    const double TT = T0 > 0.0 ? T0 : 0.5 * (I.p.T_wall[0] + I.p.T_wall[1]);
    std::vector<double> n(N, nn), u(N, 0.0), T(N, TT), q(N, 0.0), f;
    fdlb::seed_state(*S, instance, n, u, T, q, f);
    return fdlb::upload_state(*S, instance, f.data());
} FDLB_HOST_CATCH

int fdlb_init_from_moments(fdlb_handle h, int instance, const double* n, const double* u2, const double* T,
                           const double* qR, int n_points) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst || n_points < 2 || !n || !u2 || !T || !qR) return FDLB_EINVAL;
    for (int k = 0; k < n_points; ++k)
        if (!(n[k] > 0.0) || !(T[k] > 0.0) || !std::isfinite(u2[k]) || !std::isfinite(qR[k])) return FDLB_EINVAL;
    const fdlb::InstanceSetup& I = S->setup[instance];
    const int N = I.p.n_cells;
    const double a = I.grid.R_f[0], b = I.grid.R_f[N];
    std::vector<double> cn(N), cu(N), cT(N), cq(N), f;
    for (int c = 0; c < N; ++c) {
        const double x = (I.grid.R_c[c] - a) / (b - a) * (n_points - 1);
        int k = std::min(n_points - 2, std::max(0, (int)std::floor(x)));
        const double t = x - k;
        cn[c] = (1 - t) * n[k] + t * n[k + 1];
        cu[c] = (1 - t) * u2[k] + t * u2[k + 1];
        cT[c] = (1 - t) * T[k] + t * T[k + 1];
        cq[c] = (1 - t) * qR[k] + t * qR[k + 1];
    }
    fdlb::seed_state(*S, instance, cn, cu, cT, cq, f);
    return fdlb::upload_state(*S, instance, f.data());
} FDLB_HOST_CATCH

int fdlb_set_f(fdlb_handle h, int instance, const double* f_host) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst || !f_host) return FDLB_EINVAL;
    return fdlb::upload_state(*S, instance, f_host);
} FDLB_HOST_CATCH

int fdlb_get_f(fdlb_handle h, int instance, double* f_host) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst || !f_host) return FDLB_EINVAL;
    return fdlb::download_buf(*S, instance, 0, f_host);
} FDLB_HOST_CATCH

int fdlb_step(fdlb_handle h, int64_t n_steps) try {
    Solver* S = SOL(h);
    if (!S || n_steps < 0) return FDLB_EINVAL;
    return fdlb::do_steps(*S, n_steps);
} FDLB_HOST_CATCH

int fdlb_step_change(fdlb_handle h, double* rel_change) try {
    Solver* S = SOL(h);
    if (!S || !rel_change) return FDLB_EINVAL;
    const int n = S->n_inst;
    const long long C = 1LL << 16;
    long long maxc = 0;
    std::vector<long long> off(n), cnt(n);
    for (int q = 0; q < n; ++q) {
        off[q] = S->f_off[q];
        cnt[q] = (long long)S->setup[q].p.n_cells * S->Np;
        maxc = std::max(maxc, cnt[q]);
    }
    const int chunks = (int)std::max<long long>(1, (maxc + C - 1) / C);
    const size_t fbytes = S->f_elems * S->tsize;
    const size_t meta = (size_t)2 * n * sizeof(long long), pbytes = (size_t)n * chunks * 2 * sizeof(double);
    unsigned char* scratch = nullptr;
    if (cudaMalloc(&scratch, fbytes + meta + pbytes + 512) != cudaSuccess) {
        cudaGetLastError();
        return FDLB_ENOMEM;
    }
    long long* doff = reinterpret_cast<long long*>(scratch + (fbytes + 255) / 256 * 256);
    long long* dcnt = doff + n;
    double* part = reinterpret_cast<double*>(dcnt + n);
    std::vector<double> hp((size_t)n * chunks * 2);
    int rc = FDLB_OK;
    if (cudaMemcpyAsync(scratch, S->f[0], fbytes, cudaMemcpyDeviceToDevice, S->stream) != cudaSuccess ||
        cudaMemcpyAsync(doff, off.data(), n * sizeof(long long), cudaMemcpyHostToDevice, S->stream) != cudaSuccess ||
        cudaMemcpyAsync(dcnt, cnt.data(), n * sizeof(long long), cudaMemcpyHostToDevice, S->stream) != cudaSuccess)
        rc = FDLB_ECUDA;
    if (!rc) rc = fdlb::do_steps(*S, 1);
    if (!rc) rc = fdlb::cuda_status(fdlb::launch_change_sums((int)S->tsize, S->f[0], scratch, doff, dcnt, n, chunks, C, part,
                                                              S->stream));
    if (!rc && (cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
                cudaStreamSynchronize(S->stream) != cudaSuccess))
        rc = FDLB_ECUDA;
    cudaFree(scratch);
    if (rc) return rc;
    for (int q = 0; q < n; ++q) {
        double d2 = 0.0, b2 = 0.0;
        for (int k = 0; k < chunks; ++k) {
            d2 += hp[((size_t)q * chunks + k) * 2];
            b2 += hp[((size_t)q * chunks + k) * 2 + 1];
        }
        rel_change[q] = (S->active[q] && b2 > 0.0) ? std::sqrt(d2 / b2) : 0.0;
    }
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_eval_rhs(fdlb_handle h, int instance, double* L_host) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst || !L_host) return FDLB_EINVAL;
    int rc = fdlb::launch_stage(*S, 0, 0, 1, 0.0, 1.0, 1);
    if (rc) return rc;
    return fdlb::download_buf(*S, instance, 1, L_host);
} FDLB_HOST_CATCH

int fdlb_get_moments(fdlb_handle h, int instance, double* out, int on_device) try {
    Solver* S = SOL(h);
    if (!S || instance < -1 || instance >= S->n_inst || !out) return FDLB_EINVAL;
    // n, u, T, q, P_12 come from the FP64 raw sums of the current state alone (the closure's chi
    // and nbar, columns the query does not return, are not needed): the record kernel only, which
    // also writes the query's rows contiguously (into `out` itself for every instance on the device)
    static_assert(fdlb::kNmom == FDLB_NMOM, "moments query columns");
    const bool direct = on_device && instance < 0;
    double* packed = direct ? out : S->mpk;
    if (S->precision == FDLB_FP32)
        fdlb::launch_ca<float>(S->sums[0], S->cw, S->ca, S->M.slices, S->total_cells, S->stream, packed);
    else
        fdlb::launch_ca<double>(S->sums[0], S->cw, S->ca, S->M.slices, S->total_cells, S->stream, packed);
    FDLB_CUDA(cudaGetLastError());
    // instance -1: every instance's cells, in instance order (the cells of instance q follow those
    // of instances 0..q-1); one contiguous copy
    const int N = instance < 0 ? S->total_cells : S->setup[instance].p.n_cells;
    if (!direct) {
        const double* src = S->mpk + (instance < 0 ? (size_t)0 : (size_t)S->cell_off[instance] * FDLB_NMOM);
        FDLB_CUDA(cudaMemcpyAsync(out, src, (size_t)N * FDLB_NMOM * sizeof(double),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S->stream));
    }
    if (!on_device) FDLB_CUDA(cudaStreamSynchronize(S->stream));
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_get_closure(fdlb_handle h, int instance, double* nbar, double* chi, double* tau, double* n_wall2) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst) return FDLB_EINVAL;
    // a right-hand-side evaluation refreshes the closure records and the wall densities
    int rc = fdlb::launch_stage(*S, 0, 0, 1, 0.0, 1.0, 1, 1);
    if (rc) return rc;
    const int N = S->setup[instance].p.n_cells;
    std::vector<double> ca((size_t)N * fdlb::kCA);
    const int P = fdlb::kWallParts;
    std::vector<unsigned char> parts((size_t)2 * P * S->tsize);
    FDLB_CUDA(cudaMemcpyAsync(ca.data(), S->ca + (size_t)S->cell_off[instance] * fdlb::kCA, ca.size() * 8,
                              cudaMemcpyDeviceToHost, S->stream));
    FDLB_CUDA(cudaMemcpyAsync(parts.data(), (unsigned char*)S->nwp + (size_t)instance * 2 * P * S->tsize, parts.size(),
                              cudaMemcpyDeviceToHost, S->stream));
    FDLB_CUDA(cudaStreamSynchronize(S->stream));
    const fdlb::InstanceSetup& I = S->setup[instance];
    double nw[2];
    for (int side = 0; side < 2; ++side) {
        // the stage kernel's order and precision: parts summed in order, times 1 / nw_den
        const fdlb::InstDev& d = S->inst_h[instance];
        if (S->precision == FDLB_FP32) {
            const float* pp = reinterpret_cast<const float*>(parts.data()) + side * P;
            float sum = 0.f;
            for (int p = 0; p < P; ++p) sum += pp[p];
            nw[side] = (double)(sum * d.f_nw_iden[side]);
        } else {
            const double* pp = reinterpret_cast<const double*>(parts.data()) + side * P;
            double sum = 0.0;
            for (int p = 0; p < P; ++p) sum += pp[p];
            nw[side] = sum * d.nw_iden[side];
        }
    }
    for (int c = 0; c < N; ++c) {
        const double* r = &ca[(size_t)c * fdlb::kCA];
        if (nbar) nbar[c] = r[10];
        if (chi) chi[c] = r[9];
        if (tau) tau[c] = fdlb::viscosity(r[0], r[4], r[9], I.sigma) / (r[0] * r[4]);
    }
    if (n_wall2) {
        n_wall2[0] = nw[0];
        n_wall2[1] = nw[1];
    }
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_get_diagnostics(fdlb_handle h, int instance, double* total_mass, double* residual, int64_t* step) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst) return FDLB_EINVAL;
    fdlb::launch_residual(S->sums[0], S->M.slices, S->inst_d, S->geo, S->rprev, S->rout, S->n_inst, 0, S->stream);
    std::vector<double> ro((size_t)S->n_inst * 10);
    int errflag = 0;
    FDLB_CUDA(cudaMemcpyAsync(ro.data(), S->rout, ro.size() * 8, cudaMemcpyDeviceToHost, S->stream));
    FDLB_CUDA(cudaMemcpyAsync(&errflag, S->err, sizeof(int), cudaMemcpyDeviceToHost, S->stream));
    FDLB_CUDA(cudaStreamSynchronize(S->stream));
    if (total_mass) *total_mass = ro[(size_t)instance * 10 + 8];
    if (residual) *residual = S->last_res[instance];
    if (step) *step = S->inst_steps[instance];
    if (errflag) return FDLB_ETIMEOUT;
    if (ro[(size_t)instance * 10 + 9] != 0.0) return FDLB_ENAN;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_run_to_steady(fdlb_handle h, double tol, int64_t max_steps, double max_seconds, int check_every,
                       int64_t* steps_taken, double* residual) try {
    Solver* S = SOL(h);
    if (!S || !(tol > 0.0) || max_steps < 1 || check_every < 1) return FDLB_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    const int n = S->n_inst;
    std::vector<int64_t> taken(n, 0);
    std::vector<double> ro((size_t)n * 10);
    auto check = [&](int save) -> int {
        fdlb::launch_residual(S->sums[0], S->M.slices, S->inst_d, S->geo, S->rprev, S->rout, n, save, S->stream);
        FDLB_CUDA(cudaMemcpyAsync(ro.data(), S->rout, ro.size() * 8, cudaMemcpyDeviceToHost, S->stream));
        FDLB_CUDA(cudaStreamSynchronize(S->stream));
        return FDLB_OK;
    };
    int rc = check(1);
    if (rc) return rc;
    std::fill(S->active.begin(), S->active.end(), 1);
    rc = fdlb::upload_items(*S);
    if (rc) return rc;
    int status = FDLB_ENOTCONVERGED;
    bool nan_seen = false;
    std::vector<double> best(n, std::numeric_limits<double>::infinity());
    std::vector<int> since(n, 0);
    int64_t done = 0;
    while (done < max_steps) {
        const int64_t k = std::min<int64_t>(check_every, max_steps - done);
        rc = fdlb::do_steps(*S, k);
        if (rc) return rc;
        done += k;
        for (int q = 0; q < n; ++q)
            if (S->active[q]) taken[q] += k;
        rc = check(1);
        if (rc) return rc;
        bool any_active = false, changed = false;
        for (int q = 0; q < n; ++q) {
            if (!S->active[q]) continue;
            const double* r = &ro[(size_t)q * 10];
            if (r[9] != 0.0) {
                // non-finite moments: this instance stops, the others run on
                S->last_res[q] = std::numeric_limits<double>::infinity();
                S->active[q] = 0;
                changed = nan_seen = true;
                continue;
            }
            const fdlb::InstanceSetup& I = S->setup[q];
            const double T0 = 0.5 * (I.p.T_wall[0] + I.p.T_wall[1]);
            const double scale[4] = {I.n0, 1.0, T0, I.n0 * T0 * std::sqrt(T0)};
            double res = 0.0;
            for (int e = 0; e < 4; ++e) res = std::max(res, r[e] / ((double)k * std::max(r[4 + e], scale[e])));
            S->last_res[q] = res;
            if (res < 0.5 * best[q]) {
                best[q] = res;
                since[q] = 0;
            } else {
                ++since[q];
            }
            if (res <= tol || (S->stall_checks > 0 && since[q] >= S->stall_checks)) {
                S->active[q] = 0;
                changed = true;
            } else {
                any_active = true;
            }
        }
        if (!any_active) {
            bool all = true;
            for (int q = 0; q < n; ++q) all = all && S->last_res[q] <= tol;
            status = nan_seen ? FDLB_ENAN : (all ? FDLB_OK : FDLB_ENOTCONVERGED);
            break;
        }
        if (changed) {
            rc = fdlb::upload_items(*S);
            if (rc) return rc;
        }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (max_seconds > 0.0 && el > max_seconds) {
            status = nan_seen ? FDLB_ENAN : FDLB_ETIMEOUT;
            break;
        }
    }
    if (done >= max_steps && status == FDLB_ENOTCONVERGED && nan_seen) status = FDLB_ENAN;
    std::fill(S->active.begin(), S->active.end(), 1);
    rc = fdlb::upload_items(*S);
    if (rc) return rc;
    for (int q = 0; q < n; ++q) {
        if (steps_taken) steps_taken[q] = taken[q];
        if (residual) residual[q] = S->last_res[q];
    }
    return status;
} FDLB_HOST_CATCH

// The FP64 twin of an FP32 handle: the same instances (walls as set, the time step in use) with
// FP64 populations, in `workspace` when given.
static int make_fp64_twin(Solver* S, void* workspace, size_t ws_bytes, fdlb_handle* out) {
    std::vector<fdlb_params> ps(S->n_inst);
    for (int q = 0; q < S->n_inst; ++q) {
        ps[q] = S->setup[q].p;
        ps[q].precision = FDLB_FP64;
        ps[q].dt = S->setup[q].dt;
    }
    return fdlb::solver_create(ps.data(), S->n_inst, S->stream, workspace, ws_bytes, out);
}

int fdlb_polish_workspace_bytes(fdlb_handle h, size_t* bytes) try {
    Solver* S = SOL(h);
    if (!S || !bytes) return FDLB_EINVAL;
    std::vector<fdlb_params> ps(S->n_inst);
    for (int q = 0; q < S->n_inst; ++q) {
        ps[q] = S->setup[q].p;
        ps[q].precision = FDLB_FP64;
        ps[q].dt = S->setup[q].dt;
    }
    return fdlb_workspace_bytes(ps.data(), S->n_inst, bytes);
} FDLB_HOST_CATCH

// Total mass sum_c V_c n_c (FP64) of every instance's current state.
static int instance_masses(Solver* S, std::vector<double>& m) {
    fdlb::launch_residual(S->sums[0], S->M.slices, S->inst_d, S->geo, S->rprev, S->rout, S->n_inst, 0, S->stream);
    std::vector<double> ro((size_t)S->n_inst * 10);
    FDLB_CUDA(cudaMemcpyAsync(ro.data(), S->rout, ro.size() * 8, cudaMemcpyDeviceToHost, S->stream));
    FDLB_CUDA(cudaStreamSynchronize(S->stream));
    m.resize(S->n_inst);
    for (int q = 0; q < S->n_inst; ++q) m[q] = ro[(size_t)q * 10 + 8];
    return FDLB_OK;
}

int fdlb_run_to_steady_mixed(fdlb_handle h, double tol, int64_t max_steps, double max_seconds, int check_every,
                             void* fp64_workspace, size_t fp64_workspace_bytes, int64_t* steps_fp32,
                             int64_t* steps_fp64, double* residual) try {
    Solver* S = SOL(h);
    if (!S || !(tol > 0.0) || max_steps < 1 || check_every < 1) return FDLB_EINVAL;
    const int n = S->n_inst;
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<int64_t> st32(n, 0), st64(n, 0);
    std::vector<double> res(n, 0.0);
    if (S->precision != FDLB_FP32) {
        const int rc = fdlb_run_to_steady(h, tol, max_steps, max_seconds, check_every, st64.data(), res.data());
        for (int q = 0; q < n; ++q) {
            if (steps_fp32) steps_fp32[q] = 0;
            if (steps_fp64) steps_fp64[q] = st64[q];
            if (residual) residual[q] = res[q];
        }
        return rc;
    }
    // 1. the FP32 form to the tolerance (its residual reaches it; its steady state sits at the FP32
    // rounding floor, ~1e-5..1e-4 of the moment scales away from the FP64 one)
    std::vector<double> m0, m1;
    int rc = instance_masses(S, m0);
    if (rc) return rc;
    rc = fdlb_run_to_steady(h, tol, max_steps, max_seconds, check_every, st32.data(), res.data());
    if (rc != FDLB_OK && rc != FDLB_ENOTCONVERGED && rc != FDLB_ETIMEOUT && rc != FDLB_ENAN) return rc;
    const bool nan32 = rc == FDLB_ENAN;  // those instances stop at once in the FP64 phase too
    // the walls conserve mass and the steady state depends on it, but FP32 rounding walks the total
    // mass away by up to ~1e-9 of it per step: the polish starts from the FP32 state scaled back to
    // the mass this call began with
    rc = instance_masses(S, m1);
    if (rc) return rc;
    // 2. the FP64 polish from the FP32 steady state
    fdlb_handle th = nullptr;
    rc = make_fp64_twin(S, fp64_workspace, fp64_workspace_bytes, &th);
    if (rc) return rc;
    Solver* T = SOL(th);
    T->autotune_mode = S->autotune_mode;
    T->stall_checks = S->stall_checks;
    for (int q = 0; q < n; ++q) {
        const long long cnt = (long long)S->setup[q].p.n_cells * S->Np;
        const double scale = m1[q] > 0.0 && m0[q] > 0.0 ? m0[q] / m1[q] : 1.0;
        fdlb::launch_convert((const float*)S->f[0] + S->f_off[q], 1, (double*)T->f[0] + T->f_off[q], 0, cnt, S->stream,
                             scale);
    }
    rc = fdlb::cuda_status(cudaGetLastError());
    if (!rc) rc = fdlb::launch_moments_all(*T, 0);
    double left = 0.0;
    if (max_seconds > 0.0) {
        left = max_seconds - std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (left <= 0.0) left = 1e-9;
    }
    int rc64 = rc ? rc : fdlb_run_to_steady(th, tol, max_steps, left, check_every, st64.data(), res.data());
    // 3. the polished state, rounded to FP32, back into this handle (its moments are those of the
    // FP64 steady state to FP32 rounding, ~1e-7 of their scales)
    if (rc64 == FDLB_OK || rc64 == FDLB_ENOTCONVERGED || rc64 == FDLB_ETIMEOUT || rc64 == FDLB_ENAN) {
        for (int q = 0; q < n; ++q) {
            const long long cnt = (long long)S->setup[q].p.n_cells * S->Np;
            fdlb::launch_convert((const double*)T->f[0] + T->f_off[q], 0, (float*)S->f[0] + S->f_off[q], 1, cnt,
                                 S->stream);
            S->inst_steps[q] += st64[q];
            S->last_res[q] = res[q];
        }
        rc = fdlb::cuda_status(cudaGetLastError());
        if (!rc) rc = fdlb::launch_moments_all(*S, 0);
        S->prev_valid = false;
        if (rc) rc64 = rc;
    }
    fdlb_destroy(th);
    for (int q = 0; q < n; ++q) {
        if (steps_fp32) steps_fp32[q] = st32[q];
        if (steps_fp64) steps_fp64[q] = st64[q];
        if (residual) residual[q] = res[q];
    }
    if (nan32 && (rc64 == FDLB_OK || rc64 == FDLB_ENOTCONVERGED || rc64 == FDLB_ETIMEOUT)) rc64 = FDLB_ENAN;
    return rc64;
} FDLB_HOST_CATCH

int fdlb_get_info(fdlb_handle h, int instance, fdlb_info* out) try {
    Solver* S = SOL(h);
    if (!S || instance < 0 || instance >= S->n_inst || !out) return FDLB_EINVAL;
    const fdlb::InstanceSetup& I = S->setup[instance];
    out->C = I.C;
    out->sigma = I.sigma;
    out->n0 = I.n0;
    out->dt = I.dt;
    out->R_first = I.grid.R_f.front();
    out->R_last = I.grid.R_f.back();
    out->n_cells = I.p.n_cells;
    out->n_momenta = S->Np;
    out->fm_band = I.band.width;
    out->precision = S->precision;
    out->step = S->inst_steps[instance];
    return FDLB_OK;
} FDLB_HOST_CATCH

static const char kMagic[8] = {'F', 'D', 'L', 'B', 'C', 'K', 'P', '2'};

int fdlb_save(fdlb_handle h, const char* path) try {
    Solver* S = SOL(h);
    if (!S || !path) return FDLB_EINVAL;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return FDLB_EIO;
    bool ok = std::fwrite(kMagic, 1, 8, fp) == 8;
    const int32_t hdr[4] = {S->n_inst, S->Np, S->precision, S->geometry};
    ok = ok && std::fwrite(hdr, sizeof(hdr), 1, fp) == 1;
    for (int q = 0; q < S->n_inst && ok; ++q) {
        ok = std::fwrite(&S->setup[q].p, sizeof(fdlb_params), 1, fp) == 1;
        ok = ok && std::fwrite(&S->inst_steps[q], sizeof(int64_t), 1, fp) == 1;
        const size_t bytes = (size_t)S->setup[q].p.n_cells * S->Np * S->tsize;
        std::vector<unsigned char> buf(bytes);
        if (cudaMemcpyAsync(buf.data(), (unsigned char*)S->f[0] + S->f_off[q] * S->tsize, bytes, cudaMemcpyDeviceToHost,
                            S->stream) != cudaSuccess ||
            cudaStreamSynchronize(S->stream) != cudaSuccess) {
            std::fclose(fp);
            return FDLB_ECUDA;
        }
        ok = ok && std::fwrite(buf.data(), 1, bytes, fp) == bytes;
        // the raw sums of the state as the stage epilogue computed them, so that a restart
        // continues bit for bit (a recomputation sums in another order)
        const int32_t slices = S->M.slices;
        const size_t sbytes = (size_t)S->setup[q].p.n_cells * slices * fdlb::kSums * sizeof(double);
        std::vector<unsigned char> sb(sbytes);
        if (cudaMemcpyAsync(sb.data(), S->sums[0] + (size_t)S->cell_off[q] * slices * fdlb::kSums, sbytes,
                            cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
            cudaStreamSynchronize(S->stream) != cudaSuccess) {
            std::fclose(fp);
            return FDLB_ECUDA;
        }
        ok = ok && std::fwrite(&slices, sizeof(slices), 1, fp) == 1;
        ok = ok && std::fwrite(sb.data(), 1, sbytes, fp) == sbytes;
    }
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? FDLB_OK : FDLB_EIO;
} FDLB_HOST_CATCH

int fdlb_load(fdlb_handle h, const char* path) try {
    Solver* S = SOL(h);
    if (!S || !path) return FDLB_EINVAL;
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return FDLB_EIO;
    char mg[8];
    int32_t hdr[4];
    int rc = FDLB_OK;
    if (std::fread(mg, 1, 8, fp) != 8 || std::memcmp(mg, kMagic, 8) || std::fread(hdr, sizeof(hdr), 1, fp) != 1) {
        std::fclose(fp);
        return FDLB_EIO;
    }
    if (hdr[0] != S->n_inst || hdr[1] != S->Np || hdr[2] != S->precision || hdr[3] != S->geometry) {
        std::fclose(fp);
        return FDLB_EINVAL;
    }
    bool recompute = false;
    for (int q = 0; q < S->n_inst && !rc; ++q) {
        fdlb_params p;
        int64_t st;
        if (std::fread(&p, sizeof(p), 1, fp) != 1 || std::fread(&st, sizeof(st), 1, fp) != 1) {
            rc = FDLB_EIO;
            break;
        }
        const fdlb_params& mine = S->setup[q].p;
        if (p.n_cells != mine.n_cells || p.R_in != mine.R_in || p.R_out != mine.R_out || p.eta0 != mine.eta0) {
            rc = FDLB_EINVAL;
            break;
        }
        const size_t bytes = (size_t)mine.n_cells * S->Np * S->tsize;
        std::vector<unsigned char> buf(bytes);
        if (std::fread(buf.data(), 1, bytes, fp) != bytes) {
            rc = FDLB_EIO;
            break;
        }
        if (cudaMemcpyAsync((unsigned char*)S->f[0] + S->f_off[q] * S->tsize, buf.data(), bytes, cudaMemcpyHostToDevice,
                            S->stream) != cudaSuccess ||
            cudaStreamSynchronize(S->stream) != cudaSuccess) {
            rc = FDLB_ECUDA;
            break;
        }
        S->inst_steps[q] = st;
        int32_t slices = 0;
        if (std::fread(&slices, sizeof(slices), 1, fp) != 1 || slices < 1 || slices > S->n3) {
            rc = FDLB_EIO;
            break;
        }
        const size_t sbytes = (size_t)mine.n_cells * slices * fdlb::kSums * sizeof(double);
        std::vector<unsigned char> sb(sbytes);
        if (std::fread(sb.data(), 1, sbytes, fp) != sbytes) {
            rc = FDLB_EIO;
            break;
        }
        if (slices != S->M.slices) {
            recompute = true;  // saved under another momentum slicing
        } else if (cudaMemcpyAsync(S->sums[0] + (size_t)S->cell_off[q] * slices * fdlb::kSums, sb.data(), sbytes,
                                   cudaMemcpyHostToDevice, S->stream) != cudaSuccess ||
                   cudaStreamSynchronize(S->stream) != cudaSuccess) {
            rc = FDLB_ECUDA;
            break;
        }
    }
    std::fclose(fp);
    if (rc) return rc;
    S->prev_valid = false;
    if (recompute) return fdlb::launch_moments_all(*S, 0);
    const long long nd = (long long)S->total_cells * S->M.slices;
    if (S->precision == FDLB_FP32) {
        fdlb::launch_dens_from_sums<float>(S->sums[0], (float*)S->dens[0], nd, S->stream);
        fdlb::launch_sums_pairs(S->sums[0], S->sumsw[0], nd * fdlb::kSums, S->stream);
    }
    else
        fdlb::launch_dens_from_sums<double>(S->sums[0], (double*)S->dens[0], nd, S->stream);
    return fdlb::cuda_status(cudaGetLastError());
} FDLB_HOST_CATCH

const char* fdlb_error_string(int code) {
    switch (code) {
        case FDLB_OK: return "ok";
        case FDLB_EINVAL: return "invalid argument";
        case FDLB_ECUDA: return "CUDA runtime error";
        case FDLB_ENOMEM: return "out of memory or workspace too small";
        case FDLB_ENOTCONVERGED: return "not converged within max_steps";
        case FDLB_ETIMEOUT: return "time limit reached or a device wait gave up";
        case FDLB_ENAN: return "non-finite moments";
        case FDLB_EIO: return "checkpoint I/O error";
        case FDLB_ENOGPU: return "no usable CUDA device";
        default: return "unknown error";
    }
}

int fdlb_set_tiling(fdlb_handle h, int cells_per_tile, int slice_k, int threads) try {
    Solver* S = SOL(h);
    if (!S || cells_per_tile < 0 || slice_k < 0 || threads < 0) return FDLB_EINVAL;
    return fdlb::configure_tiling(*S, cells_per_tile, slice_k, threads);
} FDLB_HOST_CATCH

int fdlb_autotune(fdlb_handle h, int* cells_per_tile, int* slice_k, int* threads) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    const int rc = fdlb::run_autotune(*S, false);
    if (cells_per_tile) *cells_per_tile = S->B;
    if (slice_k) *slice_k = S->KS;
    if (threads) *threads = S->threads;
    return rc;
} FDLB_HOST_CATCH

int fdlb_set_autotune(fdlb_handle h, int mode) try {
    Solver* S = SOL(h);
    if (!S || mode < 0 || mode > 2) return FDLB_EINVAL;
    S->autotune_mode = mode;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_get_stage_kernel(fdlb_handle h, int* vector_width, int* vectors_per_thread, int* min_blocks) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    if (vector_width) *vector_width = S->scfg.vw;
    if (vectors_per_thread) *vectors_per_thread = S->scfg.nv;
    if (min_blocks) *min_blocks = S->scfg.minb;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_get_tiling(fdlb_handle h, int* cells_per_tile, int* slice_k, int* threads, int* closure_cells) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    if (cells_per_tile) *cells_per_tile = S->B;
    if (slice_k) *slice_k = S->KS;
    if (threads) *threads = S->threads;
    if (closure_cells) *closure_cells = S->closure_cells;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_set_tensor_contraction(fdlb_handle h, int enable, int* in_use) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    S->tensor = enable ? 1 : 0;
    if (S->krg_on) {
        // large radial orders: the contraction kernel on the tensor cores (FP32) or the CUDA cores
        S->kr_tc = S->tensor && S->krB ? 1 : 0;
        if (S->gexec) {
            cudaGraphExecDestroy(S->gexec);
            S->gexec = nullptr;
        }
        if (in_use) *in_use = S->kr_tc;
        return FDLB_OK;
    }
    const int rc = fdlb::configure_tiling(*S, S->B, S->KS, S->threads);
    if (in_use) *in_use = S->mma_on;
    return rc;
} FDLB_HOST_CATCH

int fdlb_set_persistent_step(fdlb_handle h, int enable, int* in_use) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    if (enable < 0) {  // query only
        if (in_use) *in_use = S->fused_on;
        return FDLB_OK;
    }
    S->fused = enable ? 1 : 0;
    const int rc = fdlb::configure_tiling(*S, S->B, S->KS, S->threads);
    if (in_use) *in_use = S->fused_on;
    return rc;
} FDLB_HOST_CATCH

int fdlb_set_wait_test(fdlb_handle h, int tx_extra_bytes, int barrier_extra) try {
    Solver* S = SOL(h);
    if (!S || tx_extra_bytes < 0 || tx_extra_bytes > 65536 || barrier_extra < 0 || barrier_extra > 65536) return FDLB_EINVAL;
    S->test_tx_extra = tx_extra_bytes;
    S->test_bar_extra = barrier_extra;
    if (S->gexec) {
        cudaGraphExecDestroy(S->gexec);
        S->gexec = nullptr;
    }
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_clear_error(fdlb_handle h) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    FDLB_CUDA(cudaMemsetAsync(S->err, 0, sizeof(int), S->stream));
    FDLB_CUDA(cudaStreamSynchronize(S->stream));
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_set_programmatic_launch(fdlb_handle h, int enable) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    S->programmatic = enable ? 1 : 0;
    if (S->gexec) {
        cudaGraphExecDestroy(S->gexec);
        S->gexec = nullptr;
    }
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_set_closure_cells(fdlb_handle h, int cells) try {
    Solver* S = SOL(h);
    if (!S || cells < 1 || cells > fdlb::kClosureCells) return FDLB_EINVAL;
    return fdlb::set_closure_grouping(*S, cells, 0);
} FDLB_HOST_CATCH

int fdlb_set_stall_checks(fdlb_handle h, int checks) try {
    Solver* S = SOL(h);
    if (!S || checks < 0) return FDLB_EINVAL;
    S->stall_checks = checks;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_set_closure_form(fdlb_handle h, int form, int* in_use) try {
    Solver* S = SOL(h);
    if (!S || form < -1 || form > 1) return FDLB_EINVAL;
    if (form >= 0) {
        const int rc = fdlb::set_closure_grouping(*S, S->closure_cells, form);
        if (rc) return rc;
    }
    if (in_use) *in_use = S->closure_batch;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_set_stage_min_blocks(fdlb_handle h, int min_blocks, int* in_use) try {
    Solver* S = SOL(h);
    if (!S || min_blocks < -1 || min_blocks == 0 || min_blocks > 5) return FDLB_EINVAL;
    if (min_blocks > 0) {
        const int old = S->stage_minb;
        S->stage_minb = min_blocks;
        int rc = fdlb::configure_tiling(*S, S->B, S->KS, S->threads);
        if (rc == FDLB_OK && S->scfg.minb != min_blocks) rc = FDLB_EINVAL;  // not built for this shape
        if (rc) {
            S->stage_minb = old;
            fdlb::configure_tiling(*S, S->B, S->KS, S->threads);
            return rc;
        }
    }
    if (in_use) *in_use = S->scfg.minb;
    return FDLB_OK;
} FDLB_HOST_CATCH

int64_t fdlb_launch_count(fdlb_handle h) {
    Solver* S = SOL(h);
    return S ? S->last_launches : -1;
}

int fdlb_set_graph_steps(fdlb_handle h, int steps) try {
    Solver* S = SOL(h);
    if (!S || steps < 1 || steps > 1000) return FDLB_EINVAL;
    if (steps != S->graph_steps && S->gexec) {
        cudaGraphExecDestroy(S->gexec);
        S->gexec = nullptr;
    }
    S->graph_steps = steps;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_set_kernel_timing(fdlb_handle h, int on) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    if (on && !S->tev[0])
        for (cudaEvent_t& e : S->tev) FDLB_CUDA(cudaEventCreate(&e));
    S->timing = on != 0;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_kernel_times(fdlb_handle h, double* stream_ms, int64_t* n_stream, double* closure_ms, int64_t* n_closure) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    if (stream_ms) *stream_ms = S->t_stream_ms;
    if (n_stream) *n_stream = S->n_stream_t;
    if (closure_ms) *closure_ms = S->t_closure_ms;
    if (n_closure) *n_closure = S->n_closure_t;
    S->t_stream_ms = S->t_closure_ms = 0.0;
    S->n_stream_t = S->n_closure_t = 0;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_step_kernel_times(fdlb_handle h, double* ms, int64_t* launches, int64_t* steps) try {
    Solver* S = SOL(h);
    if (!S) return FDLB_EINVAL;
    if (ms) *ms = S->t_step_ms;
    if (launches) *launches = S->n_step_t;
    if (steps) *steps = S->n_step_steps;
    S->t_step_ms = 0.0;
    S->n_step_t = S->n_step_steps = 0;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_get_stream(fdlb_handle h, void** stream) try {
    Solver* S = SOL(h);
    if (!S || !stream) return FDLB_EINVAL;
    *stream = (void*)S->stream;
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_set_state_raw(fdlb_handle h, int instance, const void* src, int on_device) try {
    Solver* S = SOL(h);
    if (!S || instance < -1 || instance >= S->n_inst || !src) return FDLB_EINVAL;
    if (instance < 0) {
        // the whole batch as the library stores it, one copy and one pass of the raw sums
        FDLB_CUDA(cudaMemcpyAsync(S->f[0], src, S->f_elems * S->tsize,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S->stream));
        std::fill(S->inst_steps.begin(), S->inst_steps.end(), 0);
        S->prev_valid = false;
        return fdlb::launch_moments_all(*S, 0);
    }
    const size_t bytes = (size_t)S->setup[instance].p.n_cells * S->Np * S->tsize;
    FDLB_CUDA(cudaMemcpyAsync((unsigned char*)S->f[0] + S->f_off[instance] * S->tsize, src, bytes,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S->stream));
    S->inst_steps[instance] = 0;
    return fdlb::launch_moments_all(*S, 0);
} FDLB_HOST_CATCH

int fdlb_get_state_raw(fdlb_handle h, int instance, void* dst, int on_device) try {
    Solver* S = SOL(h);
    if (!S || instance < -1 || instance >= S->n_inst || !dst) return FDLB_EINVAL;
    const size_t bytes = instance < 0 ? S->f_elems * S->tsize : (size_t)S->setup[instance].p.n_cells * S->Np * S->tsize;
    const unsigned char* src = (const unsigned char*)S->f[0] + (instance < 0 ? 0 : S->f_off[instance] * S->tsize);
    FDLB_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S->stream));
    if (!on_device) FDLB_CUDA(cudaStreamSynchronize(S->stream));
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_state_bytes(fdlb_handle h, size_t* bytes) try {
    Solver* S = SOL(h);
    if (!S || !bytes) return FDLB_EINVAL;
    *bytes = S->f_elems * S->tsize;
    return FDLB_OK;
} FDLB_HOST_CATCH

}  // extern "C"
