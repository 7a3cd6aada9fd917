// Auxiliary kernels of the FDLB step (raw sums, closure, residual); the fused stage kernel is
// in stream_kernel.cuh.  See kernels.cuh for the data layout and the launch plan.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.cuh"
#include "kernels_decl.h"
#include "closure_item.cuh"
#include "fm_volumes.h"
#include "internal.h"

namespace fdlb {

// ------------------------------------------------------------------------------ moments
// Raw quadrature sums (Eq. mom_quad) of whole cells of a state, a warp per cell: a lane per
// momentum row (k, i) of n2 contiguous values (the rows of a warp are one contiguous span of the
// cell); per row the power sums over p_2 as in the stage kernel's epilogue, the thirteen sums in
// the populations' precision over the lane's rows, then a transposed warp sum.  Written into slice
// 0 of the partial-sum array in FP64 (the other slices cleared), for FP32 populations also as the
// double-float pairs the closure reads, and the slice densities.  Every cell of the state.
constexpr int kMomMaxNodes = 2 * kMaxQR;  // radial nodes

template <typename T>
__global__ void __launch_bounds__(256) moments_kernel(const T* __restrict__ f, double* __restrict__ sums,
                                                      T* __restrict__ dens, float2* __restrict__ sumsw,
                                                      long long total_cells, const double* __restrict__ tab, MomSet M) {
    __shared__ T sp_R[kMomMaxNodes], sp_2[kMaxQ], sp_3[kMaxQ];
    const int lane = threadIdx.x & 31;
    const int nR = M.nR, n2 = M.n2, n3 = M.n3, Np = M.Np;
    for (int e = threadIdx.x; e < nR; e += blockDim.x) sp_R[e] = (T)tab[M.o_pR + e];
    for (int e = threadIdx.x; e < n2; e += blockDim.x) sp_2[e] = (T)tab[M.o_p2 + e];
    for (int e = threadIdx.x; e < n3; e += blockDim.x) sp_3[e] = (T)tab[M.o_p3 + e];
    __syncthreads();
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int rows = nR * n3;
    for (long long c = w0; c < total_cells; c += nw) {
        const T* fc = f + c * Np;
        T acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = T(0);
        for (int r = lane; r < rows; r += 32) {
            const int k = r / nR, i = r % nR;
            const T* row = fc + (long long)r * n2;
            T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
            for (int j = 0; j < n2; ++j) {
                const T v = row[j], p2v = sp_2[j];
                const T o1 = v * p2v, o2 = o1 * p2v;
                s0 += v;
                s1 += o1;
                s2 += o2;
                s3 += o2 * p2v;
            }
            const T pr = sp_R[i], p3v = sp_3[k];
            const T prs0 = pr * s0, p3s0 = p3v * s0, rr = pr * pr + p3v * p3v;
            if (M.reduced && k == 1) {
                // chi = int p_z^2 f: S2_zz and the p_z^2 p_a part of S3_a
                acc[6] += s0;
                acc[10] += prs0;
                acc[11] += s1;
                continue;
            }
            const T e10 = rr * s0 + s2;
            acc[0] += s0;
            acc[1] += prs0;
            acc[2] += s1;
            acc[3] += p3s0;
            acc[4] += pr * prs0;
            acc[5] += s2;
            acc[6] += p3v * p3s0;
            acc[7] += pr * s1;
            acc[8] += pr * p3s0;
            acc[9] += p3v * s1;
            acc[10] += pr * e10;
            acc[11] += rr * s1 + s3;
            acc[12] += p3v * e10;
        }
        const T tot = warp_sum16_transposed(acc, lane);
        const int q = lane >> 1;
        if (!(lane & 1) && q < kSums) {
            const double sd = (double)tot;
            const long long base = c * M.slices * kSums;
            sums[base + q] = sd;
            for (int sl = 1; sl < M.slices; ++sl) sums[base + sl * kSums + q] = 0.0;
            if (sumsw) {  // the double-float pairs of the FP32 closure
                sumsw[base + q] = make_float2((float)tot, 0.f);
                for (int sl = 1; sl < M.slices; ++sl) sumsw[base + sl * kSums + q] = make_float2(0.f, 0.f);
            }
            if (q == 0) {
                T* dd = dens + c * M.slices;
                dd[0] = tot;
                for (int sl = 1; sl < M.slices; ++sl) dd[sl] = T(0);
            }
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

// ------------------------------------------------------------------------------ batch closure
// The closure of a batch as two launches over all items instead of one item chain per block.  With
// many more items than co-resident blocks the chain form is bound by how many items are in flight:
// most of its phases run one lane per reach cell while the other lanes wait at its barriers, and
// its FM band rows are read one item at a time.  Here closure_band_kernel gives every band row of
// every item to a warp of its own (the band sum of Eq. fm, then chi and nbar into A.cw) and takes
// the wall items, with no block barrier; closure_records_kernel then forms each item's records from
// the raw sums of its reach and the band results, every phase spread over the whole block.  Both
// are made of the chain's per-cell functions (closure_item.cuh), so the records are the chain's.

// A warp per job of the host-formed list A.pairs: two band rows summed together by clo_band_row2
// with the loads of both in flight, then chi and nbar of the two cells; or one part of the
// outgoing flux through a wall.  A job's description is one 48-byte load, so the weights and
// densities follow it after a single dependent load.
template <typename T>
__global__ void __launch_bounds__(kClosureThreads, sizeof(T) == 4 ? 8 : 4) closure_band_kernel(ClosureArgs A, MomSet M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ClosureTabs<T> tb = closure_tables<T>(reinterpret_cast<T*>(smem_raw), A.tabT, M, tid, blockDim.x);
    __syncthreads();
    pdl_wait();  // the densities and populations of the previous kernel
    pdl_trigger();
    const T* fin_all = reinterpret_cast<const T*>(A.f_in);
    const T* band = reinterpret_cast<const T*>(A.band);
    const T* dens = reinterpret_cast<const T*>(A.dens);
    T* nwp = reinterpret_cast<T*>(A.nwp);
    T* cw = reinterpret_cast<T*>(A.cw);
    const int slices = A.slices;
    const int np = *A.n_pairs;
    const int gw = blockIdx.x * kClosureWarps + warp, nw = gridDim.x * kClosureWarps;
    for (int v = gw; v < np; v += nw) {
        const BandPair P = A.pairs[v];
        if (P.kmaxA < 0) {
            // one part of the outgoing flux through a wall, by one warp in the order of the chain
            // form's block of kClosureThreads threads: lane L takes the momenta of its threads
            // L, L + 32, L + 64, L + 96 and the four warp sums are combined as there
            const InstDev I = A.inst[P.q];
            const int side = -1 - P.kmaxA, part = P.kmaxB, WP = A.wall_parts;
            const T* wall = fin_all + I.f_off + (side == 0 ? 0LL : (long long)(I.n_cells - 1) * M.Np);
            T r[kClosureWarps];
#pragma unroll
            for (int vw = 0; vw < kClosureWarps; ++vw)
                r[vw] = warp_sum(wall_flux_partial<T>(wall, side == 0 ? (long long)M.Np : -(long long)M.Np, M, tb, side,
                                                      part, WP, 32 * vw + lane));
            if (lane == 0) nwp[((long long)P.q * 2 + side) * WP + part] = wall_part_sum(r);
            continue;
        }
        const T* ndA = dens + P.dA * slices;
        const T* ndB = dens + P.dB * slices;
        auto dA = [&](int k) {
            T x = ndA[(long long)k * slices];
            for (int sl = 1; sl < slices; ++sl) x += ndA[(long long)k * slices + sl];
            return x;
        };
        auto dB = [&](int k) {
            T x = ndB[(long long)k * slices];
            for (int sl = 1; sl < slices; ++sl) x += ndB[(long long)k * slices + sl];
            return x;
        };
        T totA, totB;
        clo_band_row2<T>(band + P.wA, dA, P.kmaxA, band + P.wB, dB, P.kmaxB, lane, totA, totB);
        // lane 0's sums: every lane ends the butterfly with the total, but each in an order of its
        // own, and the chain form takes lane 0's
        if (lane == 0) {
            const InstDev& I = A.inst[P.q];
            const T etaf = inst_param<T>(I.etafac, I.f_etafac);
            const long long gc = P.gc;
            cw[gc * 2] = clo_chi<T>(etaf, totA);
            cw[gc * 2 + 1] = totA;
            if (P.kmaxB > 0) {
                cw[gc * 2 + 2] = clo_chi<T>(etaf, totB);
                cw[gc * 2 + 3] = totB;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kClosureThreads, sizeof(T) == 4 ? 8 : 4) closure_records_kernel(ClosureArgs A, MomSet M) {
    using W = Wide<T>;
    __shared__ W sw_n[32], sw_T[32], sw_u[3][32];  // reach cells
    __shared__ T s_chi[32], snb[32];
    __shared__ T sq[kClosureCells][3], sgeo[kClosureCells][2];  // own cells
    __shared__ T ecs[kClosureCells][4][kMaxE];
    __shared__ T sgp[kClosureCells][5][5];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    const ClosureTabs<T> tb = closure_tables<T>(reinterpret_cast<T*>(smem_raw), A.tabT, M, tid, NT);
    __syncthreads();
    pdl_wait();  // the band results of closure_band_kernel
    pdl_trigger();
    T* cw = reinterpret_cast<T*>(A.cw);
    const T* geoT = reinterpret_cast<const T*>(A.geoT);
    T* rec_all = reinterpret_cast<T*>(A.rec);
    const int rs = A.rec_stride, ng = M.nR + M.n2 + M.n3;
    const ReachView<T> RV{sw_n, sw_T, {sw_u[0], sw_u[1], sw_u[2]}, s_chi, snb};
    const int nit = *A.n_items;
    for (int it = blockIdx.x; it < nit; it += gridDim.x) {
        const int4 w = A.items[it];
        if (w.w != 0) continue;  // wall items: closure_band_kernel
        const InstDev I = A.inst[w.x];
        const int c0 = w.y, cnt = w.z, N = I.n_cells;
        int h0, h1;
        clo_reach(c0, cnt, N, h0, h1);
        const int nh = h1 - h0;
        T* recb = rec_all + (long long)(I.cell_off + c0) * rs;
        const T etaf = inst_param<T>(I.etafac, I.f_etafac);
        // ---- the reach's n, u, T from the raw sums (thread per reach cell), chi and nbar from the
        // band kernel or, for chi at the local density, here; the own cells' q and geometry
        for (int e = tid; e < nh; e += NT) {
            const long long gc = (long long)I.cell_off + h0 + e;
            W sv[kSums];
            clo_load_sums<T>(A, gc, sv);
            W n, u[3], Tc;
            T q[3];
            clo_fields<T>(sv, n, u, Tc, q);
            sw_n[e] = n;
            sw_u[0][e] = u[0];
            sw_u[1][e] = u[1];
            sw_u[2][e] = u[2];
            sw_T[e] = Tc;
            const int t = h0 + e - c0;
            if (I.chi_local) {
                s_chi[e] = clo_chi<T>(etaf, w_hi(n));
                snb[e] = w_hi(n);
                if (t >= 0 && t < cnt) {
                    cw[gc * 2] = s_chi[e];
                    cw[gc * 2 + 1] = snb[e];
                }
            } else {
                s_chi[e] = cw[gc * 2];
                snb[e] = cw[gc * 2 + 1];
            }
            if (t >= 0 && t < cnt) {
                sq[t][0] = q[0];
                sq[t][1] = q[1];
                sq[t][2] = q[2];
                const T* g = geoT + gc * kGeo;
                sgeo[t][0] = g[0];
                sgeo[t][1] = g[1];
            }
        }
        __syncthreads();
        // ---- gradient terms (thread per own cell and stencil position)
        for (int e = tid; e < cnt * 5; e += NT) {
            const int t = e / 5, q = e % 5, c = c0 + t;
            int cq;
            T wq;
            stencil5_at<T>(c, N, q, cq, wq);
            T g[5];
            clo_grad_terms<T>(RV, cq - h0, c - h0, wq, etaf, I.chi_local != 0, g);
#pragma unroll
            for (int v = 0; v < 5; ++v) sgp[t][v][q] = g[v];
        }
        __syncthreads();
        // ---- expansion coefficients (warp = job, lane = own cell); the last warp, whose job (the
        // third axis) is the shortest, then the record scalars
        if (lane < cnt) {
            const int t = lane, job = warp, lt = c0 + t - h0;
            const T cT = w_hi(sw_T[lt]);
            const T tm1 = w_hi(w_sub(sw_T[lt], w_from_t(T(1))));  // T - 1 without cancellation
            T ev[kMaxE + 1];
            clo_eq_coeffs<T>(job, cT, tm1, w_hi(sw_u[0][lt]), w_hi(sw_u[job == 2 ? 1 : 2][lt]), tb, M, ev);
#pragma unroll
            for (int l = 0; l < kMaxE; ++l) ecs[t][job][l] = ev[l];
            if (warp == kClosureWarps - 1) {
                const T q[3] = {sq[t][0], sq[t][1], sq[t][2]};
                clo_record_scalars<T>(recb + (long long)t * rs, RV, lt, sgp[t], sgeo[t][0], sgeo[t][1], q, I);
            }
        }
        __syncthreads();
        // ---- per-axis equilibrium vectors
        for (int e = tid; e < cnt * ng; e += NT) {
            const int t = e / ng, k = e % ng;
            int dst;
            const T g = clo_g_entry<T>(k, ecs[t], w_hi(sw_T[c0 + t - h0]), tb, M, dst);
            recb[(long long)t * rs + dst] = g;
        }
        __syncthreads();
        // ---- discrete mass of the stored equilibrium (a thread per own cell)
        for (int t = tid; t < cnt; t += NT) clo_mass_normalise<T>(recb + (long long)t * rs, sw_n[c0 + t - h0], M);
        __syncthreads();  // shared arrays are reused by the next item
    }
}

// ------------------------------------------------------------------------------ state change
// Sums over one chunk of an instance's populations of (a - b)^2 and b^2 in FP64 (a the state after
// a step, b before it): chunk k of instance q covers elements [k C, (k + 1) C) of the instance; the
// block's sums go to part[(q * chunks + k) * 2 + {0, 1}] in a fixed tree order.
template <typename T>
__global__ void change_sums_kernel(const T* __restrict__ a, const T* __restrict__ b, const long long* __restrict__ off,
                                   const long long* __restrict__ cnt, int chunks, long long C, double* __restrict__ part) {
    __shared__ double red[2][32];
    const int q = blockIdx.x / chunks, k = blockIdx.x % chunks;
    const long long lo = k * C, hi = min(cnt[q], lo + C);
    double d2 = 0.0, b2 = 0.0;
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
        const double x = (double)a[off[q] + e], y = (double)b[off[q] + e];
        d2 += (x - y) * (x - y);
        b2 += y * y;
    }
    d2 = warp_sum(d2);
    b2 = warp_sum(b2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = d2;
        red[1][warp] = b2;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
        part[((long long)q * chunks + k) * 2 + threadIdx.x] = s;
    }
}

cudaError_t launch_change_sums(int tsize, const void* a, const void* b, const long long* off, const long long* cnt,
                               int n_inst, int chunks, long long C, double* part, cudaStream_t s) {
    const int grid = n_inst * chunks;
    if (tsize == 4)
        change_sums_kernel<float><<<grid, 256, 0, s>>>((const float*)a, (const float*)b, off, cnt, chunks, C, part);
    else
        change_sums_kernel<double><<<grid, 256, 0, s>>>((const double*)a, (const double*)b, off, cnt, chunks, C, part);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------ queries
// The FP64 closure record of every cell of the active instances (moments and closure queries,
// not the stage): n, u, T, q, P_12 (Eq. macro_def) from the raw sums in FP64, chi and nbar from
// the closure's side buffer.
template <typename T>
__global__ void ca_kernel(const double* __restrict__ sums, const void* cwv, double* __restrict__ ca, int slices,
                          int total_cells, double* __restrict__ packed) {
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
        if (packed)  // the moments query's rows: the first kNmom columns, contiguous
            for (int e = 0; e < kNmom; ++e) packed[(long long)c * kNmom + e] = r[e];
    }
}

template <typename T>
void launch_ca(const double* sums, const void* cw, double* ca, int slices, int total_cells, cudaStream_t s,
               double* packed) {
    const int g = (total_cells + 255) / 256;
    ca_kernel<T><<<g < 2048 ? (g > 0 ? g : 1) : 2048, 256, 0, s>>>(sums, cw, ca, slices, total_cells, packed);
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
void launch_moments(const T* f, double* sums, T* dens, void* sumsw, long long total_cells, int grid, const double* tab,
                    const MomSet& M, cudaStream_t s) {
    moments_kernel<T><<<grid, 256, 0, s>>>(f, sums, dens, reinterpret_cast<float2*>(sumsw), total_cells, tab, M);
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

template <typename T>
void launch_closure_batch(const ClosureArgs& A, const MomSet& M, int grid, size_t smem, cudaStream_t s) {
    launch_maybe_programmatic(closure_band_kernel<T>, grid, kClosureThreads, smem, s, A.programmatic, A, M);
    launch_maybe_programmatic(closure_records_kernel<T>, grid, kClosureThreads, smem, s, A.programmatic, A, M);
}

int closure_batch_blocks_per_sm(int tsize, size_t smem) {
    int a = 0, b = 0;
    cudaError_t e1, e2;
    if (tsize == 4) {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, closure_band_kernel<float>, kClosureThreads, smem);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, closure_records_kernel<float>, kClosureThreads, smem);
    } else {
        e1 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, closure_band_kernel<double>, kClosureThreads, smem);
        e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, closure_records_kernel<double>, kClosureThreads, smem);
    }
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGetLastError();
        return 4;
    }
    const int n = a < b ? a : b;
    return n > 0 ? n : 1;
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
__global__ void convert_kernel(const A* __restrict__ src, B* __restrict__ dst, long long n, double scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (B)((double)src[i] * scale);
}

void launch_convert(const void* src, int src_fp32, void* dst, int dst_fp32, long long n, cudaStream_t s, double scale) {
    const long long g = (n + 255) / 256;
    const int grid = (int)(g < 8192 ? (g > 0 ? g : 1) : 8192);
    if (src_fp32 && !dst_fp32)
        convert_kernel<float, double><<<grid, 256, 0, s>>>((const float*)src, (double*)dst, n, scale);
    else if (!src_fp32 && dst_fp32)
        convert_kernel<double, float><<<grid, 256, 0, s>>>((const double*)src, (float*)dst, n, scale);
    else if (src_fp32)
        convert_kernel<float, float><<<grid, 256, 0, s>>>((const float*)src, (float*)dst, n, scale);
    else
        convert_kernel<double, double><<<grid, 256, 0, s>>>((const double*)src, (double*)dst, n, scale);
}

template void launch_ca<float>(const double*, const void*, double*, int, int, cudaStream_t, double*);
template void launch_ca<double>(const double*, const void*, double*, int, int, cudaStream_t, double*);
template void launch_dens_from_sums<float>(const double*, float*, long long, cudaStream_t);
template void launch_dens_from_sums<double>(const double*, double*, long long, cudaStream_t);
template void launch_moments<float>(const float*, double*, float*, void*, long long, int, const double*, const MomSet&,
                                    cudaStream_t);
template void launch_moments<double>(const double*, double*, double*, void*, long long, int, const double*,
                                     const MomSet&, cudaStream_t);
template void launch_closure<float>(const ClosureArgs&, const MomSet&, int, int, size_t, cudaStream_t);
template void launch_closure<double>(const ClosureArgs&, const MomSet&, int, int, size_t, cudaStream_t);
template void launch_closure_batch<float>(const ClosureArgs&, const MomSet&, int, size_t, cudaStream_t);
template void launch_closure_batch<double>(const ClosureArgs&, const MomSet&, int, size_t, cudaStream_t);

}  // namespace fdlb
