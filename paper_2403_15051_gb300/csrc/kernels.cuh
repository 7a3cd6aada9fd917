// Device kernels of the FDLB step (sm_103a).
//
// Data layout in HBM (per instance, instances packed one after another):
//   f[cell][k][i][j]   T = float or double; i: 2 Q_R radial momenta, j: Q_2, k: Q_3.
//                      The passive-or-outermost axis k is outermost inside a cell so that a
//                      momentum slice (a range of k) is one contiguous run per cell.
//   sums[cell][slice][13]  FP64 raw quadrature sums (Eq. mom_quad) of the populations,
//                      one partial per momentum slice (summed by the consumer in a fixed order);
//                      for FP32 populations also as double-float pairs (float2), the closure's input.
//   dens[cell][slice]  the slice densities (sum 0) in the populations' precision, read by the
//                      FM band sums.
//   ca[cell][12]       FP64 closure record: n, u1, u2, u3, T, q1, q2, q3, P12, chi, nbar, 0.
//
// Per SSP-RK3 stage (Sec. III) two launches:
//   closure_kernel  - per cell, once: n, u, T, q from the sums (Eq. macro_def), the Fischer-
//                     Methfessel density nbar (Eq. fm) over the stored band, chi (Eq. chi /
//                     chi_ret), the J1 gradients (Eq. j1), tau (Eq. tau), Pr (Eq. prandtl) and the
//                     discrete equilibria (Sec. III.C) -> a per-cell record; the wall densities.
//   stream_kernel   - per (tile of cells) x (momentum slice), per population: WENO5 radial advection
//                     with metric factors (Sec. II.B/C), the curvature force with the K matrices
//                     (Sec. III.B), the Shakhov + J1 collision, the RK combination, the store, and
//                     the raw sums of the new populations (epilogue).
// Or, optionally, whole steps in one cooperative launch (step_kernel.cuh): the same closure and
// stage code per tile, grid barriers between stages.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdlb {

constexpr int kSums = 13;
constexpr int kCA = 12;
constexpr int kNmom = 9;           // columns of the moments query (FDLB_NMOM)
constexpr int kGeo = 6;            // per cell: R_c, 1/(dR/ds), A_+/V, A_-/V, force factor, V
constexpr int kMaxE = 8;           // expansion coefficients per axis (N <= 7)
constexpr int kMaxRed = 32;        // warps per block
constexpr int kClosureCells = 28;  // own cells per closure item (reach: 32 cells)
constexpr int kWallParts = 8;      // closure work items per wall (parts of the momentum set)

struct InstDev {
    int n_cells;
    int cell_off;                  // first global cell index of this instance
    long long f_off;               // first element of this instance in the f buffers
    int band_off;                  // first element of this instance's FM band
    int band_w;                    // entries per band row (0: local chi)
    int chi_local;                 // 1: chi at the local density
    int geometry;
    double sigma, bfac, etafac;    // sigma, 2 pi sigma^3 / 3, pi sigma^3 / 6
    double dt, ds;
    double nw_den[2];              // sum over incoming momenta of |p_R| g_wall
    double nw_iden[2];             // 1 / nw_den
    // FP32 copies for FP32 populations
    float f_sigma, f_bfac, f_etafac, f_ids, f_dt;
    float f_nw_iden[2];
};

struct MomSet {
    int nR, n2, n3, Np;            // axis sizes, momenta per cell
    int NR, N2, N3;                // expansion orders
    int slices, KS, Ms;            // momentum slices, k values per slice, momenta per slice
    int reduced;                   // cylinder with p_z integrated out: k = 0 phi, k = 1 chi
    // offsets into the FP64 table buffer
    int o_pR, o_wR, o_p2, o_w2, o_p3, o_w3, o_KR, o_K2, o_K3, o_GR, o_G2, o_G3, o_ha, o_hb, o_h0;
};

struct StageArgs {
    const void* f_in;
    const void* f_n;
    void* f_out;
    const void* rec;               // per-cell collision records of f_in (T), [cell][rec_stride]
    int rec_stride;
    const void* nwp;               // [instance][2][kWallParts] outgoing wall fluxes of f_in (T)
    double* sums_out;              // raw sums of f_out
    void* sumsw_out;               // the same as double-float pairs (FP32 populations), [cell][slice][13]
    void* dens_out;                // per-slice densities of f_out (T), [cell][slice]
    const int4* items;             // (instance, first cell, cells, slice)
    const int* n_items;
    const InstDev* inst;
    const double* tab;
    const void* tabT;              // the same tables in T
    const void* geoT;              // [cell][kGeo] in T
    const void* gwT;               // [instance][2][nR + n2 + n3] wall Maxwellians per axis, in T
    int* err;
    double a, b;                   // f_out = a f_n + b (f_in + dt L(f_in))
    float fa, fb;                  // the same in FP32
    int wall_parts;
    int mode;                      // 0: RK stage; 1: write L(f_in) to f_out
    int B;                         // cells per tile
    int use_bulk;                  // stage the tile with cp.async.bulk
    int programmatic;              // launched with programmatic stream serialization
    int mma;                       // K^h contraction on the tensor cores (FP32 compile-time shapes)
    int tx_extra;                  // test hook: bytes the staged-copy barrier waits for beyond the copy
    const void* krf;               // K^h f of f_in from the contraction kernel (T, layout of f), or
                                   // null: the stage contracts from the K^h table in shared memory
    const void* k3f;               // sphere: K_3 f of f_in (T, layout of f) when the momenta are
                                   // sliced along p_3, or null: contracted from the staged rows
};

// A warp's job in the batch closure's band kernel, formed once per work list on the host: two
// band rows (A, B) of one instance, or (kmaxA < 0) part kmaxB of the outgoing flux through wall
// -1 - kmaxA of instance q.  wA, wB: first band element of each row; dA, dB: global cell of each
// row's first column; kmaxA, kmaxB: the rows' summed extents (0: no row B); gc: global cell of A.
struct BandPair {
    long long wA, wB, dA, dB;
    int kmaxA, kmaxB, gc, q;
};

struct ClosureArgs {
    const double* sums;
    const void* sumsw;             // the raw sums as double-float pairs (FP32 populations)
    const void* dens;              // per-slice densities (T), [cell][slice], for the FM bands
    const void* f_in;              // populations (T), for the wall fluxes
    void* cw;                      // [cell][2] chi and nbar of the stage (T), for the queries
    void* rec;                     // per-cell collision records (T)
    int rec_stride;
    void* nwp;                     // [instance][2][kWallParts] outgoing wall fluxes (T)
    const int4* items;             // (instance, first cell, cells, 0) or (instance, -, part, 1 + side)
    const int* n_items;
    const InstDev* inst;
    const void* band;              // FM band values (T)
    const int* band_lo;            // per global cell: first column, stored extent
    const void* tabT;              // the tables in the populations' precision
    const void* geoT;              // [cell][kGeo] in T
    int slices;
    int max_union;                 // capacity of the shared density buffer
    int wall_parts;
    int wst_elems;                 // capacity of the staged band rows (elements)
    int programmatic;              // launched with programmatic stream serialization
    int* err;                      // set when a bulk copy never completes
    const BandPair* pairs;         // batch form: the band kernel's jobs
    const int* n_pairs;
};

struct StepArgs {
    StageArgs st;                  // the stage fields; buffers and coefficients set per stage
    ClosureArgs cl;                // the closure fields; sums, densities, populations set per stage
    void* f[3];                    // f^n (and f^{n+1}), f1, f2
    double* sums[3];
    void* sumsw[3];
    void* dens[3];
    unsigned int* bar;             // grid barrier counter (zero at launch)
    int n_steps;
    int clo_off;                   // byte offset of the closure's shared memory
    int bar_extra;                 // test hook: arrivals every grid barrier waits for beyond the grid
};

}  // namespace fdlb
