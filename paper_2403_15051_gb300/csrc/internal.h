// Internal declarations shared by the host set-up (setup.cpp) and the CUDA translation
// unit (fdlb.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/fdlb.h"
#include "fm_volumes.h"

// Handlers of the function-try-blocks around the C-ABI entry points: the host side keeps its
// tables in std::vectors, and a failed host allocation is reported as FDLB_ENOMEM, so no C++
// exception leaves the C ABI.
#define FDLB_HOST_CATCH                         \
    catch (const std::bad_alloc&) {             \
        return FDLB_ENOMEM;                     \
    }                                           \
    catch (const std::length_error&) {          \
        return FDLB_ENOMEM;                     \
    }

namespace fdlb {


constexpr int kMaxQ = 24;          // largest full-range quadrature order (the two homogeneous axes)
constexpr int kMaxQR = 100;        // largest half-range order of the radial axis (2 kMaxQR nodes)
constexpr int kMaxN = 7;           // largest equilibrium expansion order handled on the device
constexpr int kNumSums = 13;       // raw quadrature sums per cell (Eq. mom_quad)
constexpr int kCARecord = 12;      // per-cell closure record written by the closure kernel

// ------------------------------------------------------------------ quadrature / tables
struct AxisRule {
    int Q = 0;                     // order
    bool half = false;             // half-range (2Q nodes) or full-range (Q nodes)
    std::vector<double> p, w;      // nodes and weights in the ABI order
    std::vector<double> alpha, beta; // recurrence coefficients (half range: beta[0] = 1/2)
};

// Full-range Gauss-Hermite rule: Q nodes ascending, weights sum to 1.
void full_range_rule(int Q, std::vector<double>& x, std::vector<double>& w);
// Half-range recurrence coefficients alpha[0..n-1], beta[0..n-1] by the discretised
// Stieltjes procedure; beta[0] = 1/2.
void half_range_recurrence(int n, std::vector<double>& alpha, std::vector<double>& beta);
// Half-range rule: positive nodes ascending and their weights (sum 1/2).
void half_range_rule(int Q, std::vector<double>& x, std::vector<double>& w,
                     std::vector<double>& alpha, std::vector<double>& beta);
AxisRule make_axis(int Q, bool half);

// Derivative matrices of Sec. III.B (row-major).
void k_half_matrix(const AxisRule& ax, std::vector<double>& K);   // d f/dp, 2Q x 2Q
void k2_full_matrix(const AxisRule& ax, std::vector<double>& K);  // d (f p)/dp, Q x Q

// Host evaluation of the per-axis equilibrium vectors (same recurrences as the device).
void g_full_host(const AxisRule& ax, int N, double u, double T, double* g);
void g_half_host(const AxisRule& ax, int N, double u, double T, double* g);

// ------------------------------------------------------------------ physics helpers
double chi_set(double eta);
double viscosity(double n, double T, double chi, double sigma);
double prandtl(double n, double chi, double sigma);

// ------------------------------------------------------------------ grid and FM weights
struct Grid {
    int N = 0;
    double ds = 0;
    std::vector<double> R_c, R_f, dRds_c, A_f, V_c, kappa;
};
Grid make_grid(int geometry, double R_in, double R_out, double sigma, int N, double beta);

struct FMBand {
    int width = 0;                 // stored entries per row
    std::vector<int> lo;           // first column of each row
    std::vector<int> cnt;          // stored nonzero extent of each row (a multiple of 4, <= width)
    std::vector<double> W;         // [N][width], zero padded
};
// Fischer-Methfessel weights of every cell over the cells its ball reaches (Eq. fm, App. A):
// the extents (first column, stored extent, width) and, when `weights`, the weights themselves
// (a handle fills them on the device, fill_fm_weights, with the same arithmetic).
// FDLB_EINVAL, before the weights are allocated, when the band would hold more than 2^31 - 1
// entries (the device tables index it with 32-bit offsets).
int fm_band(int geometry, const Grid& g, double sigma, FMBand& b, bool weights = true);
// The quadrature rule of the cylinder volumes.
FmRule fm_rule();

// ------------------------------------------------------------------ validated instance
struct InstanceSetup {
    fdlb_params p{};
    int NR = 0, N2 = 0, N3 = 0;    // expansion orders in use
    double C = 0, sigma = 0, n0 = 0, dt = 0;
    Grid grid;
    FMBand band;
};

// Validates p and fills the derived quantities (sigma, n0, dt, grid, FM band).
int build_instance(const fdlb_params& p, const AxisRule& aR, InstanceSetup& out);
int validate_params(const fdlb_params& p);

}  // namespace fdlb
