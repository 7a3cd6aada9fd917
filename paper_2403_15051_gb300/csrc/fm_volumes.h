// Volumes behind the Fischer-Methfessel weights (Eq. fm, App. A), shared by the host set-up
// (g++) and the device kernel that fills the weights of a handle's bands (nvcc): the same
// arithmetic on both sides.
//
// W_ij = (3 / (4 pi sigma^3)) [U_i(R_{j+1}) - U_i(R_j)], with U_i(R') the volume of the ball of
// radius sigma centred at the cell centre R_i that lies inside radius R' (the sphere of radius R'
// for the spherical geometry, the infinite cylinder of radius R' for the cylindrical one).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define FDLB_HD __host__ __device__
#else
#define FDLB_HD
#endif

namespace fdlb {

constexpr int kFmGL = 24;  // points per panel of the cylinder quadrature

// The cosine-mapped Gauss-Legendre rule on [0, 1] of the cylinder quadrature: u = (1 - cos(pi s))/2
// absorbs the square-root end-point behaviour of the integrand.
struct FmRule {
    double u[kFmGL], w[kFmGL];
};

constexpr double kFmPi = 3.14159265358979323846;

FDLB_HD inline double fm_min(double a, double b) { return a < b ? a : b; }
FDLB_HD inline double fm_max(double a, double b) { return a > b ? a : b; }

// Volume common to a ball of radius r centred at distance d from the origin and the ball of
// radius Rp centred at the origin (App. A lens formula plus the nested/disjoint cases).
FDLB_HD inline double sphere_volume_inside(double r, double d, double Rp) {
    if (Rp <= 0.0) return 0.0;
    if (d >= r + Rp) return 0.0;
    if (d <= fabs(r - Rp)) {
        const double m = fm_min(r, Rp);
        return 4.0 / 3.0 * kFmPi * m * m * m;
    }
    return kFmPi * (r + Rp - d) * (r + Rp - d) * (d * d + 2 * d * Rp - 3 * Rp * Rp + 2 * d * r + 6 * r * Rp - 3 * r * r) /
           (12.0 * d);
}

// Area common to a disc of radius r at distance d from the origin and the disc of radius Rp
// centred at the origin.
FDLB_HD inline double disc_area_inside(double r, double d, double Rp) {
    if (r <= 0.0 || Rp <= 0.0) return 0.0;
    if (d >= r + Rp) return 0.0;
    if (d <= fabs(Rp - r)) {
        const double m = fm_min(r, Rp);
        return kFmPi * m * m;
    }
    double c1 = (d * d + r * r - Rp * Rp) / (2.0 * d * r);
    double c2 = (d * d + Rp * Rp - r * r) / (2.0 * d * Rp);
    c1 = fm_max(-1.0, fm_min(1.0, c1));
    c2 = fm_max(-1.0, fm_min(1.0, c2));
    const double k = (-d + r + Rp) * (d + r - Rp) * (d - r + Rp) * (d + r + Rp);
    return r * r * acos(c1) + Rp * Rp * acos(c2) - 0.5 * sqrt(fm_max(k, 0.0));
}

// Volume common to a ball (radius r, centre at distance d from the axis) and the infinite
// cylinder of radius Rp: 2 int_0^{pi/2} A(r cos t, d, Rp) r cos t dt, split where r cos t crosses
// |Rp - d| and Rp + d.
FDLB_HD inline double cylinder_volume_inside(double r, double d, double Rp, const FmRule& gl) {
    if (Rp <= 0.0) return 0.0;
    if (d >= r + Rp) return 0.0;
    if (d + r <= Rp) return 4.0 / 3.0 * kFmPi * r * r * r;
    double edges[4] = {0.0, 0.0, 0.0, 0.5 * kFmPi};
    const double b1 = fabs(Rp - d), b2 = Rp + d;
    const double t1 = (b1 > 0.0 && b1 < r) ? acos(b1 / r) : 0.0;
    const double t2 = (b2 > 0.0 && b2 < r) ? acos(b2 / r) : 0.0;
    edges[1] = fm_min(t1, t2);
    edges[2] = fm_max(t1, t2);
    double total = 0.0;
    for (int p = 0; p < 3; ++p) {
        const double a = edges[p], L = edges[p + 1] - edges[p];
        if (L <= 0.0) continue;
        for (int i = 0; i < kFmGL; ++i) {
            const double t = a + L * gl.u[i];
            const double rc = r * cos(t);
            total += 2.0 * L * gl.w[i] * disc_area_inside(rc, d, Rp) * rc;
        }
    }
    return total;
}

// U_i(R') of the ball of radius sigma centred at d = R_i (geometry: 1 sphere, else cylinder).
FDLB_HD inline double fm_volume_inside(int sphere, double sigma, double d, double Rp, const FmRule& gl) {
    const double full = 4.0 / 3.0 * kFmPi * sigma * sigma * sigma;
    if (d + sigma <= Rp) return full;
    if (Rp <= d - sigma) return 0.0;
    return sphere ? sphere_volume_inside(sigma, d, Rp) : cylinder_volume_inside(sigma, d, Rp, gl);
}

}  // namespace fdlb
