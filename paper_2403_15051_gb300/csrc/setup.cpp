// Host-side set-up of the FDLB solver: quadrature rules, derivative matrices, equilibrium
// recurrences, radial grid, Fischer-Methfessel weights and parameter checks.
//
// Quadrature (Sec. III.A): full-range Gauss-Hermite rules from the Jacobi matrix of the
// probabilists' Hermite recurrence; half-range rules from recurrence coefficients obtained by
// the discretised Stieltjes procedure on a composite Gauss-Legendre discretisation of
// omega(x) = exp(-x^2/2)/sqrt(2 pi) on [0, 40] (320 panels of 20 points).  Nodes are the eigenvalues of the Jacobi
// matrix found by Sturm-sequence bisection; weights are the Christoffel numbers
// 1 / sum_l p_l(x)^2 of the orthonormal polynomials.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace fdlb {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kSqrt2Pi = 2.50662827463100050242;

// Number of eigenvalues of the symmetric tridiagonal matrix (diag a, squared off-diagonal b2,
// b2[k] couples rows k-1 and k) that are smaller than x (Sturm count of the LDL^T pivots).
int sturm_count(const std::vector<double>& a, const std::vector<double>& b2, double x) {
    int cnt = 0;
    double d = 1.0;
    for (size_t k = 0; k < a.size(); ++k) {
        d = (a[k] - x) - (k ? b2[k] / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Eigenvalues (ascending) of the Jacobi matrix by bisection.
std::vector<double> tridiag_eigenvalues(const std::vector<double>& a, const std::vector<double>& b2) {
    const int n = (int)a.size();
    double lo = 1e300, hi = -1e300;
    for (int k = 0; k < n; ++k) {
        double r = (k ? std::sqrt(b2[k]) : 0.0) + (k + 1 < n ? std::sqrt(b2[k + 1]) : 0.0);
        lo = std::min(lo, a[k] - r);
        hi = std::max(hi, a[k] + r);
    }
    std::vector<double> ev(n);
    for (int k = 0; k < n; ++k) {
        double l = lo, h = hi;
        for (int it = 0; it < 200; ++it) {
            double m = 0.5 * (l + h);
            if (m <= l || m >= h) break;
            if (sturm_count(a, b2, m) >= k + 1) h = m; else l = m;
        }
        ev[k] = 0.5 * (l + h);
    }
    return ev;
}

// Values p_0..p_{n-1} of the orthonormal polynomials at x (p_0 = 1/sqrt(beta_0)).
void orthonormal_values(const std::vector<double>& alpha, const std::vector<double>& beta, int n,
                        double x, double* out) {
    out[0] = 1.0 / std::sqrt(beta[0]);
    if (n > 1) out[1] = (x - alpha[0]) * out[0] / std::sqrt(beta[1]);
    for (int l = 1; l + 1 < n; ++l)
        out[l + 1] = ((x - alpha[l]) * out[l] - std::sqrt(beta[l]) * out[l - 1]) / std::sqrt(beta[l + 1]);
}

void gauss_rule_from_recurrence(const std::vector<double>& alpha, const std::vector<double>& beta, int Q,
                                std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> a(alpha.begin(), alpha.begin() + Q), b2(Q, 0.0);
    for (int k = 1; k < Q; ++k) b2[k] = beta[k];
    x = tridiag_eigenvalues(a, b2);
    w.assign(Q, 0.0);
    std::vector<double> pv(Q);
    for (int i = 0; i < Q; ++i) {
        orthonormal_values(alpha, beta, Q, x[i], pv.data());
        double s = 0.0;
        for (int l = 0; l < Q; ++l) s += pv[l] * pv[l];
        w[i] = 1.0 / s;
    }
}

// m-point Gauss-Legendre rule on [-1, 1] by Newton iteration on P_m.
void gauss_legendre(int m, std::vector<double>& x, std::vector<double>& w) {
    x.assign(m, 0.0);
    w.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (m + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

double hermite_he(int l, double x) {
    double h0 = 1.0, h1 = x;
    if (l == 0) return h0;
    for (int k = 1; k < l; ++k) {
        double h2 = x * h1 - k * h0;
        h0 = h1;
        h1 = h2;
    }
    return h1;
}

}  // namespace

// ------------------------------------------------------------------------ quadrature rules
void full_range_rule(int Q, std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> alpha(Q + 1, 0.0), beta(Q + 1, 0.0);
    beta[0] = 1.0;
    for (int k = 1; k <= Q; ++k) beta[k] = k;
    gauss_rule_from_recurrence(alpha, beta, Q, x, w);
}

void half_range_recurrence(int n, std::vector<double>& alpha, std::vector<double>& beta) {
    // composite Gauss-Legendre discretisation of omega on [0, 40]: 320 panels x 20 points (panels
    // of 1/8: the recurrence coefficients agree with a 600-digit moment-based computation to 1e-15
    // up to order 101; 80 panels left a 1e-3 error at that order)
    std::vector<double> gx, gw;
    gauss_legendre(20, gx, gw);
    const int panels = 320;
    const double h = 40.0 / panels;
    std::vector<double> t, W;
    for (int p = 0; p < panels; ++p)
        for (size_t i = 0; i < gx.size(); ++i) {
            double x = h * (p + 0.5 * (gx[i] + 1.0));
            double om = std::exp(-0.5 * x * x) / kSqrt2Pi;
            t.push_back(x);
            W.push_back(0.5 * h * gw[i] * om);
        }
    const size_t M = t.size();
    alpha.assign(n, 0.0);
    beta.assign(n, 0.0);
    std::vector<double> qprev(M, 0.0), q(M), r(M);
    double mass = 0.0;
    for (size_t s = 0; s < M; ++s) mass += W[s];
    beta[0] = mass;
    for (size_t s = 0; s < M; ++s) q[s] = 1.0 / std::sqrt(mass);
    double bk = 0.0;
    for (int k = 0; k < n; ++k) {
        double a = 0.0;
        for (size_t s = 0; s < M; ++s) a += W[s] * t[s] * q[s] * q[s];
        alpha[k] = a;
        if (k + 1 == n) break;
        double nr = 0.0;
        for (size_t s = 0; s < M; ++s) {
            r[s] = (t[s] - a) * q[s] - bk * qprev[s];
            nr += W[s] * r[s] * r[s];
        }
        double bnext = std::sqrt(nr);
        beta[k + 1] = nr;
        for (size_t s = 0; s < M; ++s) {
            qprev[s] = q[s];
            q[s] = r[s] / bnext;
        }
        bk = bnext;
    }
}

void half_range_rule(int Q, std::vector<double>& x, std::vector<double>& w, std::vector<double>& alpha,
                     std::vector<double>& beta) {
    half_range_recurrence(Q + 1, alpha, beta);
    gauss_rule_from_recurrence(alpha, beta, Q, x, w);
}

AxisRule make_axis(int Q, bool half) {
    AxisRule ax;
    ax.Q = Q;
    ax.half = half;
    if (!half) {
        full_range_rule(Q, ax.p, ax.w);
        ax.alpha.assign(Q + 1, 0.0);
        ax.beta.assign(Q + 1, 0.0);
        ax.beta[0] = 1.0;
        for (int k = 1; k <= Q; ++k) ax.beta[k] = k;
    } else {
        std::vector<double> x, w;
        half_range_rule(Q, x, w, ax.alpha, ax.beta);
        ax.p.resize(2 * Q);
        ax.w.resize(2 * Q);
        for (int i = 0; i < Q; ++i) {
            ax.p[i] = x[i];
            ax.p[Q + i] = -x[i];
            ax.w[i] = ax.w[Q + i] = w[i];
        }
    }
    return ax;
}

// ------------------------------------------------------------------------ K matrices
// Half-range d f/dp in the printed form of Sec. III.B:
// K_ii' = w_i s_i { [s_i = s_i'] sum_{l=0}^{Q-2} h_l(|p_i'|) [ h_l(0)/sqrt(2pi) sum_{s=l+1}^{Q-1}
//          h_s(0) h_s(|p_i|) - (h_ll / h_{l+1,l+1}) h_{l+1}(|p_i|) ] - Phi_0(|p_i|) Phi_0(|p_i'|)/(2 sqrt(2pi)) },
// Phi_0(x) = sum_{l<Q} h_l(0) h_l(x), and h_ll / h_{l+1,l+1} = sqrt(beta_{l+1}).
void k_half_matrix(const AxisRule& ax, std::vector<double>& K) {
    const int Q = ax.Q, n = 2 * Q;
    std::vector<double> H((size_t)Q * n), h0(Q), Phi(n, 0.0), pv(Q);
    orthonormal_values(ax.alpha, ax.beta, Q, 0.0, h0.data());
    for (int i = 0; i < n; ++i) {
        orthonormal_values(ax.alpha, ax.beta, Q, std::fabs(ax.p[i]), pv.data());
        for (int l = 0; l < Q; ++l) {
            H[(size_t)l * n + i] = pv[l];
            Phi[i] += h0[l] * pv[l];
        }
    }
    K.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double si = ax.p[i] > 0 ? 1.0 : -1.0;
        for (int j = 0; j < n; ++j) {
            const double sj = ax.p[j] > 0 ? 1.0 : -1.0;
            double acc = 0.0;
            if (si == sj) {
                for (int l = 0; l + 1 < Q; ++l) {
                    double tail = 0.0;
                    for (int s = l + 1; s < Q; ++s) tail += h0[s] * H[(size_t)s * n + i];
                    double inner = h0[l] / kSqrt2Pi * tail - std::sqrt(ax.beta[l + 1]) * H[(size_t)(l + 1) * n + i];
                    acc += H[(size_t)l * n + j] * inner;
                }
            }
            acc -= Phi[i] * Phi[j] / (2.0 * kSqrt2Pi);
            K[(size_t)i * n + j] = ax.w[i] * si * acc;
        }
    }
}

// Full-range d (f p)/dp, Eq. force2:  K_ii' = -w_i sum_{l=0}^{Q-2} He_{l+1}(p_i)
// [He_{l+1}(p_i') + l He_{l-1}(p_i')] / l!
void k2_full_matrix(const AxisRule& ax, std::vector<double>& K) {
    const int Q = ax.Q;
    K.assign((size_t)Q * Q, 0.0);
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            double acc = 0.0, fact = 1.0;
            for (int l = 0; l + 1 < Q; ++l) {
                if (l > 0) fact *= l;
                double right = hermite_he(l + 1, ax.p[j]) + (l > 0 ? l * hermite_he(l - 1, ax.p[j]) : 0.0);
                acc += hermite_he(l + 1, ax.p[i]) * right / fact;
            }
            K[(size_t)i * Q + j] = -ax.w[i] * acc;
        }
}

// ------------------------------------------------------------------------ equilibria
// Full range (Sec. III.C): g_k = w_k sum_{l<=N} He_l(p_k) e_l / l!, e_l = E[He_l(X)] for
// X ~ N(u, T), from e_{l+1} = u e_l + l (T - 1) e_{l-1}.
void g_full_host(const AxisRule& ax, int N, double u, double T, double* g) {
    double e[kMaxQ + 2];
    e[0] = 1.0;
    if (N >= 1) e[1] = u;
    for (int l = 1; l < N; ++l) e[l + 1] = u * e[l] + l * (T - 1.0) * e[l - 1];
    for (int k = 0; k < ax.Q; ++k) {
        double acc = 0.0, fact = 1.0;
        for (int l = 0; l <= N; ++l) {
            if (l > 0) fact *= l;
            acc += hermite_he(l, ax.p[k]) * e[l] / fact;
        }
        g[k] = ax.w[k] * acc;
    }
}

// Half range (Sec. III.C): g_k = w_k sum_{l<=N} h_l(|p_k|) e_l^{s_k}, e_l^s = int_0^inf h_l(x)
// G(s x) dx for G the N(u, T) density.  With v = s u and the identity
// int_0^inf x h G = v int h G + T int h' G + T h(0) G_v(0):
//   e_0 = h_0 (1 + erf(v / sqrt(2T))) / 2,
//   b_{l+1} e_{l+1} = (v - alpha_l) e_l + (T - 1) b_l e_{l-1}
//                     + T h_l(0) [G_v(0) - sum_{k<l} h_k(0) e_k / sqrt(2 pi)].
void g_half_host(const AxisRule& ax, int N, double u, double T, double* g) {
    const int Q = ax.Q;
    double h0[kMaxQ + 2], pv[kMaxQ + 2];
    orthonormal_values(ax.alpha, ax.beta, N + 1, 0.0, h0);
    for (int half = 0; half < 2; ++half) {
        const double v = half == 0 ? u : -u;
        double e[kMaxQ + 2];
        const double G0 = std::exp(-v * v / (2.0 * T)) / std::sqrt(2.0 * kPi * T);
        e[0] = h0[0] * 0.5 * (1.0 + std::erf(v / std::sqrt(2.0 * T)));
        double run = 0.0;  // sum_{k<l} h_k(0) e_k
        for (int l = 0; l < N; ++l) {
            const double bl = l ? std::sqrt(ax.beta[l]) : 0.0;
            const double em1 = l ? e[l - 1] : 0.0;
            double val = (v - ax.alpha[l]) * e[l] + (T - 1.0) * bl * em1 + T * h0[l] * (G0 - run / kSqrt2Pi);
            e[l + 1] = val / std::sqrt(ax.beta[l + 1]);
            run += h0[l] * e[l];
        }
        for (int k = 0; k < Q; ++k) {
            const int idx = half * Q + k;
            orthonormal_values(ax.alpha, ax.beta, N + 1, std::fabs(ax.p[idx]), pv);
            double acc = 0.0;
            for (int l = 0; l <= N; ++l) acc += pv[l] * e[l];
            g[idx] = ax.w[idx] * acc;
        }
    }
}

// ------------------------------------------------------------------------ physics
double chi_set(double eta) { return (2.0 - eta) / (2.0 * (1.0 - eta) * (1.0 - eta) * (1.0 - eta)); }

double viscosity(double n, double T, double chi, double sigma) {
    const double br = 2.0 * kPi / 3.0 * sigma * sigma * sigma * n;
    const double mu0 = 5.0 / (16.0 * sigma * sigma) * std::sqrt(T / kPi);
    return mu0 * (1.0 / chi + 0.8 * br + 4.0 / 25.0 * (1.0 + 12.0 / kPi) * br * br * chi);
}

double prandtl(double n, double chi, double sigma) {
    const double x = 2.0 * kPi / 3.0 * sigma * sigma * sigma * n * chi;
    const double num = 1.0 + 0.8 * x + 4.0 / 25.0 * (1.0 + 12.0 / kPi) * x * x;
    const double den = 1.0 + 1.2 * x + 9.0 / 25.0 * (1.0 + 32.0 / (9.0 * kPi)) * x * x;
    return 2.0 / 3.0 * num / den;
}

// ------------------------------------------------------------------------ grid
Grid make_grid(int geometry, double R_in, double R_out, double sigma, int N, double beta) {
    Grid g;
    g.N = N;
    g.ds = 1.0 / N;
    const double RcL = R_in + 0.5 * sigma, Lc = (R_out - R_in) - sigma;
    auto map = [&](double s, double* dR) {
        if (beta == 0.0) {
            *dR = Lc;
            return RcL + Lc * s;
        }
        const double tb = std::tanh(beta), a = beta * (2.0 * s - 1.0);
        const double ch = std::cosh(a);
        *dR = Lc * beta / (ch * ch) / tb;
        return RcL + 0.5 * Lc * (1.0 + std::tanh(a) / tb);
    };
    g.R_c.resize(N);
    g.dRds_c.resize(N);
    g.R_f.resize(N + 1);
    g.A_f.resize(N + 1);
    g.V_c.resize(N);
    g.kappa.resize(N);
    double tmp;
    for (int k = 0; k <= N; ++k) g.R_f[k] = map((double)k / N, &tmp);
    for (int i = 0; i < N; ++i) g.R_c[i] = map((i + 0.5) / N, &g.dRds_c[i]);
    for (int k = 0; k <= N; ++k) g.A_f[k] = geometry == FDLB_CYL ? g.R_f[k] : g.R_f[k] * g.R_f[k];
    for (int i = 0; i < N; ++i) {
        const double a = g.R_f[i], b = g.R_f[i + 1];
        g.V_c[i] = geometry == FDLB_CYL ? 0.5 * (b * b - a * a) : (b * b * b - a * a * a) / 3.0;
        g.kappa[i] = (g.A_f[i + 1] - g.A_f[i]) / g.V_c[i];
    }
    return g;
}

// ------------------------------------------------------------------------ FM weights
FmRule fm_rule() {
    std::vector<double> x, ww;
    gauss_legendre(kFmGL, x, ww);
    FmRule r{};
    for (int i = 0; i < kFmGL; ++i) {
        // map [-1,1] -> [0,1], then u -> (1 - cos(pi u))/2 to absorb end-point singularities
        const double s = 0.5 * (x[i] + 1.0);
        r.u[i] = 0.5 * (1.0 - std::cos(kPi * s));
        r.w[i] = 0.5 * ww[i] * 0.5 * kPi * std::sin(kPi * s);
    }
    return r;
}

int fm_band(int geometry, const Grid& g, double sigma, FMBand& b, bool weights) {
    b = FMBand();
    const int N = g.N;
    b.lo.assign(N, 0);
    std::vector<int> hi(N, 0);
    for (int i = 0; i < N; ++i) {
        const double lo_r = g.R_c[i] - sigma, hi_r = g.R_c[i] + sigma;
        int lo = 0;
        while (lo < N - 1 && g.R_f[lo + 1] <= lo_r) ++lo;
        int h = N - 1;
        while (h > 0 && g.R_f[h] >= hi_r) --h;
        b.lo[i] = lo;
        hi[i] = std::max(h, lo);
        b.width = std::max(b.width, hi[i] - lo + 1);
    }
    b.width = (b.width + 3) / 4 * 4;  // rows of 16-byte multiples (bulk copies of row extents)
    if ((long long)N * b.width > 2147483647LL) return FDLB_EINVAL;
    b.cnt.assign(N, 0);
    for (int i = 0; i < N; ++i) b.cnt[i] = std::min(b.width, (hi[i] - b.lo[i] + 1 + 3) / 4 * 4);
    if (!weights) return FDLB_OK;  // the extents alone (a handle's weights are filled on the device)
    b.W.assign((size_t)N * b.width, 0.0);
    const double norm = 3.0 / (4.0 * kPi * sigma * sigma * sigma);
    const FmRule gl = fm_rule();
    const int sph = geometry == FDLB_SPH ? 1 : 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < N; ++i) {
        const double d = g.R_c[i];
        auto U = [&](double Rp) { return fm_volume_inside(sph, sigma, d, Rp, gl); };
        double prev = U(g.R_f[b.lo[i]]);
        for (int j = b.lo[i]; j <= hi[i]; ++j) {
            const double next = U(g.R_f[j + 1]);
            b.W[(size_t)i * b.width + (j - b.lo[i])] = norm * (next - prev);
            prev = next;
        }
    }
    return FDLB_OK;
}

// ------------------------------------------------------------------------ validation
int validate_params(const fdlb_params& p) {
    if (p.geometry != FDLB_CYL && p.geometry != FDLB_SPH && p.geometry != FDLB_CYL_Z) return FDLB_EINVAL;
    const bool reduced = p.geometry == FDLB_CYL_Z;  // no third momentum axis: Q_3 = 0
    if (!(p.R_in > 0.0) || !(p.R_out > p.R_in)) return FDLB_EINVAL;
    if (p.n_cells < 8) return FDLB_EINVAL;
    if (!(p.stretch_beta >= 0.0) || p.stretch_beta > 10.0) return FDLB_EINVAL;
    const int Qs[3] = {p.Q_R, p.Q_2, p.Q_3};
    const int Ns[3] = {p.N_R, p.N_2, p.N_3};
    for (int a = 0; a < 3; ++a) {
        if (a == 2 && reduced) {
            if (Qs[a] != 0) return FDLB_EINVAL;
            continue;
        }
        if (Qs[a] < 1 || Qs[a] > (a == 0 ? kMaxQR : kMaxQ)) return FDLB_EINVAL;
        if (Ns[a] >= Qs[a] || Ns[a] > kMaxN) return FDLB_EINVAL;
    }
    if (!(p.eta0 > 0.0 && p.eta0 < 0.5)) return FDLB_EINVAL;
    if (!(p.sigma > 0.0) && !(p.Kn > 0.0)) return FDLB_EINVAL;
    if (p.chi_model != FDLB_CHI_RET_FM && p.chi_model != FDLB_CHI_SET_LOCAL) return FDLB_EINVAL;
    if (p.precision != FDLB_FP64 && p.precision != FDLB_FP32) return FDLB_EINVAL;
    if (!(p.T_wall[0] > 0.0) || !(p.T_wall[1] > 0.0)) return FDLB_EINVAL;
    if (!std::isfinite(p.u_wall[0]) || !std::isfinite(p.u_wall[1])) return FDLB_EINVAL;
    if (p.geometry == FDLB_SPH && (p.u_wall[0] != 0.0 || p.u_wall[1] != 0.0)) return FDLB_EINVAL;
    if (!std::isfinite(p.dt) || !std::isfinite(p.cfl)) return FDLB_EINVAL;
    return FDLB_OK;
}

int build_instance(const fdlb_params& p_in, const AxisRule& aR, InstanceSetup& out) {
    fdlb_params p = p_in;
    auto order = [](int N, int Q) { return N < 0 ? std::min(Q - 1, kMaxN) : N; };
    p.N_R = order(p.N_R, p.Q_R);
    p.N_2 = order(p.N_2, p.Q_2);
    p.N_3 = p.geometry == FDLB_CYL_Z ? 0 : order(p.N_3, p.Q_3);
    int rc = validate_params(p);
    if (rc) return rc;
    out.p = p;
    out.NR = p.N_R;
    out.N2 = p.N_2;
    out.N3 = p.N_3;
    const double L = p.R_out - p.R_in;
    const double chi0 = chi_set(p.eta0);
    if (p.sigma > 0.0) {
        out.sigma = p.sigma;
        out.C = L / p.sigma;
    } else {
        out.C = 1.0 / (6.0 * std::sqrt(2.0) * p.eta0 * chi0 * p.Kn);
        out.sigma = L / out.C;
    }
    if (!(out.C >= 3.0)) return FDLB_EINVAL;
    out.n0 = 6.0 * p.eta0 / (kPi * out.sigma * out.sigma * out.sigma);
    const int gbase = p.geometry == FDLB_SPH ? FDLB_SPH : FDLB_CYL;  // the reduced cylinder's grid is the cylinder's
    out.grid = make_grid(gbase, p.R_in, p.R_out, out.sigma, p.n_cells, p.stretch_beta);
    if (p.dt > 0.0) {
        out.dt = p.dt;
    } else {
        double dr = 1e300;
        for (int i = 0; i < p.n_cells; ++i) dr = std::min(dr, out.grid.R_f[i + 1] - out.grid.R_f[i]);
        double pmax = 0.0;
        for (double v : aR.p) pmax = std::max(pmax, std::fabs(v));
        const double Tmax = std::max(p.T_wall[0], p.T_wall[1]);
        const double tau = viscosity(out.n0, Tmax, chi0, out.sigma) / (out.n0 * Tmax);
        const double cfl = p.cfl > 0.0 ? p.cfl : 0.4;
        out.dt = std::min(cfl * dr / (pmax * std::sqrt(Tmax)), 0.5 * tau);
    }
    if (p.chi_model == FDLB_CHI_RET_FM) return fm_band(gbase, out.grid, out.sigma, out.band, false);
    return FDLB_OK;
}

}  // namespace fdlb

// ------------------------------------------------------------------------ host-only ABI
extern "C" {

int fdlb_quadrature(int kind, int Q, double* nodes, double* weights) try {
    if (Q < 1 || Q > 128 || !nodes || !weights) return FDLB_EINVAL;
    if (kind != FDLB_QUAD_FULL && kind != FDLB_QUAD_HALF) return FDLB_EINVAL;
    fdlb::AxisRule ax = fdlb::make_axis(Q, kind == FDLB_QUAD_HALF);
    std::memcpy(nodes, ax.p.data(), ax.p.size() * sizeof(double));
    std::memcpy(weights, ax.w.data(), ax.w.size() * sizeof(double));
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_derivative_matrix(int kind, int Q, double* K) try {
    if (Q < 1 || Q > 128 || !K) return FDLB_EINVAL;
    std::vector<double> M;
    if (kind == FDLB_QUAD_HALF) {
        fdlb::k_half_matrix(fdlb::make_axis(Q, true), M);
    } else if (kind == FDLB_QUAD_FULL) {
        fdlb::k2_full_matrix(fdlb::make_axis(Q, false), M);
    } else {
        return FDLB_EINVAL;
    }
    std::memcpy(K, M.data(), M.size() * sizeof(double));
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_physical_parameters(double Kn, double eta0, double L, double* C, double* sigma, double* n0) {
    if (!(Kn > 0.0) || !(eta0 > 0.0 && eta0 < 0.5) || !(L > 0.0)) return FDLB_EINVAL;
    const double c = 1.0 / (6.0 * std::sqrt(2.0) * eta0 * fdlb::chi_set(eta0) * Kn);
    const double s = L / c;
    if (C) *C = c;
    if (sigma) *sigma = s;
    if (n0) *n0 = 6.0 * eta0 / (fdlb::kPi * s * s * s);
    return FDLB_OK;
}

int fdlb_grid(int geometry, double R_in, double R_out, double sigma, int n_cells, double beta, double* R_c,
              double* R_f, double* V, double* kappa) try {
    if ((geometry != FDLB_CYL && geometry != FDLB_SPH) || n_cells < 8 || !(R_out - R_in > sigma) || !(sigma > 0))
        return FDLB_EINVAL;
    fdlb::Grid g = fdlb::make_grid(geometry, R_in, R_out, sigma, n_cells, beta);
    if (R_c) std::memcpy(R_c, g.R_c.data(), n_cells * sizeof(double));
    if (R_f) std::memcpy(R_f, g.R_f.data(), (n_cells + 1) * sizeof(double));
    if (V) std::memcpy(V, g.V_c.data(), n_cells * sizeof(double));
    if (kappa) std::memcpy(kappa, g.kappa.data(), n_cells * sizeof(double));
    return FDLB_OK;
} FDLB_HOST_CATCH

int fdlb_fm_weights(int geometry, double R_in, double R_out, double sigma, int n_cells, double beta, double* W) try {
    if ((geometry != FDLB_CYL && geometry != FDLB_SPH) || n_cells < 8 || !(R_out - R_in > sigma) || !(sigma > 0) || !W)
        return FDLB_EINVAL;
    fdlb::Grid g = fdlb::make_grid(geometry, R_in, R_out, sigma, n_cells, beta);
    fdlb::FMBand b;
    const int rc = fdlb::fm_band(geometry, g, sigma, b);
    if (rc) return rc;
    std::memset(W, 0, sizeof(double) * (size_t)n_cells * n_cells);
    for (int i = 0; i < n_cells; ++i)
        for (int k = 0; k < b.width && b.lo[i] + k < n_cells; ++k)
            W[(size_t)i * n_cells + b.lo[i] + k] = b.W[(size_t)i * b.width + k];
    return FDLB_OK;
} FDLB_HOST_CATCH

}  // extern "C"
