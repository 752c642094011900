// Host FP64 quadrature for the plan (Sec. 4, eq. approxG; Sec. 4.1).
//
// * |q| rule: N_rho-point Gauss-Legendre on [0, R], nodes ascending.
// * qhat rule: the spherical designs of the paper are not available; M = 12 uses the
//   icosahedron (a spherical 5-design, equal weights), M = 2n^2 (or n^2) a product of
//   n Gauss-Legendre points in cos(theta) and 2n (or n) azimuths 2 pi (b + 1/2)/n_phi;
//   the caller may pass its own rule instead.
// * terms p = i*M + j (radial index i major), c_p = w_i w_j r_i^gamma r_i^2 (eq. approxG).
// * angular kernel constants and the part-I moments A1, A2, A3 over [0, eps] (Sec. 4.1).
// * part-II theta rule per radial node: composite Gauss-Legendre on [eps, pi].
#include <cmath>
#include <vector>

#include "bz_internal.h"

namespace bz {

// Gauss-Legendre by Newton iteration on the three-term recurrence of P_n.
int gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        // descending guess cos(pi (i + 3/4) / (n + 1/2)); stored ascending below
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // one more evaluation at the converged node for the weight
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = pk;
                }
                if (n == 1) { p1 = z; p0 = 1.0; }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        int j = n - 1 - i;
        x[j] = 0.5 * (b - a) * z + 0.5 * (b + a);
        w[j] = 0.5 * (b - a) * 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return n;
}

static void icosahedron(std::vector<double> &xyz, std::vector<double> &w) {
    const double phi = 0.5 * (1.0 + std::sqrt(5.0));
    const double nrm = std::sqrt(1.0 + phi * phi);
    xyz.clear();
    for (int a = 0; a < 2; ++a) {
        double s1 = a ? 1.0 : -1.0;
        for (int b = 0; b < 2; ++b) {
            double s2 = b ? 1.0 : -1.0;
            const double v[3][3] = {{0.0, s1, s2 * phi}, {s1, s2 * phi, 0.0}, {s2 * phi, 0.0, s1}};
            for (int c = 0; c < 3; ++c)
                for (int d = 0; d < 3; ++d) xyz.push_back(v[c][d] / nrm);
        }
    }
    w.assign(12, 4.0 * M_PI / 12.0);
}

static bool product_rule(int M, std::vector<double> &xyz, std::vector<double> &w) {
    int nt = 0, np = 0;
    int n = (int)std::lround(std::sqrt(M / 2.0));
    if (n > 0 && 2 * n * n == M) { nt = n; np = 2 * n; }
    else {
        n = (int)std::lround(std::sqrt((double)M));
        if (n > 0 && n * n == M) { nt = n; np = n; }
        else return false;
    }
    std::vector<double> ct, wt;
    gauss_legendre(nt, -1.0, 1.0, ct, wt);
    xyz.clear();
    w.clear();
    for (int a = 0; a < nt; ++a) {
        double st = std::sqrt(1.0 - ct[a] * ct[a]);
        for (int b = 0; b < np; ++b) {
            double ph = 2.0 * M_PI * (b + 0.5) / np;
            xyz.push_back(st * std::cos(ph));
            xyz.push_back(st * std::sin(ph));
            xyz.push_back(ct[a]);
            w.push_back(wt[a] * 2.0 * M_PI / np);
        }
    }
    return true;
}

bz_status build_terms(Plan &pl, const double *sphere_xyz, const double *sphere_w) {
    std::vector<double> r, wr, q, wq;
    gauss_legendre(pl.N_rho, 0.0, pl.R, r, wr);
    if (pl.dim == 2) {
        // midpoint rule on the circle (Sec. 5.2), stored as 3-vectors with a zero third component
        if (sphere_xyz || sphere_w) return BZ_ERR_ARG;
        for (int j = 0; j < pl.M; ++j) {
            const double ph = 2.0 * M_PI * (j + 0.5) / pl.M;
            q.push_back(std::cos(ph));
            q.push_back(std::sin(ph));
            q.push_back(0.0);
            wq.push_back(2.0 * M_PI / pl.M);
        }
    } else if (sphere_xyz && sphere_w) {
        q.assign(sphere_xyz, sphere_xyz + 3 * pl.M);
        wq.assign(sphere_w, sphere_w + pl.M);
    } else if (pl.M == 12) {
        icosahedron(q, wq);
    } else if (!product_rule(pl.M, q, wq)) {
        return BZ_ERR_ARG;
    }
    HostTerms &T = pl.terms;
    pl.P = pl.N_rho * pl.M;
    T.r.resize(pl.P); T.wr.resize(pl.P); T.q.resize(3 * pl.P); T.wq.resize(pl.P);
    T.c.resize(pl.P); T.radial_index.resize(pl.P);
    for (int i = 0; i < pl.N_rho; ++i) {
        for (int j = 0; j < pl.M; ++j) {
            int p = i * pl.M + j;
            T.r[p] = r[i];
            T.wr[p] = wr[i];
            T.wq[p] = wq[j];
            for (int d = 0; d < 3; ++d) T.q[3 * p + d] = q[3 * j + d];
            // c_p = w_i w_j Phi(r_i) r_i^(d-1) (eq. approxG)
            T.c[p] = wr[i] * wq[j] * std::pow(r[i], pl.gamma) * (pl.dim == 2 ? r[i] : r[i] * r[i]);
            T.radial_index[p] = i;
        }
    }
    return BZ_OK;
}

// The weight of the part-II theta integral: g(t) = sin(t) b(cos t) in 3D (the sphere's
// measure), b(cos t) itself in 2D (eqs. b1-b4; the circle's measure is dt).
static double kernel_g(const Plan &pl, double t) {
    double h = std::sin(0.5 * t);
    switch (pl.kernel) {
        case BZ_KERNEL_B1: return pl.kc;
        case BZ_KERNEL_B2: return pl.kc / h;
        case BZ_KERNEL_B3: return pl.kc / (h * h);
        case BZ_KERNEL_B4: return pl.kc * std::fabs(std::cos(0.5 * t)) * std::pow(h, -2.5);
        case BZ_KERNEL_DEBYE: return std::fabs(std::log(2.0 * h)) / (2.0 * h);
        case BZ_KERNEL_FAMILY: return pl.kc * std::pow(h, -1.0 - 2.0 * pl.s);
        case BZ_KERNEL_B5: return pl.kc * std::sin(t);
        default: return pl.kc * std::cos(0.5 * t) * std::pow(h, -2.5);
    }
}

// int_0^eps sin^alpha(t/2) dt = 2 int_0^U sin^alpha(u) du, U = eps/2, evaluated with the
// substitution u = U tau^(1/(alpha+1)), which turns it into
// 2 U^(alpha+1)/(alpha+1) int_0^1 (sin(u)/u)^alpha dtau (a smooth integrand).
static double int_sin_half_pow(double alpha, double eps) {
    const double U = 0.5 * eps;
    std::vector<double> x, w;
    gauss_legendre(24, 0.0, 1.0, x, w);
    double acc = 0.0;
    for (int i = 0; i < 24; ++i) {
        double u = U * std::pow(x[i], 1.0 / (alpha + 1.0));
        double sr = (u > 0.0) ? std::sin(u) / u : 1.0;
        acc += w[i] * std::pow(sr, alpha);
    }
    return 2.0 * std::pow(U, alpha + 1.0) / (alpha + 1.0) * acc;
}

bz_status build_kernel_constants(Plan &pl) {
    const double eps = pl.eps;
    const double W = std::sin(0.5 * eps);
    if ((pl.dim == 2) != (pl.kernel >= BZ_KERNEL_B1 && pl.kernel <= BZ_KERNEL_B4)) return BZ_ERR_ARG;
    switch (pl.kernel) {
        case BZ_KERNEL_DEBYE: {
            // g (1 - cos) = h |log 2h|, g (1 - cos)^2 = 2 h^3 |log 2h| (h = sin(t/2)); with t = eps u^2
            // the integrands are smooth in u: 32-point Gauss-Legendre
            pl.kc = 1.0;
            std::vector<double> x, w;
            gauss_legendre(32, 0.0, 1.0, x, w);
            double a1 = 0.0, a2 = 0.0;
            for (int i = 0; i < 32; ++i) {
                const double t = eps * x[i] * x[i], jac = 2.0 * eps * x[i];
                const double h = std::sin(0.5 * t), lg = std::fabs(std::log(2.0 * h));
                a1 += w[i] * jac * h * lg;
                a2 += w[i] * jac * 2.0 * h * h * h * lg;
            }
            pl.A[0] = a1;
            pl.A[1] = a2;
            break;
        }
        // 2D kernels b = c sin^beta(t/2): b (1 - cos) = 2 c sin^(beta+2)(t/2), b (1 - cos)^2 =
        // 4 c sin^(beta+4)(t/2) over [0, eps] (parts I and III of Sec. 4.1 (i))
        case BZ_KERNEL_B1:
            pl.kc = 1.0 / (2.0 * M_PI);
            pl.A[0] = 2.0 * pl.kc * int_sin_half_pow(2.0, eps);
            pl.A[1] = 4.0 * pl.kc * int_sin_half_pow(4.0, eps);
            break;
        case BZ_KERNEL_B2:
            pl.kc = 3.0 / 32.0;
            pl.A[0] = 2.0 * pl.kc * int_sin_half_pow(1.0, eps);
            pl.A[1] = 4.0 * pl.kc * int_sin_half_pow(3.0, eps);
            break;
        case BZ_KERNEL_B3:
            pl.kc = 1.0 / (8.0 * M_PI);
            pl.A[0] = 2.0 * pl.kc * eps;
            pl.A[1] = 4.0 * pl.kc * int_sin_half_pow(2.0, eps);
            break;
        case BZ_KERNEL_B4:
            pl.kc = 5.0 / 256.0;
            // w = sin(t/2), cos(t/2) dt = 2 dw: A1 = 2 c int 2 w^(-1/2) dw, A2 = 4 c int 2 w^(3/2) dw
            pl.A[0] = 8.0 * pl.kc * std::sqrt(W);
            pl.A[1] = 3.2 * pl.kc * std::pow(W, 2.5);
            break;
        case BZ_KERNEL_FAMILY: {
            if (!(pl.s >= 0.0 && pl.s < 1.0)) return BZ_ERR_ARG;
            // lambda = 2 pi c B(1 - s, 3/2) = 1/6
            double lb = std::lgamma(1.0 - pl.s) + std::lgamma(1.5) - std::lgamma(2.5 - pl.s);
            pl.kc = 1.0 / (12.0 * M_PI * std::exp(lb));
            // g (1 - cos) = 2 c sin^(1-2s)(t/2); g (1 - cos)^2 = 4 c sin^(3-2s)(t/2)
            pl.A[0] = 2.0 * pl.kc * int_sin_half_pow(1.0 - 2.0 * pl.s, eps);
            pl.A[1] = 4.0 * pl.kc * int_sin_half_pow(3.0 - 2.0 * pl.s, eps);
            break;
        }
        case BZ_KERNEL_B5: {
            pl.kc = 1.0 / (4.0 * M_PI);
            double omc = 2.0 * W * W;     // 1 - cos(eps)
            pl.A[0] = pl.kc * 0.5 * omc * omc;            // int sin t (1 - cos t)
            pl.A[1] = pl.kc * omc * omc * omc / 3.0;      // int sin t (1 - cos t)^2
            break;
        }
        case BZ_KERNEL_B8: {
            pl.kc = 5.0 / (192.0 * M_PI);
            // with w = sin(t/2): cos(t/2) dt = 2 dw, so g dt = 2 c w^(-5/2) dw and
            // 1 - cos t = 2 w^2: A1 = 4 c int_0^W w^(-1/2) dw, A2 = 8 c int_0^W w^(3/2) dw
            pl.A[0] = 4.0 * pl.kc * 2.0 * std::sqrt(W);
            pl.A[1] = 8.0 * pl.kc * 0.4 * std::pow(W, 2.5);
            break;
        }
        default: return BZ_ERR_ARG;
    }
    pl.A[2] = 2.0 * pl.A[0] - pl.A[1];   // sin^2 t = 2 (1 - cos t) - (1 - cos t)^2
    if (pl.theta0 > 0.0) pl.A[0] = pl.A[1] = pl.A[2] = 0.0;   // a cutoff kernel vanishes near 0: no part I
    return BZ_OK;
}

// Part II theta rule for each radial node: 16-point Gauss-Legendre panels; graded
// panels [eps 2^j, eps 2^(j+1)] up to 0.25, then equal panels to pi; every panel at
// most min(0.25, 10 / z) wide with z = pi r |k|_max / (2L) (the largest phase rate).
void build_theta_rules(Plan &pl) {
    std::vector<double> gx, gw;
    gauss_legendre(16, -1.0, 1.0, gx, gw);
    const double kmax = std::sqrt((double)pl.dim) * (pl.N / 2);
    std::vector<double> rr;
    std::vector<double> wr;
    gauss_legendre(pl.N_rho, 0.0, pl.R, rr, wr);
    pl.rules.assign(pl.N_rho, ThetaRule());
    for (int i = 0; i < pl.N_rho; ++i) {
        double z = M_PI * rr[i] * kmax / (2.0 * pl.L);
        double width = std::fmin(0.25, 10.0 / std::fmax(z, 1e-300));
        std::vector<double> edges;
        double lo = pl.theta0 > 0.0 ? pl.theta0 : pl.eps;   // part II starts at the cutoff if there is one
        const double tg = 0.25;
        edges.push_back(lo);
        while (lo < tg) {
            double hi = std::fmin(2.0 * lo, tg);
            int ns = (int)std::ceil((hi - lo) / width);
            for (int k = 1; k <= ns; ++k) edges.push_back(lo + (hi - lo) * k / ns);
            lo = hi;
        }
        // equal panels to pi; the Debye-Yukawa kernel's |log(2 sin(t/2))| has a kink at pi/3
        std::vector<double> stops;
        if (pl.kernel == BZ_KERNEL_DEBYE && lo < M_PI / 3.0) stops.push_back(M_PI / 3.0);
        stops.push_back(M_PI);
        for (double stop : stops) {
            int nu = (int)std::ceil((stop - lo) / width);
            for (int k = 1; k <= nu; ++k) edges.push_back(lo + (stop - lo) * k / nu);
            lo = stop;
        }
        ThetaRule &R = pl.rules[i];
        for (size_t e = 0; e + 1 < edges.size(); ++e) {
            double a = edges[e], b = edges[e + 1];
            for (int q = 0; q < 16; ++q) {
                double t = 0.5 * (b - a) * gx[q] + 0.5 * (a + b);
                double h = std::sin(0.5 * t);
                R.omc.push_back(2.0 * h * h);
                R.sn.push_back(std::sin(t));
                R.W.push_back(0.5 * (b - a) * gw[q] * kernel_g(pl, t));
            }
        }
    }
}

}  // namespace bz
