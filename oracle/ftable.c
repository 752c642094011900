/*
 * Oracle (test infrastructure): F(k, |q|, qhat) of Sec. 2.1, eq. FF, computed by
 * the split of Sec. 4.1 (3D case).  Plain FP64 C with OpenMP; shares no code with
 * the CUDA library.
 *
 *   F(k, r, qhat) = int_{S^2} b(sigma.qhat) (exp(i a k.(qhat - sigma)) - 1) dsigma,
 *   a = pi r / (2 L).
 *
 * With sigma = h sin(t) cos(phi) + j sin(t) sin(phi) + qhat cos(t) (eq. FF3D1),
 * k.(qhat - sigma) = kappa (1 - cos t) - kperp sin t cos(phi - phi0), where
 * kappa = k.qhat and kperp = |k - kappa qhat|.  The phi integral is taken exactly:
 * int_0^{2pi} exp(-i y sin t cos phi) dphi = 2 pi J0(y sin t) (the limit of the
 * paper's midpoint rule in phi).  With x = a kappa, y = a kperp, g = sin(t) b:
 *
 *   part I  (t in [0, eps]): second-order Taylor expansion of the exponential,
 *           averaged over phi, integrated exactly through the kernel moments
 *           A1 = int g (1-cos), A2 = int g (1-cos)^2, A3 = int g sin^2:
 *           I = 2 pi [ i x A1 - x^2 A2 / 2 - y^2 A3 / 4 ].
 *   part II (t in [eps, pi]): 2 pi int g [exp(i x (1-cos t)) J0(y sin t) - 1] dt
 *           by composite Gauss-Legendre: panels [eps 2^j, eps 2^(j+1)] up to 0.5,
 *           then equal panels up to pi; every panel is at most min(0.5, 6 / z)
 *           wide, z = a |k|_max (graded panels are split to meet that).
 *           (The paper uses an adaptive quadrature here; any rule converged to
 *           rounding gives the same table.)
 *
 * The bracket is evaluated without cancellation as
 *   (exp(i x c) - 1) J0 + (J0 - 1),  exp(i x c) - 1 = -2 sin^2(x c / 2) + i sin(x c),
 * with a power series for J0(z) - 1 when z is small.  J0 is libm's j0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double kernel_g(double t, int kid, double s, double c) {
    double h = sin(0.5 * t);
    if (kid == 0) return c * pow(h, -1.0 - 2.0 * s);        /* family: c sin^(-1-2s)(t/2) */
    if (kid == 1) return c * sin(t);                         /* b5: sin(t) / (4 pi)        */
    if (kid == 7) return fabs(log(2.0 * h)) / (2.0 * h);     /* Debye-Yukawa (eq. ApproximatedDebye) */
    return c * cos(0.5 * t) * pow(h, -2.5);                  /* b8                          */
}

static double j0_minus_1(double z) {
    if (fabs(z) < 0.25) {
        /* J0(z) - 1 = sum_{m>=1} (-1)^m (z^2/4)^m / (m!)^2 */
        double u = 0.25 * z * z, term = 1.0, sum = 0.0;
        for (int m = 1; m <= 10; ++m) {
            term *= -u / ((double)m * (double)m);
            sum += term;
        }
        return sum;
    }
    return j0(z) - 1.0;
}

/* Builds the part-II rule for one radial node: theta nodes and weights w * g(theta).
 * Returns the number of nodes (<= cap). */
static int part2_rule(double eps, double zmax, int npts, const double *glx, const double *glw,
                      int kid, double s, double c, double *th, double *wg, double *cth, double *sth, int cap) {
    int n = 0;
    double lo = eps;
    const double tg = 0.5;
    double width = fmin(0.5, 6.0 / fmax(zmax, 1e-300));
    while (lo < tg) {
        double hi = fmin(2.0 * lo, tg);
        int nsub = (int)ceil((hi - lo) / width);   /* keep each panel within the oscillation limit */
        double dsub = (hi - lo) / nsub;
        for (int sp = 0; sp < nsub; ++sp) {
            double a = lo + sp * dsub, b = lo + (sp + 1) * dsub;
            for (int q = 0; q < npts && n < cap; ++q) {
                double t = 0.5 * (b - a) * glx[q] + 0.5 * (b + a);
                th[n] = t;
                wg[n] = 0.5 * (b - a) * glw[q] * kernel_g(t, kid, s, c);
                n++;
            }
        }
        lo = hi;
    }
    /* equal panels from max(lower bound, tg) to pi; the Debye-Yukawa kernel's |log(2 sin(t/2))|
     * has a kink at pi/3, which gets a panel edge */
    double stops[2];
    int nst = 0;
    if (kid == 7 && lo < M_PI / 3.0) stops[nst++] = M_PI / 3.0;
    stops[nst++] = M_PI;
    for (int si = 0; si < nst; ++si) {
        int npan = (int)ceil((stops[si] - lo) / width);
        double dw = (stops[si] - lo) / npan;
        for (int pn = 0; pn < npan; ++pn) {
            double a = lo + pn * dw, b = lo + (pn + 1) * dw;
            for (int q = 0; q < npts && n < cap; ++q) {
                double t = 0.5 * (b - a) * glx[q] + 0.5 * (b + a);
                th[n] = t;
                wg[n] = 0.5 * (b - a) * glw[q] * kernel_g(t, kid, s, c);
                n++;
            }
        }
        lo = stops[si];
    }
    if (n >= cap) return -1;   /* rule does not fit: report instead of truncating */
    for (int q = 0; q < n; ++q) {
        double h = sin(0.5 * th[q]);
        cth[q] = 2.0 * h * h;  /* 1 - cos(t) */
        sth[q] = sin(th[q]);
    }
    return n;
}

static void f_entry(double x, double y, const double A[3], int n, const double *wg,
                    const double *cth, const double *sth, double *re, double *im) {
    double sr = -0.5 * x * x * A[1] - 0.25 * y * y * A[2];
    double si = x * A[0];
    for (int q = 0; q < n; ++q) {
        double z = y * sth[q];
        double jm1 = j0_minus_1(z);
        double J = 1.0 + jm1;
        double ph = x * cth[q];
        double sh = sin(0.5 * ph);
        sr += wg[q] * (-2.0 * sh * sh * J + jm1);
        si += wg[q] * (sin(ph) * J);
    }
    *re = 2.0 * M_PI * sr;
    *im = 2.0 * M_PI * si;
}

#define RULE_CAP 8192

/* F for all N^3 modes (FFT-natural order, signed index) and each of the P terms.
 * out has P * N^3 complex entries (interleaved re, im).  Returns 0 on success. */
int oracle_ftable(int N, double L, int P, const double *r, const double *qhat,
                  int kid, double s, double c, double eps, const double *A,
                  int npts, const double *glx, const double *glw, double *out) {
    const long n3 = (long)N * N * N;
    const double kmax = sqrt(3.0) * (N / 2);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (long pk = 0; pk < (long)P * N; ++pk) {
        int p = (int)(pk / N), i1 = (int)(pk % N);
        double *th = malloc(sizeof(double) * RULE_CAP * 4);
        if (!th) { err = 1; continue; }
        double *wg = th + RULE_CAP, *cth = th + 2 * RULE_CAP, *sth = th + 3 * RULE_CAP;
        double a = M_PI * r[p] / (2.0 * L);
        int n = part2_rule(eps, a * kmax, npts, glx, glw, kid, s, c, th, wg, cth, sth, RULE_CAP);
        if (n < 0) { err = 1; free(th); continue; }
        const double *qh = qhat + 3 * p;
        int k1 = i1 < N / 2 ? i1 : i1 - N;
        for (int i2 = 0; i2 < N; ++i2) {
            int k2 = i2 < N / 2 ? i2 : i2 - N;
            for (int i3 = 0; i3 < N; ++i3) {
                int k3 = i3 < N / 2 ? i3 : i3 - N;
                double kap = k1 * qh[0] + k2 * qh[1] + k3 * qh[2];
                double kk = (double)k1 * k1 + (double)k2 * k2 + (double)k3 * k3;
                double kp2 = kk - kap * kap;
                double kp = kp2 > 0.0 ? sqrt(kp2) : 0.0;
                long idx = (long)p * n3 + ((long)i1 * N + i2) * N + i3;
                f_entry(a * kap, a * kp, A, n, wg, cth, sth, &out[2 * idx], &out[2 * idx + 1]);
            }
        }
        free(th);
    }
    return err;
}

/* F at a list of (signed k, r, qhat) entries; used to sample large tables. */
int oracle_fentries(int count, const int *k, const double *r, const double *qhat, double L, int N,
                    int kid, double s, double c, double eps, const double *A,
                    int npts, const double *glx, const double *glw, double *out) {
    const double kmax = sqrt(3.0) * (N / 2);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int e = 0; e < count; ++e) {
        double *th = malloc(sizeof(double) * RULE_CAP * 4);
        if (!th) { err = 1; continue; }
        double *wg = th + RULE_CAP, *cth = th + 2 * RULE_CAP, *sth = th + 3 * RULE_CAP;
        double a = M_PI * r[e] / (2.0 * L);
        int n = part2_rule(eps, a * kmax, npts, glx, glw, kid, s, c, th, wg, cth, sth, RULE_CAP);
        if (n < 0) { err = 1; free(th); continue; }
        const double *qh = qhat + 3 * e;
        const int *kk = k + 3 * e;
        double kap = kk[0] * qh[0] + kk[1] * qh[1] + kk[2] * qh[2];
        double k2 = (double)kk[0] * kk[0] + (double)kk[1] * kk[1] + (double)kk[2] * kk[2];
        double kp2 = k2 - kap * kap;
        double kp = kp2 > 0.0 ? sqrt(kp2) : 0.0;
        f_entry(a * kap, a * kp, A, n, wg, cth, sth, &out[2 * e], &out[2 * e + 1]);
        free(th);
    }
    return err;
}
