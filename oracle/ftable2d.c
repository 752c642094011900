/*
 * Oracle (test infrastructure): the 2D weight F(k, |q|, qhat) of Sec. 2.1, eq. FF2D1,
 * computed by the three-part split of Sec. 4.1 (2D case).  Plain FP64 C with OpenMP;
 * shares no code with the CUDA library.
 *
 *   F(k, r, qhat) = int_0^{2 pi} b(cos t) (exp(i a k.[qhat (1 - cos t) - qperp sin t]) - 1) dt,
 *   a = pi r / (2 L),  sigma = qhat cos t + qperp sin t.
 *
 * With x = a k.qhat and y = a k.qperp the exponent is i [x (1 - cos t) - y sin t].
 *   parts I + III (t in [0, eps] and [2 pi - eps, 2 pi]): second-order Taylor expansion of
 *       the exponential; under t -> 2 pi - t the kernel and 1 - cos t are unchanged and
 *       sin t changes sign, so the terms odd in sin t cancel between I and III:
 *       I + III = 2 [ i x A1 - x^2 A2 / 2 - y^2 A3 / 2 ],
 *       A1 = int_0^eps b (1-cos), A2 = int_0^eps b (1-cos)^2, A3 = int_0^eps b sin^2.
 *   part II (t in [eps, 2 pi - eps]): folded onto [eps, pi] by the same symmetry,
 *       II = 2 int_eps^pi b(cos t) [exp(i x (1 - cos t)) cos(y sin t) - 1] dt,
 *       by the composite Gauss-Legendre rule of the 3D oracle (panels graded from eps to 0.5,
 *       then equal panels to pi, each at most min(0.5, 6 / z) wide, z = a |k|_max).
 * The bracket is evaluated without cancellation as
 *   (exp(i x c) - 1) cos(y s) + (cos(y s) - 1),  cos(y s) - 1 = -2 sin^2(y s / 2).
 *
 * Kernels (eqs. b1-b4, t in (0, pi]):
 *   kid 3: b1 = 1 / (2 pi);  kid 4: b2 = 3 / (32 sin(t/2));  kid 5: b3 = 1 / (8 pi sin^2(t/2));
 *   kid 6: b4 = 5 |cos(t/2)| / (256 sin^(5/2)(t/2)).  c is the constant factor.
 */
#include <math.h>
#include <stdlib.h>

static double kernel_b2d(double t, int kid, double c) {
    double h = sin(0.5 * t);
    if (kid == 3) return c;
    if (kid == 4) return c / h;
    if (kid == 5) return c / (h * h);
    return c * fabs(cos(0.5 * t)) * pow(h, -2.5);
}

/* One panel's Gauss-Legendre nodes: weights w * b(t), 1 - cos t and sin t.  Returns the new
 * node count, or -1 when the rule would exceed cap. */
static int add_panel(double a, double b, int npts, const double *glx, const double *glw, int kid, double c,
                     double *wg, double *cth, double *sth, int n, int cap) {
    for (int q = 0; q < npts; ++q) {
        if (n >= cap) return -1;
        double th = 0.5 * (b - a) * glx[q] + 0.5 * (b + a);
        double h = sin(0.5 * th);
        wg[n] = 0.5 * (b - a) * glw[q] * kernel_b2d(th, kid, c);
        cth[n] = 2.0 * h * h;
        sth[n] = sin(th);
        n++;
    }
    return n;
}

static int part2_rule_2d(double eps, double zmax, int npts, const double *glx, const double *glw,
                         int kid, double c, double *wg, double *cth, double *sth, int cap) {
    int n = 0;
    double lo = eps;
    const double tg = 0.5;
    double width = fmin(0.5, 6.0 / fmax(zmax, 1e-300));
    while (lo < tg) {
        double hi = fmin(2.0 * lo, tg);
        int nsub = (int)ceil((hi - lo) / width);
        double dsub = (hi - lo) / nsub;
        for (int sp = 0; sp < nsub && n >= 0; ++sp)
            n = add_panel(lo + sp * dsub, lo + (sp + 1) * dsub, npts, glx, glw, kid, c, wg, cth, sth, n, cap);
        if (n < 0) return -1;
        lo = hi;
    }
    /* equal panels from max(lower bound, 0.5) to pi (the lower bound is eps, or the cutoff angle) */
    int npan = (int)ceil((M_PI - lo) / width);
    double dw = (M_PI - lo) / npan;
    for (int pn = 0; pn < npan && n >= 0; ++pn)
        n = add_panel(lo + pn * dw, lo + (pn + 1) * dw, npts, glx, glw, kid, c, wg, cth, sth, n, cap);
    return n;
}

static void f_entry_2d(double x, double y, const double A[3], int n, const double *wg,
                       const double *cth, const double *sth, double *re, double *im) {
    double sr = -0.5 * x * x * A[1] - 0.5 * y * y * A[2];
    double si = x * A[0];
    for (int q = 0; q < n; ++q) {
        double ys = y * sth[q];
        double cs = cos(ys);
        double hs = sin(0.5 * ys);
        double ph = x * cth[q];
        double sh = sin(0.5 * ph);
        sr += wg[q] * (-2.0 * sh * sh * cs - 2.0 * hs * hs);
        si += wg[q] * (sin(ph) * cs);
    }
    *re = 2.0 * sr;
    *im = 2.0 * si;
}

#define RULE_CAP_2D 8192

/* F for all N^2 modes (FFT-natural order, signed index) of each of the P terms (r[p],
 * qhat[2p..2p+1]); out has P * N^2 complex entries (interleaved).  Returns 0 on success. */
int oracle_ftable2d(int N, double L, int P, const double *r, const double *qhat, int kid, double c,
                    double eps, const double *A, int npts, const double *glx, const double *glw,
                    double *out) {
    const long n2 = (long)N * N;
    const double kmax = sqrt(2.0) * (N / 2);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < P; ++p) {
        double *wg = malloc(sizeof(double) * RULE_CAP_2D * 3);
        if (!wg) { err = 1; continue; }
        double *cth = wg + RULE_CAP_2D, *sth = wg + 2 * RULE_CAP_2D;
        double a = M_PI * r[p] / (2.0 * L);
        int n = part2_rule_2d(eps, a * kmax, npts, glx, glw, kid, c, wg, cth, sth, RULE_CAP_2D);
        if (n < 0) { err = 1; free(wg); continue; }
        const double q0 = qhat[2 * p], q1 = qhat[2 * p + 1];
        for (int i1 = 0; i1 < N; ++i1) {
            int k1 = i1 < N / 2 ? i1 : i1 - N;
            for (int i2 = 0; i2 < N; ++i2) {
                int k2 = i2 < N / 2 ? i2 : i2 - N;
                double kq = k1 * q0 + k2 * q1;          /* k . qhat */
                double kp = -k1 * q1 + k2 * q0;         /* k . qperp, qperp = (-q1, q0) */
                long idx = (long)p * n2 + (long)i1 * N + i2;
                f_entry_2d(a * kq, a * kp, A, n, wg, cth, sth, &out[2 * idx], &out[2 * idx + 1]);
            }
        }
        free(wg);
    }
    return err;
}
