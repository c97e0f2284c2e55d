/* cg_closed.c -- hand-written closed-form CPU gradients (OpenMP) of two of the
 * fit objectives: TEST AND BASELINE INFRASTRUCTURE ONLY, like the tape oracle
 * beside it (no code shared with the GPU path, none with cg_oracle.c).
 *
 * The paper compares reverse-mode AD gradients with numerical ones inside the
 * fitting loop (Sec. 4); these are the derivatives written out by hand, the
 * fastest plain CPU way to the same numbers, and serve (a) as the CPU
 * baseline timed beside the GPU kernels and (b) as a second, independent
 * statement of the gradient that the tape oracle must reproduce.
 *
 * Each function sums its per-element terms in per-thread Neumaier partials
 * (OpenMP static schedule) and merges the partials in thread order, so the
 * result is deterministic for a given thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define CLF_MAX 32

typedef struct {
    double s, c;
} nsum_t;

static void nadd(nsum_t *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double nval(const nsum_t *a) { return a->s + a->c; }

static double std_pdf(double z) { return exp(-0.5 * z * z) / sqrt(2.0 * M_PI); }
static double std_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

static int nthreads(int threads) {
#ifdef _OPENMP
    return threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
    return 1;
#endif
}

/* Unbinned NLL of p(x) = f G(x) + (1 - f) E(x) on [lo, hi], theta = (f, mu,
 * s, lambda): G = exp(-(x-mu)^2/(2 s^2)) / (s sqrt(2 pi) Z_G), Z_G =
 * Phi((hi-mu)/s) - Phi((lo-mu)/s); E = lambda exp(-lambda x) / Z_E, Z_E =
 * exp(-lambda lo) - exp(-lambda hi).  NLL = -sum log p; d/dtheta by hand:
 *   dG/dmu = G ((x-mu)/s^2 - Z_G,mu / Z_G),  Z_G,mu = (phi(z_lo) - phi(z_hi)) / s
 *   dG/ds  = G ((x-mu)^2/s^3 - 1/s - Z_G,s / Z_G),  Z_G,s = (z_lo phi(z_lo) - z_hi phi(z_hi)) / s
 *   dE/dlambda = E (1/lambda - x - Z_E,lambda / Z_E),  Z_E,lambda = hi e^{-lambda hi} - lo e^{-lambda lo}
 * grad may be NULL (value only).  Returns 0, or 1 for invalid input. */
int clf_mix(int64_t n, const double *x, double lo, double hi, const double *theta, double *value, double *grad,
            int threads) {
    const double f = theta[0], mu = theta[1], s = theta[2], lam = theta[3];
    if (!(s > 0.0) || !(hi > lo) || n < 0) return 1;
    const double zl = (lo - mu) / s, zh = (hi - mu) / s;
    const double ZG = std_cdf(zh) - std_cdf(zl);
    const double ZE = exp(-lam * lo) - exp(-lam * hi);
    const double dZG_mu = (std_pdf(zl) - std_pdf(zh)) / s;
    const double dZG_s = (zl * std_pdf(zl) - zh * std_pdf(zh)) / s;
    const double dZE_l = hi * exp(-lam * hi) - lo * exp(-lam * lo);
    const double cG = 1.0 / (s * sqrt(2.0 * M_PI) * ZG);
    const double cE = lam / ZE;
    const int T = nthreads(threads);
    nsum_t *part = (nsum_t *)calloc((size_t)T * 5, sizeof(nsum_t));
    if (!part) return 1;
#pragma omp parallel num_threads(T)
    {
#ifdef _OPENMP
        const int t = omp_get_thread_num();
#else
        const int t = 0;
#endif
        nsum_t a[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};   /* local: no false sharing */
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const double xi = x[i], d = xi - mu;
            const double G = cG * exp(-d * d / (2.0 * s * s));
            const double E = cE * exp(-lam * xi);
            const double p = f * G + (1.0 - f) * E;
            nadd(&a[0], -log(p));
            if (grad) {
                const double r = 1.0 / p;
                nadd(&a[1], -(G - E) * r);
                nadd(&a[2], -f * G * (d / (s * s) - dZG_mu / ZG) * r);
                nadd(&a[3], -f * G * (d * d / (s * s * s) - 1.0 / s - dZG_s / ZG) * r);
                nadd(&a[4], -(1.0 - f) * E * (1.0 / lam - xi - dZE_l / ZE) * r);
            }
        }
        for (int k = 0; k < 5; ++k) part[5 * t + k] = a[k];
    }
    nsum_t tot[5] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 5; ++k) {
            nadd(&tot[k], part[5 * t + k].s);
            nadd(&tot[k], part[5 * t + k].c);
        }
    free(part);
    *value = nval(&tot[0]);
    if (grad)
        for (int k = 0; k < 4; ++k) grad[k] = nval(&tot[k + 1]);
    return 0;
}

/* chi2 of K Gaussian peaks A_k exp(-(x-mu_k)^2/(2 s_k^2)) + a degree-D
 * polynomial in u (u = x, or u = (2x - lo - hi)/(hi - lo) with poly_mode 1)
 * over n uniform bins on [lo, hi] with centres x_i = lo + (i + 0.5)(hi-lo)/n:
 * chi2 = sum w_i (y_i - f_i)^2, w_i = 1/max(y_i, 1).  With g_i = -2 w_i (y_i - f_i):
 *   d/dA_k = sum g e_k,  d/dmu_k = sum g A_k e_k (x-mu_k)/s_k^2,
 *   d/ds_k = sum g A_k e_k (x-mu_k)^2/s_k^3,  d/dc_j = sum g u^j.
 * grad may be NULL.  Returns 0, or 1 for invalid input. */
int clf_gauss_poly_chi2(int K, int D, int poly_mode, int64_t n, double lo, double hi, const double *y,
                        const double *theta, double *value, double *grad, int threads) {
    const int P = 3 * K + D + 1;
    if (K < 0 || D < -1 || P > CLF_MAX || n < 0 || !(hi > lo)) return 1;
    const double h = (hi - lo) / (double)n;
    const int T = nthreads(threads);
    nsum_t *part = (nsum_t *)calloc((size_t)T * (P + 1), sizeof(nsum_t));
    if (!part) return 1;
#pragma omp parallel num_threads(T)
    {
#ifdef _OPENMP
        const int t = omp_get_thread_num();
#else
        const int t = 0;
#endif
        nsum_t a[CLF_MAX + 1];   /* local: no false sharing */
        for (int k = 0; k <= P; ++k) a[k].s = a[k].c = 0.0;
        double e[CLF_MAX];
#pragma omp for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const double x = lo + ((double)i + 0.5) * h;
            const double u = poly_mode ? (2.0 * x - lo - hi) / (hi - lo) : x;
            double f = 0.0, up = 1.0;
            for (int j = 0; j <= D; ++j) {
                f += theta[3 * K + j] * up;
                up *= u;
            }
            for (int k = 0; k < K; ++k) {
                const double d = x - theta[3 * k + 1], sk = theta[3 * k + 2];
                e[k] = exp(-d * d / (2.0 * sk * sk));
                f += theta[3 * k] * e[k];
            }
            const double w = 1.0 / (y[i] > 1.0 ? y[i] : 1.0);
            const double res = y[i] - f;
            nadd(&a[0], w * res * res);
            if (grad) {
                const double g = -2.0 * w * res;
                for (int k = 0; k < K; ++k) {
                    const double A = theta[3 * k], d = x - theta[3 * k + 1], sk = theta[3 * k + 2];
                    nadd(&a[1 + 3 * k], g * e[k]);
                    nadd(&a[2 + 3 * k], g * A * e[k] * d / (sk * sk));
                    nadd(&a[3 + 3 * k], g * A * e[k] * d * d / (sk * sk * sk));
                }
                up = 1.0;
                for (int j = 0; j <= D; ++j) {
                    nadd(&a[1 + 3 * K + j], g * up);
                    up *= u;
                }
            }
        }
        for (int k = 0; k <= P; ++k) part[(size_t)(P + 1) * t + k] = a[k];
    }
    nsum_t tot[CLF_MAX + 1];
    for (int k = 0; k <= P; ++k) tot[k].s = tot[k].c = 0.0;
    for (int t = 0; t < T; ++t)
        for (int k = 0; k <= P; ++k) {
            nadd(&tot[k], part[(size_t)(P + 1) * t + k].s);
            nadd(&tot[k], part[(size_t)(P + 1) * t + k].c);
        }
    free(part);
    *value = nval(&tot[0]);
    if (grad)
        for (int k = 0; k < P; ++k) grad[k] = nval(&tot[k + 1]);
    return 0;
}

/* Central-difference gradient of the mixture NLL from 2P = 8 value-only
 * evaluations, steps h_k = 1e-6 max(|theta_k|, 1e-3): the numerical gradient
 * the paper's AD replaces. */
int clf_mix_fd(int64_t n, const double *x, double lo, double hi, const double *theta, double *grad, int threads) {
    double t[4];
    for (int k = 0; k < 4; ++k) {
        for (int j = 0; j < 4; ++j) t[j] = theta[j];
        const double hk = 1e-6 * fmax(fabs(theta[k]), 1e-3);
        double vp, vm;
        t[k] = theta[k] + hk;
        if (clf_mix(n, x, lo, hi, t, &vp, NULL, threads)) return 1;
        t[k] = theta[k] - hk;
        if (clf_mix(n, x, lo, hi, t, &vm, NULL, threads)) return 1;
        grad[k] = (vp - vm) / (2.0 * hk);
    }
    return 0;
}
