/*
 * cg_oracle.c -- CPU oracle for the fit-objective gradients.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py may load this library.
 * The CUDA product path never links, loads or calls it, and it shares no
 * code, header or constant with that path.
 *
 * What it is: a plain scalar *tape-based* reverse-mode AD (the "tracing"
 * approach of Sec. 2, reverse accumulation as in Sec. 1), applied to fit
 * objectives summed over histogram bins or events (the histogram-fitting
 * use of AD gradients in Sec. 4, Fig. 3).  Every elementary operation is
 * recorded on a tape with its local partial derivatives; one reverse sweep
 * over the tape gives the exact gradient of the recorded expression.
 *
 * Structure of one evaluation F(theta) = sum_i T_i(theta):
 *   1. the parameters theta_k are the first P tape entries (leaves);
 *   2. quantities that depend on theta alone and appear in the model's
 *      definition (normalisation integrals Z of a pdf, cos/sin of an angle)
 *      are recorded once after the leaves ("prologue");
 *   3. for each bin/event i the term T_i is recorded on top of the prologue,
 *      swept in reverse from dT_i/dT_i = 1 down to the leaves, and then
 *      popped from the tape.  Because dF/dT_i = 1, the gradient of F is the
 *      sum over i of these per-term gradients.
 * Sums over terms (the value and each gradient component) use Neumaier
 * compensated summation, so the result is, to a few ulps, the exact sum of
 * the oracle's own per-term values.  For each component k the oracle also
 * returns S_k = sum_i |dT_i/dtheta_k|, the scale used by the relative-error
 * metric of the parity tests.
 *
 * Compile with -ffp-contract=off (no FMA contraction): every operation is
 * rounded as written.  Nothing here is blocked, fused or reordered beyond
 * the definitions below.
 *
 * Definitions (parameter order is part of the interface):
 *  - Gaussian peak, amplitude = peak height (the "gaus" formula of Fig. 3a):
 *        G(x) = A exp(-(x - mu)^2 / (2 s^2)).
 *  - 1-D binned model "K peaks + degree-D polynomial":
 *        f(x) = sum_k G_k(x) + sum_{j<=D} c_j u^j,
 *    u = x (poly_mode 0) or u = (2x - lo - hi)/(hi - lo) (poly_mode 1);
 *    theta = (A_1, mu_1, s_1, ..., A_K, mu_K, s_K, c_0, ..., c_D).
 *  - 1-D bin centres: x_i = lo + (i + 0.5) (hi - lo)/n, or given explicitly.
 *  - objectives over bins with counts y_i and model f_i = f(x_i):
 *        chi2      : sum_i w_i (y_i - f_i)^2,  w_i = 1/max(y_i, 1)
 *        poisson   : sum_i (f_i - y_i log f_i)            (log y_i! dropped)
 *        poisson_bc: sum_i 2 (f_i - y_i + y_i log(y_i/f_i)) (Baker-Cousins;
 *                    the y_i = 0 term is 2 f_i)
 *  - unbinned mixture on [lo, hi], theta = (frac, mu, s, lambda):
 *        p(x) = frac N(x; mu, s)/Z_G + (1 - frac) lambda e^{-lambda x}/Z_E,
 *        N(x; mu, s) = exp(-(x-mu)^2/(2 s^2)) / (s sqrt(2 pi)),
 *        Z_G = Phi((hi - mu)/s) - Phi((lo - mu)/s),  Phi(z) = erfc(-z/sqrt2)/2,
 *        Z_E = e^{-lambda lo} - e^{-lambda hi},
 *        NLL = -sum_i w_i log p(x_i)     (w_i = 1 when no weights are given).
 *  - 2-D binned model: K rotated Gaussians plus a constant, Poisson NLL,
 *        theta = (A, mu_x, mu_y, s_x, s_y, phi) x K, then C,
 *        u =  cos(phi)(x - mu_x) + sin(phi)(y - mu_y),
 *        v = -sin(phi)(x - mu_x) + cos(phi)(y - mu_y),
 *        mu(x, y) = C + sum_k A_k exp(-(u^2/s_x^2 + v^2/s_y^2)/2),
 *    bin (i, j) has centre (lx + (i+0.5)(hx-lx)/nx, ly + (j+0.5)(hy-ly)/ny)
 *    and its count at counts[j*nx + i] (x index fastest).
 *
 * Return codes: 0 ok, 1 invalid argument, 2 domain error (log of a
 * non-positive value, or a non-finite term); the value and gradient are
 * still written (they may be non-finite).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_DOMAIN 2

#define OBJ_CHI2 0
#define OBJ_POISSON 1
#define OBJ_POISSON_BC 2

/* ------------------------------------------------------------------ */
/* The tape.                                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    double v;        /* value */
    double pa, pb;   /* local partials d v / d parent_a, d v / d parent_b */
    int32_t a, b;    /* parent indices, -1 when absent */
} node;

typedef struct {
    node *n;
    int32_t len, cap;
    int domain;      /* set when log() sees a non-positive argument */
} tape;

static int tape_init(tape *T, int32_t cap) {
    T->n = (node *)malloc(sizeof(node) * (size_t)cap);
    T->len = 0;
    T->cap = cap;
    T->domain = 0;
    return T->n != NULL;
}

static void tape_free(tape *T) { free(T->n); T->n = NULL; }

static int32_t push(tape *T, double v, int32_t a, double pa, int32_t b, double pb) {
    if (T->len == T->cap) {
        int32_t nc = T->cap * 2;
        node *nn = (node *)realloc(T->n, sizeof(node) * (size_t)nc);
        if (!nn) abort();
        T->n = nn;
        T->cap = nc;
    }
    node *x = &T->n[T->len];
    x->v = v; x->a = a; x->pa = pa; x->b = b; x->pb = pb;
    return T->len++;
}

#define VAL(i) (T->n[(i)].v)

static int32_t t_var(tape *T, double v) { return push(T, v, -1, 0.0, -1, 0.0); }
static int32_t t_const(tape *T, double v) { return push(T, v, -1, 0.0, -1, 0.0); }
static int32_t t_add(tape *T, int32_t a, int32_t b) { return push(T, VAL(a) + VAL(b), a, 1.0, b, 1.0); }
static int32_t t_sub(tape *T, int32_t a, int32_t b) { return push(T, VAL(a) - VAL(b), a, 1.0, b, -1.0); }
static int32_t t_mul(tape *T, int32_t a, int32_t b) { return push(T, VAL(a) * VAL(b), a, VAL(b), b, VAL(a)); }
static int32_t t_div(tape *T, int32_t a, int32_t b) {
    double q = VAL(a) / VAL(b);
    return push(T, q, a, 1.0 / VAL(b), b, -q / VAL(b));
}
static int32_t t_neg(tape *T, int32_t a) { return push(T, -VAL(a), a, -1.0, -1, 0.0); }
/* a + c and a * c for a constant c */
static int32_t t_addc(tape *T, int32_t a, double c) { return push(T, VAL(a) + c, a, 1.0, -1, 0.0); }
static int32_t t_mulc(tape *T, int32_t a, double c) { return push(T, VAL(a) * c, a, c, -1, 0.0); }
/* c - a */
static int32_t t_rsubc(tape *T, double c, int32_t a) { return push(T, c - VAL(a), a, -1.0, -1, 0.0); }
static int32_t t_exp(tape *T, int32_t a) { double e = exp(VAL(a)); return push(T, e, a, e, -1, 0.0); }
static int32_t t_log(tape *T, int32_t a) {
    double x = VAL(a);
    if (!(x > 0.0)) T->domain = 1;
    return push(T, log(x), a, 1.0 / x, -1, 0.0);
}
static int32_t t_erfc(tape *T, int32_t a) {
    double z = VAL(a);
    /* d erfc(z)/dz = -2/sqrt(pi) exp(-z^2) */
    return push(T, erfc(z), a, -2.0 / sqrt(M_PI) * exp(-z * z), -1, 0.0);
}
static int32_t t_sqrt(tape *T, int32_t a) {
    double r = sqrt(VAL(a));
    if (!(VAL(a) >= 0.0)) T->domain = 1;
    return push(T, r, a, 0.5 / r, -1, 0.0);
}
/* a^k for an integer k: d/da = k a^(k-1) */
static int32_t t_powi(tape *T, int32_t a, int k) {
    double x = VAL(a);
    if (k == 0) return t_const(T, 1.0);
    return push(T, pow(x, (double)k), a, (double)k * pow(x, (double)(k - 1)), -1, 0.0);
}
/* max(a, b): the derivative goes to a when a >= b */
static int32_t t_max(tape *T, int32_t a, int32_t b) {
    if (VAL(a) >= VAL(b)) return push(T, VAL(a), a, 1.0, b, 0.0);
    return push(T, VAL(b), a, 0.0, b, 1.0);
}
static int32_t t_sin(tape *T, int32_t a) { return push(T, sin(VAL(a)), a, cos(VAL(a)), -1, 0.0); }
static int32_t t_cos(tape *T, int32_t a) { return push(T, cos(VAL(a)), a, -sin(VAL(a)), -1, 0.0); }

/* ------------------------------------------------------------------ */
/* Compensated accumulation (Neumaier's variant of Kahan summation).    */
/* ------------------------------------------------------------------ */

typedef struct { double s, c; } nsum;

static void nadd(nsum *acc, double v) {
    double t = acc->s + v;
    if (fabs(acc->s) >= fabs(v)) acc->c += (acc->s - t) + v;
    else acc->c += (v - t) + acc->s;
    acc->s = t;
}
static double nval(const nsum *acc) { return acc->s + acc->c; }

/* ------------------------------------------------------------------ */
/* Reverse sweeps.                                                     */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t P;        /* leaves occupy tape[0..P) */
    int32_t mark;     /* leaves + prologue occupy tape[0..mark) */
    double *adj;      /* adjoint per tape entry, grown with the tape */
    int32_t adj_cap;
    nsum value;
    nsum *grad;       /* [P] */
    double *scale;    /* [P], S_k = sum_i |dT_i/dtheta_k| (plain sum) */
    int nonfinite;
} accum;

static int accum_init(accum *A, int32_t P) {
    A->P = P;
    A->mark = 0;
    A->adj_cap = 1024;
    A->adj = (double *)malloc(sizeof(double) * (size_t)A->adj_cap);
    A->grad = (nsum *)calloc((size_t)P, sizeof(nsum));
    A->scale = (double *)calloc((size_t)P, sizeof(double));
    A->value.s = A->value.c = 0.0;
    A->nonfinite = 0;
    return A->adj && A->grad && A->scale;
}

static void accum_free(accum *A) { free(A->adj); free(A->grad); free(A->scale); }

/* Record-then-sweep for one term whose output is tape entry `out`:
 * seed dT/dT = 1, propagate adjoints down through the term and the
 * prologue to the leaves, add the leaf adjoints to the gradient, and pop
 * the term off the tape. */
static void finish_term(tape *T, accum *A, int32_t out) {
    int32_t top = T->len;
    if (A->adj_cap < top) {
        while (A->adj_cap < top) A->adj_cap *= 2;
        A->adj = (double *)realloc(A->adj, sizeof(double) * (size_t)A->adj_cap);
        if (!A->adj) abort();
    }
    for (int32_t i = 0; i < top; ++i) A->adj[i] = 0.0;
    A->adj[out] = 1.0;
    for (int32_t i = top - 1; i >= A->P; --i) {
        double g = A->adj[i];
        if (g == 0.0) continue;
        const node *x = &T->n[i];
        if (x->a >= 0) A->adj[x->a] += g * x->pa;
        if (x->b >= 0) A->adj[x->b] += g * x->pb;
    }
    double tv = VAL(out);
    if (!isfinite(tv)) A->nonfinite = 1;
    nadd(&A->value, tv);
    for (int32_t k = 0; k < A->P; ++k) {
        nadd(&A->grad[k], A->adj[k]);
        A->scale[k] += fabs(A->adj[k]);
    }
    T->len = A->mark;   /* pop the term */
}

static int finish(tape *T, accum *A, double *value, double *grad, double *scale) {
    *value = nval(&A->value);
    for (int32_t k = 0; k < A->P; ++k) {
        grad[k] = nval(&A->grad[k]);
        if (scale) scale[k] = A->scale[k];
    }
    int rc = (T->domain || A->nonfinite) ? ORC_DOMAIN : ORC_OK;
    return rc;
}

/* ------------------------------------------------------------------ */
/* Model pieces, written straight from the definitions above.           */
/* ------------------------------------------------------------------ */

/* A exp(-(x - mu)^2 / (2 s^2)) with A, mu, s tape entries and x a constant. */
static int32_t rec_gauss_peak(tape *T, int32_t A_, int32_t mu, int32_t s, double x) {
    int32_t d = t_rsubc(T, x, mu);                 /* x - mu */
    int32_t num = t_mul(T, d, d);                  /* (x - mu)^2 */
    int32_t den = t_mulc(T, t_mul(T, s, s), 2.0);  /* 2 s^2 */
    int32_t q = t_div(T, num, den);
    int32_t e = t_exp(T, t_neg(T, q));
    return t_mul(T, A_, e);
}

/* f(x) for K peaks + degree-D polynomial in u. Leaves are tape[0..P). */
static int32_t rec_gauss_poly(tape *T, int K, int D, double x, double u) {
    int32_t f = -1;
    for (int k = 0; k < K; ++k) {
        int32_t g = rec_gauss_peak(T, 3 * k, 3 * k + 1, 3 * k + 2, x);
        f = (f < 0) ? g : t_add(T, f, g);
    }
    double upow = 1.0;
    for (int j = 0; j <= D; ++j) {
        int32_t c = 3 * K + j;
        int32_t t = (j == 0) ? c : t_mulc(T, c, upow);
        f = (f < 0) ? t : t_add(T, f, t);
        upow = upow * u;
    }
    if (f < 0) f = t_const(T, 0.0);
    return f;
}

/* One bin's objective term from the model value f (tape entry) and count y. */
static int32_t rec_binned_term(tape *T, int obj, int32_t f, double y) {
    if (obj == OBJ_CHI2) {
        double w = 1.0 / fmax(y, 1.0);
        int32_t r = t_rsubc(T, y, f);              /* y - f */
        return t_mulc(T, t_mul(T, r, r), w);
    }
    if (obj == OBJ_POISSON) {
        if (y == 0.0) return f;
        return t_sub(T, f, t_mulc(T, t_log(T, f), y));
    }
    /* Baker-Cousins: 2 (f - y + y log(y / f)); 2 f when y = 0 */
    if (y == 0.0) return t_mulc(T, f, 2.0);
    int32_t lr = t_log(T, t_div(T, t_const(T, y), f));
    int32_t inner = t_add(T, t_addc(T, f, -y), t_mulc(T, lr, y));
    return t_mulc(T, inner, 2.0);
}

/* ------------------------------------------------------------------ */
/* Public entry points (called from Python through ctypes).            */
/* ------------------------------------------------------------------ */

int orc_num_params_gauss_poly(int K, int D) { return 3 * K + D + 1; }

/* 1-D binned objective.  centres may be NULL (uniform bins on [lo, hi]).
 * scale may be NULL. */
int orc_binned1d(int K, int D, int poly_mode, int obj, int64_t n, double lo, double hi,
                 const double *centres, const double *y, const double *theta,
                 double *value, double *grad, double *scale) {
    if (K < 0 || D < -1 || n < 0 || (K == 0 && D < 0) || obj < 0 || obj > 2) return ORC_INVALID;
    int32_t P = 3 * K + D + 1;
    tape T;
    accum A;
    if (!tape_init(&T, 256) || !accum_init(&A, P)) return ORC_INVALID;
    for (int32_t k = 0; k < P; ++k) t_var(&T, theta[k]);
    A.mark = T.len;
    double h = (hi - lo) / (double)n;
    for (int64_t i = 0; i < n; ++i) {
        double x = centres ? centres[i] : lo + ((double)i + 0.5) * h;
        double u = (poly_mode == 1) ? (2.0 * x - lo - hi) / (hi - lo) : x;
        int32_t f = rec_gauss_poly(&T, K, D, x, u);
        int32_t t = rec_binned_term(&T, obj, f, y[i]);
        finish_term(&T, &A, t);
    }
    int rc = finish(&T, &A, value, grad, scale);
    tape_free(&T);
    accum_free(&A);
    return rc;
}

/* Gauss-Newton matrix of a 1-D binned objective:
 *     GN_ab = sum_i h_i (d f_i / d theta_a) (d f_i / d theta_b),
 * h_i as for the diagonal below.  It is the Hessian of the objective with
 * the terms in the model's own second derivatives dropped; the second-order
 * fit step (Levenberg-Marquardt) solves with it.  gn: P x P, row-major. */
int orc_binned1d_gnmat(int K, int D, int poly_mode, int obj, int64_t n, double lo, double hi,
                       const double *centres, const double *y, const double *theta, double *gn) {
    int32_t P = 3 * K + D + 1;
    tape T;
    if (!tape_init(&T, 256)) return ORC_INVALID;
    for (int32_t k = 0; k < P; ++k) t_var(&T, theta[k]);
    int32_t mark = T.len;
    double *adj = (double *)malloc(sizeof(double) * 256);
    int32_t cap = 256;
    nsum *acc = (nsum *)calloc((size_t)P * (size_t)P, sizeof(nsum));
    double h = (hi - lo) / (double)n;
    for (int64_t i = 0; i < n; ++i) {
        double x = centres ? centres[i] : lo + ((double)i + 0.5) * h;
        double u = (poly_mode == 1) ? (2.0 * x - lo - hi) / (hi - lo) : x;
        int32_t f = rec_gauss_poly(&T, K, D, x, u);
        if (cap < T.len) { while (cap < T.len) cap *= 2; adj = (double *)realloc(adj, sizeof(double) * (size_t)cap); }
        for (int32_t j = 0; j < T.len; ++j) adj[j] = 0.0;
        adj[f] = 1.0;
        for (int32_t j = T.len - 1; j >= P; --j) {
            const node *nd = &T.n[j];
            if (nd->a >= 0) adj[nd->a] += adj[j] * nd->pa;
            if (nd->b >= 0) adj[nd->b] += adj[j] * nd->pb;
        }
        double fv = T.n[f].v, hi_;
        if (obj == OBJ_CHI2) hi_ = 2.0 / fmax(y[i], 1.0);
        else if (obj == OBJ_POISSON) hi_ = (y[i] > 0.0) ? y[i] / (fv * fv) : 0.0;
        else hi_ = (y[i] > 0.0) ? 2.0 * y[i] / (fv * fv) : 0.0;
        for (int32_t a = 0; a < P; ++a)
            for (int32_t b = a; b < P; ++b) nadd(&acc[(size_t)a * P + b], hi_ * adj[a] * adj[b]);
        T.len = mark;
    }
    /* symmetric by definition: the upper triangle, mirrored */
    for (int32_t a = 0; a < P; ++a)
        for (int32_t b = 0; b < P; ++b) gn[(size_t)a * P + b] = nval(&acc[a <= b ? (size_t)a * P + b : (size_t)b * P + a]);
    free(acc);
    free(adj);
    tape_free(&T);
    return ORC_OK;
}

/* Model value f(x) of the 1-D family at explicit points (no objective). */
int orc_gauss_poly_eval(int K, int D, int poly_mode, double lo, double hi, int64_t n,
                        const double *x, const double *theta, double *f_out) {
    int32_t P = 3 * K + D + 1;
    tape T;
    if (!tape_init(&T, 256)) return ORC_INVALID;
    for (int32_t k = 0; k < P; ++k) t_var(&T, theta[k]);
    int32_t mark = T.len;
    for (int64_t i = 0; i < n; ++i) {
        double u = (poly_mode == 1) ? (2.0 * x[i] - lo - hi) / (hi - lo) : x[i];
        int32_t f = rec_gauss_poly(&T, K, D, x[i], u);
        f_out[i] = T.n[f].v;
        T.len = mark;
    }
    tape_free(&T);
    return ORC_OK;
}

/* Gauss-Newton diagonal of a 1-D binned objective:
 *     GN_k = sum_i h_i (d f_i / d theta_k)^2,
 * with h_i = d^2 T_i / d f_i^2 of the bin term: 2 w_i (chi2), y_i / f_i^2
 * (poisson), 2 y_i / f_i^2 (poisson_bc); 0 for an empty bin of the latter two.  Used only to scale the initial
 * inverse Hessian of the BFGS fit. */
int orc_binned1d_gn(int K, int D, int poly_mode, int obj, int64_t n, double lo, double hi,
                    const double *centres, const double *y, const double *theta, double *gn) {
    int32_t P = 3 * K + D + 1;
    tape T;
    if (!tape_init(&T, 256)) return ORC_INVALID;
    for (int32_t k = 0; k < P; ++k) t_var(&T, theta[k]);
    int32_t mark = T.len;
    double *adj = (double *)malloc(sizeof(double) * 256);
    int32_t cap = 256;
    nsum *acc = (nsum *)calloc((size_t)P, sizeof(nsum));
    double h = (hi - lo) / (double)n;
    for (int64_t i = 0; i < n; ++i) {
        double x = centres ? centres[i] : lo + ((double)i + 0.5) * h;
        double u = (poly_mode == 1) ? (2.0 * x - lo - hi) / (hi - lo) : x;
        int32_t f = rec_gauss_poly(&T, K, D, x, u);
        if (cap < T.len) { while (cap < T.len) cap *= 2; adj = (double *)realloc(adj, sizeof(double) * (size_t)cap); }
        for (int32_t j = 0; j < T.len; ++j) adj[j] = 0.0;
        adj[f] = 1.0;
        for (int32_t j = T.len - 1; j >= P; --j) {
            const node *nd = &T.n[j];
            if (nd->a >= 0) adj[nd->a] += adj[j] * nd->pa;
            if (nd->b >= 0) adj[nd->b] += adj[j] * nd->pb;
        }
        double fv = T.n[f].v, hi_;
        /* an empty bin's term is T = f (times 2 for poisson_bc): linear in f,
         * curvature exactly 0 even where f itself underflows to 0 */
        if (obj == OBJ_CHI2) hi_ = 2.0 / fmax(y[i], 1.0);
        else if (obj == OBJ_POISSON) hi_ = (y[i] > 0.0) ? y[i] / (fv * fv) : 0.0;
        else hi_ = (y[i] > 0.0) ? 2.0 * y[i] / (fv * fv) : 0.0;
        for (int32_t k = 0; k < P; ++k) nadd(&acc[k], hi_ * adj[k] * adj[k]);
        T.len = mark;
    }
    for (int32_t k = 0; k < P; ++k) gn[k] = nval(&acc[k]);
    free(acc);
    free(adj);
    tape_free(&T);
    return ORC_OK;
}

/* Standard normal CDF on the tape: Phi(z) = erfc(-z / sqrt 2) / 2. */
static int32_t rec_Phi(tape *T, int32_t z) {
    return t_mulc(T, t_erfc(T, t_mulc(T, z, -1.0 / sqrt(2.0))), 0.5);
}

/* Unbinned mixture NLL, theta = (frac, mu, s, lambda).  weights may be NULL. */
int orc_unbinned_mix(int64_t n, const double *x, const double *weights, double lo, double hi,
                     const double *theta, double *value, double *grad, double *scale) {
    if (n < 0 || !(hi > lo)) return ORC_INVALID;
    const int32_t P = 4;
    tape T;
    accum A;
    if (!tape_init(&T, 256) || !accum_init(&A, P)) return ORC_INVALID;
    int32_t fr = t_var(&T, theta[0]);
    int32_t mu = t_var(&T, theta[1]);
    int32_t s = t_var(&T, theta[2]);
    int32_t lam = t_var(&T, theta[3]);
    /* prologue: the two normalisation integrals over [lo, hi] */
    int32_t zhi = t_div(&T, t_rsubc(&T, hi, mu), s);   /* (hi - mu)/s */
    int32_t zlo = t_div(&T, t_rsubc(&T, lo, mu), s);   /* (lo - mu)/s */
    int32_t ZG = t_sub(&T, rec_Phi(&T, zhi), rec_Phi(&T, zlo));
    int32_t ZE = t_sub(&T, t_exp(&T, t_mulc(&T, lam, -lo)), t_exp(&T, t_mulc(&T, lam, -hi)));
    int32_t one_m_f = t_rsubc(&T, 1.0, fr);
    A.mark = T.len;
    const double sqrt2pi = sqrt(2.0 * M_PI);
    for (int64_t i = 0; i < n; ++i) {
        double xi = x[i];
        /* Gaussian component: exp(-(x-mu)^2/(2 s^2)) / (s sqrt(2 pi)) / Z_G */
        int32_t d = t_rsubc(&T, xi, mu);
        int32_t q = t_div(&T, t_mul(&T, d, d), t_mulc(&T, t_mul(&T, s, s), 2.0));
        int32_t gN = t_div(&T, t_exp(&T, t_neg(&T, q)), t_mulc(&T, s, sqrt2pi));
        int32_t gpdf = t_div(&T, gN, ZG);
        /* exponential component: lambda exp(-lambda x) / Z_E */
        int32_t epdf = t_div(&T, t_mul(&T, lam, t_exp(&T, t_mulc(&T, lam, -xi))), ZE);
        int32_t p = t_add(&T, t_mul(&T, fr, gpdf), t_mul(&T, one_m_f, epdf));
        int32_t nll = t_neg(&T, t_log(&T, p));
        if (weights) nll = t_mulc(&T, nll, weights[i]);
        finish_term(&T, &A, nll);
    }
    int rc = finish(&T, &A, value, grad, scale);
    tape_free(&T);
    accum_free(&A);
    return rc;
}

/* 2-D binned Poisson NLL of K rotated Gaussians + constant. */
int orc_binned2d(int K, int64_t nx, int64_t ny, double lx, double hx, double ly, double hy,
                 const double *counts, const double *theta, double *value, double *grad,
                 double *scale) {
    if (K < 0 || nx < 0 || ny < 0) return ORC_INVALID;
    const int32_t P = 6 * K + 1;
    tape T;
    accum A;
    if (!tape_init(&T, 512) || !accum_init(&A, P)) return ORC_INVALID;
    for (int32_t k = 0; k < P; ++k) t_var(&T, theta[k]);
    /* prologue: cos(phi_k), sin(phi_k) */
    int32_t *cs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * K + 1));
    for (int k = 0; k < K; ++k) {
        cs[2 * k] = t_cos(&T, 6 * k + 5);
        cs[2 * k + 1] = t_sin(&T, 6 * k + 5);
    }
    A.mark = T.len;
    const int32_t C = 6 * K;
    double hxw = (hx - lx) / (double)nx, hyw = (hy - ly) / (double)ny;
    for (int64_t j = 0; j < ny; ++j) {
        double yc = ly + ((double)j + 0.5) * hyw;
        for (int64_t i = 0; i < nx; ++i) {
            double xc = lx + ((double)i + 0.5) * hxw;
            int32_t mu = C;
            for (int k = 0; k < K; ++k) {
                int32_t Ak = 6 * k, mx = 6 * k + 1, my = 6 * k + 2, sx = 6 * k + 3, sy = 6 * k + 4;
                int32_t c = cs[2 * k], s = cs[2 * k + 1];
                int32_t dx = t_rsubc(&T, xc, mx);
                int32_t dy = t_rsubc(&T, yc, my);
                int32_t u = t_add(&T, t_mul(&T, c, dx), t_mul(&T, s, dy));
                int32_t v = t_add(&T, t_neg(&T, t_mul(&T, s, dx)), t_mul(&T, c, dy));
                int32_t qu = t_div(&T, t_mul(&T, u, u), t_mul(&T, sx, sx));
                int32_t qv = t_div(&T, t_mul(&T, v, v), t_mul(&T, sy, sy));
                int32_t e = t_exp(&T, t_mulc(&T, t_add(&T, qu, qv), -0.5));
                mu = t_add(&T, mu, t_mul(&T, Ak, e));
            }
            double n = counts[j * nx + i];
            int32_t term = (n == 0.0) ? mu : t_sub(&T, mu, t_mulc(&T, t_log(&T, mu), n));
            finish_term(&T, &A, term);
        }
    }
    free(cs);
    int rc = finish(&T, &A, value, grad, scale);
    tape_free(&T);
    accum_free(&A);
    return rc;
}

/* The Gaussian of Listing 1 and its gradient with respect to (x, p):
 *   gauss(x, p, sigma) = (2 pi)^(-1/2) sigma^(-1/2) exp(-(x - p)^2 / (2 sigma^2)),
 * taken exactly as printed (including the sigma^(-1/2) factor). */
int orc_listing1_gauss(double x, double p, double sigma, double *value, double *dx, double *dp) {
    tape T;
    if (!tape_init(&T, 32)) return ORC_INVALID;
    int32_t X = t_var(&T, x), Pp = t_var(&T, p), S = t_var(&T, sigma);
    int32_t d = t_sub(&T, X, Pp);
    int32_t t = t_div(&T, t_neg(&T, t_mul(&T, d, d)), t_mulc(&T, t_mul(&T, S, S), 2.0));
    /* sigma^(-1/2) = exp(-log(sigma)/2) */
    int32_t sp = t_exp(&T, t_mulc(&T, t_log(&T, S), -0.5));
    int32_t g = t_mul(&T, t_mulc(&T, sp, pow(2.0 * M_PI, -0.5)), t_exp(&T, t));
    double *adj = (double *)calloc((size_t)T.len, sizeof(double));
    adj[g] = 1.0;
    for (int32_t i = T.len - 1; i >= 0; --i) {
        const node *nd = &T.n[i];
        if (nd->a >= 0) adj[nd->a] += adj[i] * nd->pa;
        if (nd->b >= 0) adj[nd->b] += adj[i] * nd->pb;
    }
    *value = T.n[g].v;
    *dx = adj[X];
    *dp = adj[Pp];
    free(adj);
    tape_free(&T);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Expression programs.                                                */
/* ------------------------------------------------------------------ */

/* Objective sum_e T_e of an expression program and its gradient: the nodes
 * (op[j], a[j], b[j], i[j], c[j]) in topological order, the last one the
 * per-element term T_e.  Operations: 0 constant c, 1 parameter theta[i],
 * 2 input i at the element, 3 the element index, 4 a+b, 5 a-b, 6 a*b,
 * 7 a/b, 8 -a, 9 exp a, 10 log a, 11 sqrt a, 12 erfc a, 13 a^i, 14 max(a, b)
 * (derivative to a when a >= b).  inputs: n_inputs arrays of n doubles.
 * Every element records all its nodes on the tape afresh (parameters are
 * the tape's leaves), is swept in reverse and popped: no hoisting of the
 * parameter-only part, so nothing but the definitions above is involved. */
int orc_expr(int n_nodes, const int32_t *op, const int32_t *na, const int32_t *nb, const int32_t *ni,
             const double *nc, int n_params, int n_inputs, const double *const *inputs, int64_t n,
             const double *theta, double *value, double *grad, double *scale) {
    if (n_nodes < 1 || n_params < 0 || n < 0) return ORC_INVALID;
    tape T;
    accum A;
    if (!tape_init(&T, 64 + 2 * n_nodes) || !accum_init(&A, n_params > 0 ? n_params : 1)) return ORC_INVALID;
    for (int k = 0; k < n_params; ++k) t_var(&T, theta[k]);
    A.P = n_params;
    A.mark = T.len;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_nodes);
    int rc = ORC_OK;
    for (int64_t e = 0; e < n && rc == ORC_OK; ++e) {
        for (int j = 0; j < n_nodes; ++j) {
            const int32_t a = na[j] >= 0 ? t[na[j]] : -1, b = nb[j] >= 0 ? t[nb[j]] : -1;
            switch (op[j]) {
                case 0: t[j] = t_const(&T, nc[j]); break;
                case 1:
                    if (ni[j] < 0 || ni[j] >= n_params) { rc = ORC_INVALID; break; }
                    t[j] = ni[j];
                    break;
                case 2:
                    if (ni[j] < 0 || ni[j] >= n_inputs) { rc = ORC_INVALID; break; }
                    t[j] = t_const(&T, inputs[ni[j]][e]);
                    break;
                case 3: t[j] = t_const(&T, (double)e); break;
                case 4: t[j] = t_add(&T, a, b); break;
                case 5: t[j] = t_sub(&T, a, b); break;
                case 6: t[j] = t_mul(&T, a, b); break;
                case 7: t[j] = t_div(&T, a, b); break;
                case 8: t[j] = t_neg(&T, a); break;
                case 9: t[j] = t_exp(&T, a); break;
                case 10: t[j] = t_log(&T, a); break;
                case 11: t[j] = t_sqrt(&T, a); break;
                case 12: t[j] = t_erfc(&T, a); break;
                case 13: t[j] = t_powi(&T, a, ni[j]); break;
                case 14: t[j] = t_max(&T, a, b); break;
                default: rc = ORC_INVALID;
            }
            if (rc != ORC_OK) break;
        }
        if (rc == ORC_OK) finish_term(&T, &A, t[n_nodes - 1]);
    }
    if (rc == ORC_OK) rc = finish(&T, &A, value, grad, scale);
    free(t);
    tape_free(&T);
    accum_free(&A);
    return rc;
}

