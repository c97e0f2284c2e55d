// cg_models_fp64.cuh -- FP64 forward + adjoint of the three model families on
// the table-driven FP64 functions of cg_fp64.cuh (the FP64 path of
// cg_batch_gradient / cg_gradient / cg_objective).
//
// Same reverse-mode structure and the same accumulators as the elements of
// cg_models.cuh (whose epilogue they feed), with three changes that cut FP64
// instructions and leave every value in FP64:
//  - exponentials as exp2 of exponents whose per-point constants carry
//    log2(e) (no extra instruction), reciprocals by frcp, logarithms by flog
//    or, for a plain sum of logs, by a running product (logprod_*);
//  - work that depends on the bin or event only (centre, weight 1/max(y,1),
//    y log y, the sign of y) is done once per element for all the points of
//    a multi-point tile (the elem functions take it precomputed);
//  - constant factors of an objective (-2 of chi2's adjoint, 2 of
//    Baker-Cousins) are applied to the per-thread sums once per tile
//    (exact: powers of two), and non-finite terms are detected from those
//    sums (a NaN or infinity in any term reaches the sum).
#pragma once
#include <type_traits>

#include "cg_fp64.cuh"
#include "cg_models.cuh"

namespace cg {

// ===========================================================================
// 1-D binned: K Gaussian peaks + polynomial of degree D.
// ===========================================================================

// log2(e)-scaled exponent coefficients of the peaks: e_k = 2^(c2_k d_k^2).
struct GP1C2 {
    double c2[CG_MAX_PEAKS_1D];
};

__device__ __forceinline__ void gp1_c2(const GP1Consts& cs, int K, GP1C2& c) {
    for (int k = 0; k < K; ++k) c.c2[k] = cs.c[k] * kLog2e;
}

// Point-independent part of one bin.
struct GP1Bin {
    double x, u, y;
    double ny;    // -y (Poisson / Baker-Cousins); chi2: the weight 1 / max(y, 1)
    double ymy;   // Baker-Cousins: y log y - y (0 for y = 0)
    bool ypos;    // y > 0 (Poisson / Baker-Cousins)
};

// max(y, 1) by an integer test of y's sign and exponent (y >= 1 exactly when
// its high word is at least that of 1.0 and the sign is clear).
__device__ __forceinline__ double max_y_1(double y) { return (__double2hiint(y) >= 0x3ff00000) ? y : 1.0; }

// PM: the polynomial's variable, x (0) or t = au x + bu (1), fixed at compile
// time so that neither is computed in vain.  DATA = false leaves out the
// Baker-Cousins term y log y - y, which depends on the count alone (callers
// that evaluate one histogram many times add its sum once instead).
template <int OBJ, int PM, bool DATA = true>
__device__ __forceinline__ GP1Bin gp1_bin(double x, double y, const GP1Data& d, const Fp64Tab& tab) {
    GP1Bin b;
    b.x = x;
    b.u = PM ? fma(x, d.au, d.bu) : x;
    b.y = y;
    b.ypos = __double_as_longlong(y) > 0;   // exact test of y > 0 (a NaN count reads as positive: its term is NaN)
    b.ymy = 0.0;
    if (OBJ == CG_OBJ_CHI2) {
        b.ny = frcp_any(max_y_1(y));
    } else {
        b.ny = -y;
        if (OBJ == CG_OBJ_POISSON_BC && DATA && b.ypos) b.ymy = fma(y, flog(y, tab), -y);
    }
    return b;
}

// One bin at one point.  Accumulators as gp1_elem_fp64 (value, per peak
// g e, g e d, g e d^2, then g u^j), except the scale: chi2 accumulates T in
// acc[0] and w r = -g/2 elsewhere (gp1_tile_scale multiplies those by -2);
// Poisson accumulates T and g; Baker-Cousins accumulates T/2 and g/2
// (gp1_tile_scale doubles everything).  D: the
// polynomial's degree (-1: none), fixed at compile time: with a run-time
// degree the compiler evaluates every Horner step and adjoint term of the
// largest degree and selects, several FP64 instructions per bin in vain.
// DATA as gp1_bin (false: the bin's y log y - y is not added).
template <int K, int OBJ, int D, bool DATA = true>
__device__ __forceinline__ void gp1_elem_f64(const GP1Bin& b, const GP1Consts& cs, const GP1C2& c2,
                                             const Fp64Tab& tab, double (&acc)[GP1Acc<K>::N], bool& bad) {
    double f = 0.0;
#pragma unroll
    for (int j = 3; j >= 0; --j) {   // Horner from the leading coefficient
        if (j == D) f = cs.poly[j];
        else if (j < D) f = fma(f, b.u, cs.poly[j]);
    }
    double dk[K > 0 ? K : 1], ek[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dk[k] = b.x - cs.mu[k];
        ek[k] = fexp2_prod(c2.c2[k] * dk[k], dk[k], tab);
        f = fma(cs.A[k], ek[k], f);
    }
    double g;
    if (OBJ == CG_OBJ_CHI2) {
        const double r = b.y - f;
        g = b.ny * r;                     // w r = -g/2
        acc[0] = fma(g, r, acc[0]);       // w r^2
    } else {
        double L, rf;
        if (fp64_fast_range(f)) {
            L = flog_fast(f, tab);
            rf = frcp(f);
        } else {
            L = flog_slow(f);
            rf = frcp_slow(f);
            bad |= b.ypos && !(f > 0.0);
        }
        if (b.ypos) {
            acc[0] += fma(b.ny, L, (OBJ == CG_OBJ_POISSON_BC && DATA) ? f + b.ymy : f);
            g = fma(b.ny, rf, 1.0);
        } else {                          // empty bin: T = f (2 f), even where f underflows to 0
            acc[0] += f;
            g = 1.0;
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double t = g * ek[k];
        const double td = t * dk[k];
        acc[1 + 3 * k] += t;
        acc[2 + 3 * k] += td;
        acc[3 + 3 * k] = fma(td, dk[k], acc[3 + 3 * k]);
    }
    if (D >= 0) acc[1 + 3 * K] += g;
    double up = b.u;
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        if (j <= D) acc[1 + 3 * K + j] = fma(g, up, acc[1 + 3 * K + j]);
        if (j < D) up *= b.u;
    }
}

// Calls f(std::integral_constant<int, D>, std::integral_constant<int, PM>)
// for the run-time degree d (-1..3) and polynomial mode pm: one switch per
// tile or evaluation, outside the bin loops, so that every bin loop is
// compiled for its degree.
template <typename F>
__device__ __forceinline__ void gp1_dispatch(int d, int pm, F&& f) {
#define CG_GP1_D(DD)                                                                              \
    case DD:                                                                                      \
        if (pm) f(std::integral_constant<int, DD>{}, std::integral_constant<int, 1>{});           \
        else f(std::integral_constant<int, DD>{}, std::integral_constant<int, 0>{});              \
        break;
    switch (d) {
        CG_GP1_D(-1) CG_GP1_D(0) CG_GP1_D(1) CG_GP1_D(2) CG_GP1_D(3)
        default: break;
    }
#undef CG_GP1_D
}

// The objective's constant factor of accumulator a (see gp1_elem_f64): a
// power of two, so applying it to a sum is exact.
template <int OBJ>
__device__ __forceinline__ double gp1_acc_factor(int a) {
    return OBJ == CG_OBJ_CHI2 ? (a == 0 ? 1.0 : -2.0) : (OBJ == CG_OBJ_POISSON_BC ? 2.0 : 1.0);
}

// The objective's constant factors on one thread's sums (see gp1_elem_f64).
template <int K, int OBJ>
__device__ __forceinline__ void gp1_tile_scale(double (&acc)[GP1Acc<K>::N]) {
    if (OBJ == CG_OBJ_CHI2) {
#pragma unroll
        for (int a = 1; a < GP1Acc<K>::N; ++a) acc[a] *= -2.0;
    } else if (OBJ == CG_OBJ_POISSON_BC) {
#pragma unroll
        for (int a = 0; a < GP1Acc<K>::N; ++a) acc[a] *= 2.0;
    }
}

// ===========================================================================
// Unbinned mixture: p = a 2^(c2 d^2) + b 2^(nl2 x + nl2lo),
// c2 = -log2(e)/(2 s^2), nl2 = -lambda log2(e), nl2lo = -nl2 lo (the
// exponent -lambda (x - lo) log2(e) in one FMA).  Accumulators as
// mix_elem_fp64, except that acc[5] accumulates V x and mix_tile_finish
// turns it into sum V (x - lo) = sum V x - lo sum V once per thread; without
// weights acc[0] is not touched per event: the log of p goes into the
// running product lp (mix_tile_finish adds its logarithm).
// ===========================================================================
struct MixC2 {
    double c2, nl2, nl2lo;
};

__device__ __forceinline__ void mix_c2(const MixConsts& cs, MixC2& c) {
    c.c2 = cs.c * kLog2e;
    c.nl2 = -cs.lam * kLog2e;
    c.nl2lo = -c.nl2 * cs.lo;
}

template <bool W>
__device__ __forceinline__ void mix_elem_f64(double x, double w, const MixConsts& cs, const MixC2& c2,
                                             const Fp64Tab& tab, double (&acc)[MixAcc::N], LogProd& lp,
                                             bool& bad) {
    const double d = x - cs.mu;
    const double eG = fexp2((c2.c2 * d) * d, tab);
    const double eE = fexp2(fma(c2.nl2, x, c2.nl2lo), tab);
    const double p = fma(cs.a, eG, cs.b * eE);
    double r;
    if (fp64_fast_range(p)) {
        r = frcp(p);
        if (W) acc[0] = fma(w, flog_fast(p, tab), acc[0]);
        else logprod_mul(lp, p);
    } else {                              // p <= 0, subnormal, huge or NaN: IEEE path
        r = frcp_slow(p);
        acc[0] += W ? w * flog_slow(p) : flog_slow(p);
        bad |= !(p > 0.0);
    }
    if (W) r *= w;
    const double U = eG * r, V = eE * r;
    const double Ud = U * d;
    acc[1] += U;
    acc[2] += Ud;
    acc[3] = fma(Ud, d, acc[3]);
    acc[4] += V;
    acc[5] = fma(V, x, acc[5]);
}

// End of a thread's events: sum V (x - lo) from sum V x and sum V, and the
// log of the running product into the value (without weights).
template <bool W>
__device__ __forceinline__ void mix_tile_finish(const MixConsts& cs, const Fp64Tab& tab, double (&acc)[MixAcc::N],
                                                const LogProd& lp) {
    acc[5] = fma(-cs.lo, acc[4], acc[5]);
    if (!W) acc[0] += logprod_log(lp, tab);
}

// ---------------------------------------------------------------------------
// Ratio form of the same mixture, for a > 0 and b > 0: one exponential per
// event instead of two.
//   p = b eE (1 + u),  u = a eG / (b eE) = 2^t,
//   t = c2 d^2 + lam log2(e) (x - lo) + log2(a / b).
// With s = 1 + u, V = 1/s and r = u V (the Gaussian's share of p; the
// exponential's is V = 1 - r):
//   eG / p = r / a,  eE / p = V / b,  log p = log b - lam (x - lo) + log s.
// A thread sums r (1, d, d^2), V (1, x) and the running product of s;
// mix_ratio_sums turns a tile's block sums into the accumulators of
// mix_elem_f64 (same meaning, same epilogue).  The sum of x - lo that the
// value needs follows from r + V = 1 without an accumulator of its own:
//   sum (x - lo) = sum V (x - lo) + sum r d + (mu - lo) sum r.
// An event whose s leaves the fast range (u above 2^1021, or NaN) is taken
// in the two-exponential form by mix_ratio_slow.
// ---------------------------------------------------------------------------
struct MixR2 {
    double c2;    // -log2(e) / (2 s^2)
    double ml2;   // lam log2(e)
    double k0;    // log2(a / b) - lam log2(e) lo
    double lb;    // log b
    int ok;       // a > 0, b > 0, k0 and lb finite: the ratio form applies
};

__device__ inline void mix_r2(const MixConsts& cs, MixR2& c) {
    c.c2 = cs.c * kLog2e;
    c.ml2 = cs.lam * kLog2e;
    const bool pos = cs.a > 0.0 && cs.b > 0.0;
    c.k0 = pos ? fma(-c.ml2, cs.lo, log2(cs.a) - log2(cs.b)) : 0.0;
    c.lb = pos ? log(cs.b) : 0.0;
    c.ok = pos && isfinite(c.k0) && isfinite(c.lb) && isfinite(c.c2) && isfinite(c.ml2);
}

// One event in the two-exponential form, returning the ratio form's r, V
// and log s (IEEE reciprocal and log; rare, out of line).
static __device__ __noinline__ void mix_ratio_slow(double x, double d, const MixConsts& cs, const MixR2& c,
                                                   const Fp64Tab& tab, double& r, double& V, double& ls,
                                                   bool& bad) {
    const double xl = x - cs.lo;
    const double aG = cs.a * fexp2((c.c2 * d) * d, tab);
    const double bE = cs.b * fexp2(-c.ml2 * xl, tab);
    const double p = aG + bE;
    bad |= !(p > 0.0);
    const double ip = 1.0 / p;
    r = aG * ip;
    V = bE * ip;
    ls = fma(cs.lam, xl, log(p) - c.lb);
}

template <bool W>
__device__ __forceinline__ void mix_elem_ratio(double x, double w, const MixConsts& cs, const MixR2& c,
                                               const Fp64Tab& tab, double (&acc)[MixAcc::N], LogProd& lp,
                                               bool& bad) {
    const double d = x - cs.mu;
    const double u = fexp2(fma(c.c2 * d, d, fma(c.ml2, x, c.k0)), tab);
    const double s = 1.0 + u;
    double r, V;
    if (fp64_fast_range(s)) {             // s in [1, 2^1021): every event but the most extreme
        V = frcp(s);
        if (W) {
            acc[0] = fma(w, flog_fast(s, tab), acc[0]);
            V *= w;
        } else {
            logprod_mul(lp, s);
        }
        r = u * V;
    } else {
        double ls;
        mix_ratio_slow(x, d, cs, c, tab, r, V, ls, bad);
        if (W) {
            r *= w;
            V *= w;
        }
        acc[0] += W ? w * ls : ls;
    }
    const double rd = r * d;
    acc[1] += r;
    acc[2] += rd;
    acc[3] = fma(rd, d, acc[3]);
    acc[4] += V;
    acc[5] = fma(V, x, acc[5]);
}

// Lean ratio form: as mix_elem_ratio, but only the Gaussian's sums r (1, d,
// d^2) and the logs per event (21 FP64 instructions instead of 23 without
// weights); the exponential's sums follow per tile from V = 1 - r and the
// chunk's sums of the data (mix_lean_sums).
template <bool W>
__device__ __forceinline__ void mix_elem_lean(double x, double w, const MixConsts& cs, const MixR2& c,
                                              const Fp64Tab& tab, double (&acc)[MixAcc::N], LogProd& lp,
                                              bool& bad) {
    const double d = x - cs.mu;
    const double u = fexp2(fma(c.c2 * d, d, fma(c.ml2, x, c.k0)), tab);
    const double s = 1.0 + u;
    double r;
    if (fp64_fast_range(s)) {
        const double V = frcp(s);
        if (W) acc[0] = fma(w, flog_fast(s, tab), acc[0]);
        else logprod_mul(lp, s);
        r = u * V;
        if (W) r *= w;
    } else {
        double V, ls;
        mix_ratio_slow(x, d, cs, c, tab, r, V, ls, bad);
        if (W) r *= w;
        acc[0] += W ? w * ls : ls;
    }
    const double rd = r * d;
    acc[1] += r;
    acc[2] += rd;
    acc[3] = fma(rd, d, acc[3]);
}

// A tile's block sums of the ratio form (after mix_tile_finish: tot[5] is
// sum V (x - lo)) into the accumulators of mix_elem_f64.  n_w and sxl: the
// tile's event count (or sum of weights) and sum w (x - lo), from the data.
__device__ inline void mix_ratio_sums(const MixConsts& cs, const MixR2& c, double n_w, double sxl, double* tot) {
    tot[0] = fma(n_w, c.lb, fma(-cs.lam, sxl, tot[0]));
    tot[1] /= cs.a;
    tot[2] /= cs.a;
    tot[3] /= cs.a;
    tot[4] /= cs.b;
    tot[5] /= cs.b;
}

// The same for the lean form: the exponential's sums as differences,
//   sum w V = n_w - sum w r,  sum w V (x - lo) = sxl - (sum w r d + (mu - lo) sum w r).
// Returns false, leaving tot as it is, where either difference is below 1/16
// of its first term (the subtraction would cancel more than 4 bits): the
// tile is then summed again in the full ratio form.
__device__ inline bool mix_lean_sums(const MixConsts& cs, const MixR2& c, double n_w, double sxl, double* tot) {
    const double sv = n_w - tot[1];
    const double svx = sxl - fma(cs.mu - cs.lo, tot[1], tot[2]);
    if (!(sv >= 0.0625 * n_w && svx >= 0.0625 * sxl)) return false;
    tot[4] = sv;
    tot[5] = svx;
    mix_ratio_sums(cs, c, n_w, sxl, tot);
    return true;
}

// ===========================================================================
// 2-D binned Poisson NLL of K rotated Gaussians + C.  The exponent is taken
// as a quadratic form in (dx, dy) = (x - mu_x, y - mu_y):
//   q log2(e) = qa dx^2 + 2 qb dx dy + qc dy^2,
//   qa = (al c^2 + be s^2) log2 e, qb = (al - be) c s log2 e,
//   qc = (al s^2 + be c^2) log2 e   (c, s = cos, sin phi),
// and the adjoint sums are kept in (dx, dy): sum g e (1, dx, dy, dx^2, dy^2,
// dx dy); rg2_rotate_moments turns them into the (u, v) sums of rg2_elem_fp64
// (1, u, v, u^2, v^2, u v) once per tile, a rotation of the moments.
// ===========================================================================
struct RG2Q {
    double qa[CG_MAX_PEAKS_2D], qb2[CG_MAX_PEAKS_2D], qc[CG_MAX_PEAKS_2D];   // qb2 = 2 qb (tile culling)
};

// The Gaussians that survive a tile's culling, packed in slots 0 .. n-1 (see
// rg2_act_one and the column form below).
struct RG2Act {
    double A[CG_MAX_PEAKS_2D], mx[CG_MAX_PEAKS_2D], my[CG_MAX_PEAKS_2D];
    double sa[CG_MAX_PEAKS_2D], ca[CG_MAX_PEAKS_2D], sb[CG_MAX_PEAKS_2D], cb[CG_MAX_PEAKS_2D];
    // the row recurrence (rg2_act_rec): 2 sa H, 2 cb H, (sa^2 + cb^2) H^2, and
    // q - 1 (NaN where |q - 1| is too large for the series: no recurrence)
    double a2[CG_MAX_PEAKS_2D], b2[CG_MAX_PEAKS_2D], kk[CG_MAX_PEAKS_2D], qm[CG_MAX_PEAKS_2D];
    int k[CG_MAX_PEAKS_2D];   // the Gaussian's index in the parameter vector
    int n;                    // how many survive
};

__device__ __forceinline__ void rg2_q_one(const RG2Consts& c, int k, RG2Q& q) {
    const double cs = c.cs[k], sn = c.sn[k], al = c.al[k], be = c.be[k];
    q.qa[k] = fma(al, cs * cs, be * sn * sn) * kLog2e;
    q.qb2[k] = 2.0 * ((al - be) * cs * sn) * kLog2e;
    q.qc[k] = fma(al, sn * sn, be * cs * cs) * kLog2e;
}

// Gaussian k into slot j of the tile's kept set: the exponent evaluated per
// bin as -(u'^2 + v'^2), u' = ra u, v' = rb v, ra = sqrt(-al log2 e),
// rb = sqrt(-be log2 e):  u' = sa dy + ca dx, v' = cb dy - sb dx
// (sa = ra s, ca = ra c, sb = rb s, cb = rb c).
__device__ __forceinline__ void rg2_act_one(const RG2Consts& c, int k, int j, RG2Act& a) {
    const double ra = sqrt(-c.al[k] * kLog2e), rb = sqrt(-c.be[k] * kLog2e);
    a.A[j] = c.A[k];
    a.mx[j] = c.mx[k];
    a.my[j] = c.my[k];
    a.sa[j] = ra * c.sn[k];
    a.ca[j] = ra * c.cs[k];
    a.sb[j] = rb * c.sn[k];
    a.cb[j] = rb * c.cs[k];
    a.k[j] = k;
}

// ---------------------------------------------------------------------------
// Row recurrence of the factors down a column.  With x fixed the exponent
// e(dy) = -(u'^2 + v'^2) is a concave parabola in dy, so for the rows
// dy_j = dy_0 + j H of one thread,
//   e_{j+1} = e_j R_j,  R_j = 2^(-(u'_j 2 sa H + v'_j 2 cb H + (sa^2 + cb^2) H^2)),
//   R_{j+1} = R_j q,    q = 2^(-2 (sa^2 + cb^2) H^2)
// (e_j here the factor 2^e(dy_j)).  After two exponentials at the start of
// a run each further factor costs a product and an FMA, R + R (q - 1), in
// place of u', v', v'^2, an FMA and exp2 (11 FP64 instructions).  q - 1 is
// taken from its Taylor series to degree 8 (|2 (sa^2 + cb^2) H^2| < 2^-6:
// below 1e-20 absolute), not through the table, so no rounding is shared by
// all runs of a Gaussian beyond that of (sa^2 + cb^2) H^2 itself (its effect
// after j steps, j^2/2 |q - 1| 2^-52, stays near 1e-15 on 32 steps); R_0
// comes from its own exponential per run.  The kernel takes the recurrence
// only where every kept Gaussian's exponent at both ends of every thread's
// run is above -1000 (so every factor and ratio is normal), else the direct
// form for the whole tile.
// ---------------------------------------------------------------------------
constexpr double kRgRecQMax = 0.015625;   // |2 (sa^2 + cb^2) H^2| below 2^-6

__device__ __forceinline__ void rg2_act_rec(int j, double H, RG2Act& a) {
    const double sa = a.sa[j], cb = a.cb[j];
    a.a2[j] = (2.0 * H) * sa;
    a.b2[j] = (2.0 * H) * cb;
    const double kk = fma(sa, sa, cb * cb) * (H * H);
    a.kk[j] = kk;
    const double lq = -2.0 * kk;
    double qm = __longlong_as_double(0x7ff8000000000000LL);
    if (fabs(lq) < kRgRecQMax) {   // q - 1 = e^z - 1, z = lq ln 2, Horner to degree 8
        const double z = lq * 0.6931471805599453;
        double t = 1.0 + z * (1.0 / 8.0);
        t = fma(z * (1.0 / 7.0), t, 1.0);
        t = fma(z * (1.0 / 6.0), t, 1.0);
        t = fma(z * (1.0 / 5.0), t, 1.0);
        t = fma(z * (1.0 / 4.0), t, 1.0);
        t = fma(z * (1.0 / 3.0), t, 1.0);
        t = fma(z * 0.5, t, 1.0);
        qm = z * t;
    }
    a.qm[j] = qm;
}

// Largest exponent (log2 units) of Gaussian k over the box [X0, X1] x [Y0, Y1]
// of offsets (dx, dy) from its centre: the exponent qa dx^2 + qb2 dx dy +
// qc dy^2 is a concave quadratic, so its maximum over the box is 0 when the
// centre lies inside, else on one of the four edges, where it is a concave
// parabola maximised at its vertex clamped to the edge.  NaN for degenerate
// coefficients (the caller keeps the Gaussian then).
__device__ __forceinline__ double rg2_box_max_exponent(const RG2Q& q, int k, double X0, double X1, double Y0,
                                                       double Y1) {
    if (X0 <= 0.0 && 0.0 <= X1 && Y0 <= 0.0 && 0.0 <= Y1) return 0.0;
    const double qa = q.qa[k], qb2 = q.qb2[k], qc = q.qc[k];
    const auto E = [&](double dx, double dy) { return fma(dx, fma(qa, dx, qb2 * dy), (qc * dy) * dy); };
    const auto clamp = [](double v, double lo, double hi) { return fmin(fmax(v, lo), hi); };
    const double ry = -0.5 * qb2 / qc, rx = -0.5 * qb2 / qa;   // vertices: dy* = ry dx, dx* = rx dy
    double m = E(X0, clamp(ry * X0, Y0, Y1));
    m = fmax(m, E(X1, clamp(ry * X1, Y0, Y1)));
    m = fmax(m, E(clamp(rx * Y0, X0, X1), Y0));
    m = fmax(m, E(clamp(rx * Y1, X0, X1), Y1));
    return (qa < 0.0 && qc < 0.0) ? m : __longlong_as_double(0x7ff8000000000000LL);
}

// ---------------------------------------------------------------------------
// Column form of the element, for a thread that walks one column of bins
// (x fixed), over the NA Gaussians that survive the tile's culling, packed
// in RG2Act (NA fixed at compile time: a culled Gaussian costs nothing,
// where a run-time skip inside an unrolled loop leaves its instructions
// issued with every lane predicated off).  The exponent is taken in the
// Gaussian's own axes, scaled,
//   q log2(e) = -(u'^2 + v'^2),  u' = sa dy + ua,  v' = cb dy - vb,
// with the column's parts ua = ca dx, vb = sb dx once per tile: a sum of two
// squares, so its rounding error stays near eps |q| however elongated the
// Gaussian (expanding the quadratic form in dx, dy instead cancels terms
// larger than q by the squared aspect ratio).  The adjoint moments are kept
// in (dx, dy) and, since dx is fixed, those with dx follow from sums over dy
// alone:  sum w dx = dx sum w,  sum w dx^2 = dx^2 sum w,  sum w dx dy = dx sum w dy.
// A thread sums [ T | (w, w dy, w dy^2) per kept Gaussian | g ], w = g e_j;
// rg2_col_moments turns its sums into [ T | (S, Sx, Sy, Sxx, Syy, Sxy) per
// kept Gaussian | sum g ], the layout of rg2_elem_fp64's accumulators over
// the kept Gaussians.
// ---------------------------------------------------------------------------
template <int NA>
struct RG2Col {
    double dx[NA > 0 ? NA : 1], ua[NA > 0 ? NA : 1], vb[NA > 0 ? NA : 1];
};

template <int NA>
__device__ __forceinline__ void rg2_col(double x, const RG2Act& a, RG2Col<NA>& col) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const double dx = x - a.mx[j];
        col.dx[j] = dx;
        col.ua[j] = a.ca[j] * dx;
        col.vb[j] = a.sb[j] * dx;
    }
}

// One bin from the kept Gaussians' dy_j and factors e_j (the direct form
// rg2_elem_col takes them per bin; the row recurrence from the run).
template <int NA>
__device__ __forceinline__ void rg2_elem_col_de(double n, double C, const RG2Act& a,
                                                const double (&dy)[NA > 0 ? NA : 1],
                                                const double (&e)[NA > 0 ? NA : 1], const Fp64Tab& tab,
                                                double (&acc)[2 + 3 * NA], bool& bad) {
    double mu = C;
#pragma unroll
    for (int j = 0; j < NA; ++j) mu = fma(a.A[j], e[j], mu);
    const bool npos = __double_as_longlong(n) > 0;
    double L, rm;
    if (fp64_fast_range(mu)) {
        L = flog_fast(mu, tab);
        rm = frcp(mu);
    } else {
        L = flog_slow(mu);
        rm = frcp_slow(mu);
        bad |= npos && !(mu > 0.0);
    }
    const double g = npos ? fma(-n, rm, 1.0) : 1.0;
    acc[0] += npos ? fma(-n, L, mu) : mu;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const double w = g * e[j];
        const double wy = w * dy[j];
        acc[1 + 3 * j] += w;
        acc[2 + 3 * j] += wy;
        acc[3 + 3 * j] = fma(wy, dy[j], acc[3 + 3 * j]);
    }
    acc[1 + 3 * NA] += g;
}

template <int NA>
__device__ __forceinline__ void rg2_elem_col(double y, double n, double C, const RG2Act& a, const RG2Col<NA>& col,
                                             const Fp64Tab& tab, double (&acc)[2 + 3 * NA], bool& bad) {
    double dy[NA > 0 ? NA : 1], e[NA > 0 ? NA : 1];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        dy[j] = y - a.my[j];
        const double up = fma(a.sa[j], dy[j], col.ua[j]), vp = fma(a.cb[j], dy[j], -col.vb[j]);
        e[j] = fexp2(fma(-up, up, -(vp * vp)), tab);
    }
    rg2_elem_col_de<NA>(n, C, a, dy, e, tab, acc, bad);
}

// The exponent of slot j at offset dy of a column (rg2_elem_col's form).
template <int NA>
__device__ __forceinline__ double rg2_col_exponent(const RG2Act& a, const RG2Col<NA>& col, int j, double dy,
                                                   double& up, double& vp) {
    up = fma(a.sa[j], dy, col.ua[j]);
    vp = fma(a.cb[j], dy, -col.vb[j]);
    return fma(-up, up, -(vp * vp));
}

// One thread's column-form sums into (dx, dy) moments (layout above).
template <int NA>
__device__ __forceinline__ void rg2_col_moments(const RG2Col<NA>& col, const double (&c)[2 + 3 * NA],
                                                double (&m)[2 + 6 * NA]) {
    m[0] = c[0];
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const double dx = col.dx[j], S = c[1 + 3 * j], Sy = c[2 + 3 * j];
        const double Sx = dx * S;
        m[1 + 6 * j] = S;
        m[2 + 6 * j] = Sx;
        m[3 + 6 * j] = Sy;
        m[4 + 6 * j] = dx * Sx;
        m[5 + 6 * j] = c[3 + 3 * j];
        m[6 + 6 * j] = dx * Sy;
    }
    m[1 + 6 * NA] = c[1 + 3 * NA];
}

// (dx, dy) moments of one Gaussian -> (u, v) moments, in place: S[0..5] =
// sum g e (1, dx, dy, dx^2, dy^2, dx dy) on entry, (1, u, v, u^2, v^2, u v) on exit,
// u = c dx + s dy, v = -s dx + c dy.
__device__ __forceinline__ void rg2_rotate_moments(double* S, double cs, double sn) {
    const double Sx = S[1], Sy = S[2], Sxx = S[3], Syy = S[4], Sxy = S[5];
    S[1] = fma(cs, Sx, sn * Sy);
    S[2] = fma(cs, Sy, -sn * Sx);
    const double cc = cs * cs, ss = sn * sn, c2s = 2.0 * cs * sn;
    S[3] = fma(cc, Sxx, fma(c2s, Sxy, ss * Syy));
    S[4] = fma(ss, Sxx, fma(-c2s, Sxy, cc * Syy));
    S[5] = fma(cs * sn, Syy - Sxx, (cc - ss) * Sxy);
}

}  // namespace cg
