// cg_fp64.cuh -- FP64 elementary functions of the fused FP64 kernels.
//
// GB300's FP64 unit issues 2 DFMA per clock per SM (one warp instruction per
// 16 cycles), against 64-128 lanes per clock for integer and FP32 work, so in
// an FP64 kernel every FP64 instruction counts and integer work is nearly
// free.  These functions keep every value in FP64 and move only the parts
// that are exact in integer arithmetic (rounding to a grid, table indices,
// exponent fields) off the FP64 unit.  Own implementations of published
// methods:
//
//  exp2 (P. T. P. Tang, "Table-driven implementation of the exponential
//  function in IEEE floating-point arithmetic", ACM TOMS 15(2), 1989, with
//  base 2 and a 4096-entry table): y = n/4096 + r with n = round(4096 y),
//  |r| <= 2^-13, and 2^y = 2^(n >> 12) * T[n & 4095] * e^(r ln2), T[j] =
//  2^(j/4096) rounded to nearest (cg_fp64_tables.inc), e^(r ln2) - 1 by its
//  Taylor polynomial to degree 3 (the first dropped term is below 2.2e-18).
//  The rounding of y to the 1/4096 grid is the addition of 1.5 * 2^40 (whose
//  ulp is 2^-12), and r = y - round(y) is then exact (Sterbenz).  FP64
//  instructions: 3 for the reduction, 3 for the polynomial, 1 for T (1 + p);
//  the factor 2^(n >> 12) is an integer add to the exponent field.  Error:
//  table 0.5 ulp + final rounding 0.5 ulp + polynomial below 0.1 ulp.
//  Callers fold log2(e) into their per-point constants, so e^q is computed
//  as exp2 of q log2(e) with no extra instruction.  For an exponent that is
//  a product a b (a peak's c2 d x d) the product is folded into the
//  reduction (fexp2_prod): one instruction fewer and no rounding of a b.
//
//  reciprocal: the hardware estimate rcp.approx.ftz.f64 refined by one
//  third-order Newton-Raphson step, r = r0 (1 + e + e^2) with e = 1 - p r0
//  (three FMAs): a relative error eps of r0 becomes eps^3 plus the final
//  rounding.
//
//  log (P. T. P. Tang, "Table-driven implementation of the logarithm
//  function in IEEE floating-point arithmetic", ACM TOMS 16(4), 1990, with
//  130 breakpoints): p = 2^E m with m in [sqrt 2 / 2, sqrt 2), F = the
//  breakpoint nearest m on the grid of 1/128 (m >= 1) or 1/256 (m < 1),
//  u = (m - F)/F with m - F exact (Sterbenz) and |u| <= 2^-8, log p =
//  E ln2 + log F + log1p(u), log1p by its Taylor polynomial to degree 7
//  (the first dropped term is below 0.05 ulp of log1p(u)).  F = 1 is a
//  breakpoint, so next to p = 1 the result is log1p(u) itself and keeps its
//  relative accuracy.  Tables log F and 1/F rounded to nearest.  FP64
//  instructions: 2 for u, 7 for the polynomial, 1 for the conversion of E,
//  3 to combine.  Error: below 1.9 ulp of the exact value (an exact CPU
//  emulation of these steps over 9,000 arguments, most of them near 1).
//
//  sum of logarithms: sum_i log p_i = log prod_i p_i.  A running product
//  m 2^E with m in [1, 2) takes one DMUL per factor; its exponent is moved
//  into the integer E after every factor (integer operations), so it can
//  neither overflow nor underflow, and one log call per flush gives
//  E ln2 + log m.  Each product adds at most 2^-53 relative error, i.e. at
//  most 1.1e-16 absolute to the sum of logs, the same order as summing
//  correctly rounded logarithms.
//
//  The tables live in shared memory (Fp64Tab, 35 KB, loaded once per block
//  by fp64_tab_load): random per-lane indices cost a few shared-memory
//  wavefronts, far below the 16 cycles of one FP64 warp instruction.
#pragma once
#include <math.h>
#include <stdint.h>

#include "cg_fp64_tables.inc"

namespace cg {

constexpr int kExp2Bits = 12;
constexpr int kExp2N = 1 << kExp2Bits;
constexpr double kLog2e = 1.4426950408889634074;   // log2(e), the double nearest
constexpr double kLn2Hi = 0x1.62e42fefa39efp-1;     // ln 2 = kLn2Hi + kLn2Lo to 2^-108
constexpr double kLn2Lo = 0x1.abc9e3b39803fp-56;

constexpr int kLogN = 130;   // log breakpoints: 54 in [1, sqrt 2), 76 in [sqrt 2 / 2, 1]

// The lookup tables of one block, in shared memory: exp2 entries, then
// (log F_j, 1/F_j) pairs so that one 16-byte load fetches both.
struct Fp64Tab {
    double exp2[kExp2N];
    double2 logf[kLogN];
};

// Copy the tables into shared memory (the log table only with LOG); every
// thread of the block calls it, the caller synchronises.
template <bool LOG = true>
__device__ __forceinline__ void fp64_tab_load(Fp64Tab& s) {
    const double2* src = reinterpret_cast<const double2*>(g_exp2_tab);
    double2* dst = reinterpret_cast<double2*>(s.exp2);
    for (int i = threadIdx.x; i < kExp2N / 2; i += blockDim.x) dst[i] = src[i];
    if (LOG)
        for (int i = threadIdx.x; i < kLogN; i += blockDim.x) s.logf[i] = make_double2(g_log_tab[i], g_invf_tab[i]);
}

// 2^y for |y| < 1022 (no range check): the result is normal.
__device__ __forceinline__ double exp2_core(double y, const Fp64Tab& tab) {
    const double S = 1649267441664.0;          // 1.5 * 2^40: ulp 2^-12
    const double ks = y + S;                   // S + n / 4096, n = round(4096 y)
    const double kd = ks - S;                  // n / 4096 (exact)
    const double r = y - kd;                   // exact, |r| <= 2^-13
    const int n = __double2loint(ks);          // low word of S + n ulp = n (two's complement)
    const double t = tab.exp2[n & (kExp2N - 1)];
    // e^(r ln2) - 1 = r (b1 + r (b2 + r b3)), b_k = (ln 2)^k / k!
    const double b1 = 0.6931471805599453, b2 = 0.24022650695910072, b3 = 0.05550410866482158;
    const double p = r * fma(r, fma(r, b3, b2), b1);
    const double v = fma(t, p, t);             // in [1, 2.0002]
    return __hiloint2double(__double2hiint(v) + (n >> kExp2Bits) * (1 << 20), __double2loint(v));
}

// 2^y for |y| >= 1022, infinities and NaN (rare, out of line).
static __device__ __noinline__ double exp2_slow(double y, const Fp64Tab& tab) {
    if (y != y) return y;
    if (y >= 1024.0) return __longlong_as_double(0x7ff0000000000000LL);
    if (y < -1075.0) return 0.0;
    if (y > 0.0) return exp2_core(y - 64.0, tab) * 18446744073709551616.0;   // 2^(y-64) * 2^64
    return exp2_core(y + 512.0, tab) * 0x1p-512;                              // one rounding (subnormal)
}

// 2^y, y in FP64; tab: the tables in shared memory.  Arguments below -1075
// (far tails of narrow peaks) return 0 after two integer tests.
__device__ __forceinline__ double fexp2(double y, const Fp64Tab& tab) {
    const int yh = __double2hiint(y);
    const int ya = yh & 0x7fffffff;
    if (ya >= 0x408ff000) {                                     // |y| >= 1022, inf or NaN
        if (yh < 0 && ya >= 0x4090cc00 && ya < 0x7ff00000) return 0.0;   // -inf < y <= -1075
        return exp2_slow(y, tab);
    }
    return exp2_core(y, tab);
}

// 2^(a b) of the exact product a b: the product enters the reduction itself,
// ks = fma(a, b, S) rounds a b to the 1/4096 grid and r = fma(a, b, -kd) is
// the exact remainder, so the product is never rounded on its own (no
// |a b| 2^-53 error from it) and takes no instruction of its own: 7 FP64
// instructions against 8 for fexp2(a * b).  Far tails first, by integer
// tests alone: the high word of |x| read as a fixed-point number with 20
// fraction bits is 1023 + e + m for |x| = 2^e (1 + m), a lower bound of
// 1023 + log2 |x| (m <= log2(1 + m) on [0, 1]), so the two high words add up
// to at most 2046 + log2 |a b|; from 2046 + log2(1076) on, 2^(a b) is 0 for
// a finite negative product (the far side of a narrow peak, most bins of a
// wide histogram) without any FP64 instruction.  Overflow, infinities and
// NaN, and 1022 <= |kd| below that bound, go to fexp2 of the rounded
// product.
__device__ __forceinline__ double fexp2_prod(double a, double b, const Fp64Tab& tab) {
    const int ha = __double2hiint(a), hb = __double2hiint(b);
    if ((unsigned)(ha & 0x7fffffff) + (unsigned)(hb & 0x7fffffff) >= 2155947190U) {   // |a b| >= 1076, or inf / NaN
        const bool finite = (ha & 0x7ff00000) != 0x7ff00000 && (hb & 0x7ff00000) != 0x7ff00000;
        if (finite && (ha ^ hb) < 0) return 0.0;                          // a b <= -1076
        return fexp2(a * b, tab);
    }
    const double S = 1649267441664.0;          // 1.5 * 2^40: ulp 2^-12
    const double ks = fma(a, b, S);            // S + n / 4096, n = round(4096 a b)
    const double kd = ks - S;                  // n / 4096 (exact)
    if ((__double2hiint(kd) & 0x7fffffff) >= 0x408ff000) return fexp2(a * b, tab);
    const double r = fma(a, b, -kd);           // a b - n / 4096, |r| <= 2^-13 (one rounding below 2^-66)
    const int n = __double2loint(ks);
    const double t = tab.exp2[n & (kExp2N - 1)];
    const double b1 = 0.6931471805599453, b2 = 0.24022650695910072, b3 = 0.05550410866482158;
    const double p = r * fma(r, fma(r, b3, b2), b1);
    const double v = fma(t, p, t);
    return __hiloint2double(__double2hiint(v) + (n >> kExp2Bits) * (1 << 20), __double2loint(v));
}

// e^q = 2^(q log2 e); the kernels fold log2(e) into their constants instead.
// The rounding of the product adds |q| 2^-53 relative error (the condition
// number of exp), the same order as the rounding of q itself.
__device__ __forceinline__ double fexp(double q, const Fp64Tab& tab) { return fexp2(q * kLog2e, tab); }

// 1/p for positive normal p (the callers check the range): hardware estimate
// and one third-order Newton-Raphson step.
__device__ __forceinline__ double frcp(double p) {
    double r0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(p));
    const double e = fma(-p, r0, 1.0);
    return fma(r0, fma(e, e, e), r0);
}

// True when p is positive, normal, finite and below 2^1022: the range in
// which frcp and the running product below are valid (integer test).
__device__ __forceinline__ bool fp64_fast_range(double p) {
    return (unsigned)(__double2hiint(p) - 0x00100000) < (unsigned)(0x7fd00000 - 0x00100000);
}

// log p for p in the fast range (fp64_fast_range).
__device__ __forceinline__ double flog_fast(double p, const Fp64Tab& tab) {
    const int hi = __double2hiint(p);
    const int mh = hi & 0x000fffff;                             // top 20 fraction bits
    const int big = mh >= 0x6a09e ? 1 : 0;                      // m >= sqrt 2: take m/2 and E + 1
    const int base = big ? 0x3fe00000 : 0x3ff00000;
    const double m = __hiloint2double(base | mh, __double2loint(p));       // [sqrt 2 / 2, sqrt 2)
    const int j = (mh + 0x1000) >> 13;                          // 7 fraction bits, rounded: 0..128
    const double F = __hiloint2double(base + (j << 13), 0);    // nearest breakpoint (j = 128: F = 1)
    const double2 lt = tab.logf[j + big];                       // (log F, 1/F)
    const double u = (m - F) * lt.y;
    // log1p(u) = u + u^2 (-1/2 + u (1/3 + u (-1/4 + u (1/5 + u (-1/6 + u/7)))))
    double c = fma(u, 0.14285714285714285, -0.16666666666666666);
    c = fma(u, c, 0.2);
    c = fma(u, c, -0.25);
    c = fma(u, c, 0.33333333333333333);
    c = fma(u, c, -0.5);
    const double l1 = fma(u * u, c, u);
    const double ed = (double)((hi >> 20) - 1023 + big);
    return fma(ed, kLn2Hi, lt.x) + fma(ed, kLn2Lo, l1);
}

// log p for any p (IEEE semantics outside the fast range, through the CUDA
// math library there: zero, subnormal, huge, negative, infinite, NaN).
static __device__ __noinline__ double flog_slow(double p) { return log(p); }

__device__ __forceinline__ double flog(double p, const Fp64Tab& tab) {
    return fp64_fast_range(p) ? flog_fast(p, tab) : flog_slow(p);
}

// 1/p for any p (IEEE division outside the fast range).
static __device__ __noinline__ double frcp_slow(double p) { return 1.0 / p; }

__device__ __forceinline__ double frcp_any(double p) { return fp64_fast_range(p) ? frcp(p) : frcp_slow(p); }

// True when x is infinite or NaN (integer test of the exponent field).
__device__ __forceinline__ bool nonfinite(double x) { return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000; }

// Running product m 2^E for a sum of logarithms.
struct LogProd {
    double m;
    int e;
};

__device__ __forceinline__ void logprod_init(LogProd& s) {
    s.m = 1.0;
    s.e = 0;
}

// s *= p for p in the fast range (fp64_fast_range): m in [1, 2) times p
// stays normal and finite, and its exponent moves into e.
__device__ __forceinline__ void logprod_mul(LogProd& s, double p) {
    const double t = s.m * p;
    const int hi = __double2hiint(t);
    const int ex = (hi >> 20) - 1023;
    s.e += ex;
    s.m = __hiloint2double(hi - ex * (1 << 20), __double2loint(t));
}

// log of the running product: E ln2 + log m.
__device__ __forceinline__ double logprod_log(const LogProd& s, const Fp64Tab& tab) {
    const double ed = (double)s.e;
    return fma(ed, kLn2Hi, fma(ed, kLn2Lo, flog_fast(s.m, tab)));
}

}  // namespace cg
