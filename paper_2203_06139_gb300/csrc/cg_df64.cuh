// cg_df64.cuh -- double-float ("df64") arithmetic on the FP32 pipe.
//
// A df64 value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significand bits.  GB300's FP64 unit issues 2
// DFMA per clock per SM against 128 FFMA for FP32, so the per-element work
// of the fused kernels runs here on the FP32 pipe with these error-free
// transformations, while accumulation stays in FP64.
//
// Published methods used (own implementations):
//  - TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker 1971),
//    TwoProduct with a fused multiply-add;
//  - exp: table-driven method of P. T. P. Tang, "Table-driven implementation
//    of the exponential function in IEEE floating-point arithmetic", ACM
//    TOMS 15(2), 1989: q = (64 N + j) ln2/64 + r, exp(q) = 2^N 2^(j/64) e^r,
//    |r| <= ln2/128, e^r from its Taylor series;
//  - log: table-driven method of P. T. P. Tang, "Table-driven implementation
//    of the logarithm function in IEEE floating-point arithmetic", ACM TOMS
//    16(4), 1990: p = 2^E m, F = 1 + (2j+1)/128 nearest m, log p = E ln2 +
//    log F + log1p((m - F)/F), log1p from its Taylor series;
//  - reciprocal: one Newton step in df64 from a float estimate.
// The tables (2^(j/64), log F, 1/F) are generated offline as float pairs
// from 60-digit mpmath values (gen_df64_tables.py, cg_df64_tables.inc) and
// copied into shared memory at block start by df_tables_init.
//
// Every float operation below is written with explicit round-to-nearest
// intrinsics (or fmaf) so the compiler cannot contract or reorder the
// error-free transformations.
#pragma once
#include <math.h>
#include <stdint.h>

namespace cg {

struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(float h, float l) { df r; r.h = h; r.l = l; return r; }

__device__ __forceinline__ df df_from_double(double x) {
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(x - (double)h);
    return df_make(h, l);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

// Split a double into a float pair with integer operations only (no FP64
// instruction): hi = the leading 24 significand bits, lo = the next 29 bits
// rounded to 23; |x - (hi + lo)| <= 2^-47 |x|.  Doubles with exponents
// outside [-80, 127] go through the conversion instructions instead.
static __device__ __noinline__ df df_from_double_slow(double x) { return df_from_double(x); }

__device__ __forceinline__ df df_split(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
    // rare: a call is never if-converted, so its conversions stay off the common path
    if (e < -80 || e > 127) return df_from_double_slow(x);
    const unsigned sign = hw & 0x80000000u;
    const float h = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    // remaining 29 bits r of the significand; value r 2^(e-52)
    const unsigned rt = ((lw & 0x1fffffffu) + 32u) >> 6;                  // 23 bits, rounded (may reach 2^23)
    float l = __fsub_rn(__uint_as_float(0x4b000000u | rt), 8388608.0f);   // exact float(rt)
    if (rt == 0x800000u) l = 8388608.0f;
    l = __fmul_rn(l, __uint_as_float((unsigned)(e + 81) << 23));          // * 2^(e - 46)
    return df_make(h, __uint_as_float(__float_as_uint(l) | sign));
}

// Products whose result only feeds an accumulator or another product do not
// need the final renormalisation: hi + lo is still the rounded product.
__device__ __forceinline__ df df_mul_nn(df a, df b);

// s + e = a + b exactly
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df_make(s, e);
}

// s + e = a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return df_make(s, e);
}

// p + e = a * b exactly
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    return df_make(p, e);
}

__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.h, b.h);
    const float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return fast_two_sum(s.h, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_make(-b.h, -b.l)); }

__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.h, b);
    return fast_two_sum(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.h, b.h);
    float e = fmaf(a.h, b.l, p.l);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p.h, e);
}

__device__ __forceinline__ df df_mul_nn(df a, df b) {
    df p = two_prod(a.h, b.h);
    float e = fmaf(a.h, b.l, p.l);
    return df_make(p.h, fmaf(a.l, b.h, e));
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.h, b);
    return fast_two_sum(p.h, fmaf(a.l, b, p.l));
}

__device__ __forceinline__ df df_sqr(df a) {
    df p = two_prod(a.h, a.h);
    const float e = fmaf(__fadd_rn(a.h, a.h), a.l, p.l);
    return fast_two_sum(p.h, e);
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/a: float estimate refined by one FP32 Newton step, then one df64 Newton step.
__device__ __forceinline__ df df_rcp(df a) {
    float r = rcp_approx(a.h);
    r = fmaf(r, fmaf(-a.h, r, 1.0f), r);
    // residual 1 - a r, exact for the hi part by the fused multiply-add
    float e = fmaf(-a.h, r, 1.0f);
    e = fmaf(-a.l, r, e);
    return fast_two_sum(r, __fmul_rn(r, e));
}

// ---------------------------------------------------------------------------
// Tables, built per block in shared memory.
// ---------------------------------------------------------------------------
struct DfTables {
    float2 exp2j[64];   // 2^(j/64), j = 0..63
    float2 logF[64];    // log(F_j), F_j = 1 + (2j + 1)/128
    float2 invF[64];    // 1/F_j
};

#include "cg_df64_tables.inc"

// Copy the tables (generated, exactly rounded float pairs) into shared memory.
// Call from all threads of a block, followed by __syncthreads().
__device__ __forceinline__ void df_tables_init(DfTables& t) {
    for (int j = threadIdx.x; j < 64; j += blockDim.x) {
        t.exp2j[j] = g_df_exp2j[j];
        t.logF[j] = g_df_logF[j];
        t.invF[j] = g_df_invF[j];
    }
}

// ln2/64 split into three floats; the first has 11 significant bits so that
// k * C1 is exact for |k| < 2^13.
#define CG_LN2_64_C1 1.0833740234375e-02f
#define CG_LN2_64_C2 (-3.3155381516e-06f)
#define CG_LN2_64_C3 2.5728046e-14f
#define CG_INV_LN2_64 92.33248261689366f
// ln 2 split: 16 significant bits, then two floats
#define CG_LN2_H 0.693145751953125f
#define CG_LN2_M 1.4286067653e-06f
#define CG_LN2_L 5.4979230187e-14f

// exp(q) for df64 q.  Results below exp(-69) (about 1e-30) are returned as 0
// with *flushed set; q above 88 returns +inf.
__device__ __forceinline__ df df_exp(df q, const DfTables& tab, bool& flushed) {
    if (q.h < -69.0f) {
        flushed = true;
        return df_make(0.0f, 0.0f);
    }
    if (q.h > 88.0f) return df_make(__int_as_float(0x7f800000), 0.0f);
    const int k = __float2int_rn(__fmul_rn(q.h, CG_INV_LN2_64));
    const float kf = (float)k;
    // r = q - k ln2/64 in df64 (the first step is exact)
    const float a = fmaf(-kf, CG_LN2_64_C1, q.h);
    df s = two_sum(a, q.l);
    df p2 = two_prod(kf, CG_LN2_64_C2);
    df s2 = two_sum(s.h, -p2.h);
    float lo = __fadd_rn(__fsub_rn(__fadd_rn(s.l, s2.l), p2.l), __fmul_rn(-kf, CG_LN2_64_C3));
    const df r = fast_two_sum(s2.h, lo);
    // e^r - 1 = r + r^2/2 + r^3 (1/6 + r/24 + r^2/120 + r^3/720) (+ O(r^7))
    const float rh = r.h;
    float tail = fmaf(rh, 1.0f / 720.0f, 1.0f / 120.0f);
    tail = fmaf(rh, tail, 1.0f / 24.0f);
    tail = fmaf(rh, tail, 1.0f / 6.0f);
    tail = __fmul_rn(__fmul_rn(__fmul_rn(rh, rh), rh), tail);
    df sq = two_prod(rh, rh);
    df u = fast_two_sum(rh, __fmul_rn(0.5f, sq.h));   // exact: |r| > r^2/2 for |r| < ln2/128
    lo = __fadd_rn(__fadd_rn(u.l, r.l), __fadd_rn(fmaf(0.5f, sq.l, __fmul_rn(rh, r.l)), tail));
    const df em1 = fast_two_sum(u.h, lo);
    // 2^(j/64) (1 + em1)
    const float2 T = tab.exp2j[k & 63];
    df pm = two_prod(T.x, em1.h);
    float plo = fmaf(T.x, em1.l, fmaf(T.y, em1.h, pm.l));
    df sum = fast_two_sum(T.x, pm.h);
    const df R = fast_two_sum(sum.h, __fadd_rn(__fadd_rn(sum.l, T.y), plo));
    // scale by 2^N, N = floor(k / 64) in [-101, 127]
    const float sc = __int_as_float(((k >> 6) + 127) << 23);
    return df_make(__fmul_rn(R.h, sc), __fmul_rn(R.l, sc));
}

// log(p) for df64 p > 0 (normal hi part).
__device__ __forceinline__ df df_log(df p, const DfTables& tab) {
    const int bits = __float_as_int(p.h);
    const int E = ((bits >> 23) & 0xff) - 127;
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);   // [1, 2)
    const int j = (bits >> 17) & 63;
    const float F = __fadd_rn(1.0f, __fmul_rn((float)(2 * j + 1), 1.0f / 128.0f));
    const float v = __fsub_rn(m, F);                                     // exact
    const float2 iv = tab.invF[j];
    df u = two_prod(v, iv.x);
    u = fast_two_sum(u.h, fmaf(v, iv.y, u.l));                           // (m - F)/F
    // lo part of p: log(p.h + p.l) = log(p.h) + p.l/p.h + O(2^-48)
    const float corr = __fmul_rn(p.l, rcp_approx(p.h));
    // log1p(u) = u - u^2/2 + u^3 (1/3 - u/4 + u^2/5 - u^3/6 + u^4/7)
    const float uh = u.h;
    float tail = fmaf(uh, 1.0f / 7.0f, -1.0f / 6.0f);
    tail = fmaf(uh, tail, 1.0f / 5.0f);
    tail = fmaf(uh, tail, -0.25f);
    tail = fmaf(uh, tail, 1.0f / 3.0f);
    tail = __fmul_rn(__fmul_rn(__fmul_rn(uh, uh), uh), tail);
    df sq = two_prod(uh, uh);
    df w = two_sum(uh, __fmul_rn(-0.5f, sq.h));
    float lo = __fadd_rn(__fadd_rn(w.l, u.l), __fadd_rn(fmaf(-0.5f, sq.l, -__fmul_rn(uh, u.l)), tail));
    lo = __fadd_rn(lo, corr);
    // + E ln2 + log F
    const float Ef = (float)E;
    const float2 lf = tab.logF[j];
    df a = two_sum(__fmul_rn(Ef, CG_LN2_H), lf.x);                        // E * LN2_H is exact
    df b = two_prod(Ef, CG_LN2_M);
    df c = two_sum(a.h, w.h);
    float l2 = __fadd_rn(__fadd_rn(a.l, c.l),
                         __fadd_rn(__fadd_rn(b.h, fmaf(Ef, CG_LN2_L, b.l)), __fadd_rn(lf.y, lo)));
    return fast_two_sum(c.h, l2);
}

// Running product of positive df64 factors with its binary exponent kept
// apart (so a long product neither underflows nor overflows): value =
// (m.h + m.l) 2^E.  log of it = df_log(m) + E ln2.
struct DfProd {
    df m;
    int E;
};

__device__ __forceinline__ void dfprod_mul(DfProd& P, df x) {
    df r = df_mul(P.m, x);
    // move the binary exponent eb of r.h (r.h > 0, normal) into E: scale by 2^-eb exactly
    const int eb = (int)((__float_as_uint(r.h) >> 23) & 0xffu) - 127;
    const float sc = __uint_as_float((unsigned)(127 - eb) << 23);
    P.m.h = __fmul_rn(r.h, sc);
    P.m.l = __fmul_rn(r.l, sc);
    P.E += eb;
}

__device__ __forceinline__ df dfprod_log(const DfProd& P, const DfTables& tab) {
    df l = df_log(P.m, tab);
    const float Ef = (float)P.E;
    df a = two_sum(l.h, __fmul_rn(Ef, CG_LN2_H));
    df b = two_prod(Ef, CG_LN2_M);
    return fast_two_sum(a.h, __fadd_rn(__fadd_rn(a.l, l.l), __fadd_rn(b.h, fmaf(Ef, CG_LN2_L, b.l))));
}

// Compensated per-thread accumulator of df64 terms, flushed into an FP64 sum.
struct DfAcc {
    float s, c;
};

__device__ __forceinline__ void dfacc_add(DfAcc& A, df x) {
    df t = two_sum(A.s, x.h);
    A.s = t.h;
    A.c = __fadd_rn(A.c, __fadd_rn(t.l, x.l));
}

__device__ __forceinline__ void dfacc_flush(DfAcc& A, double& sum) {
    sum += (double)A.s + (double)A.c;
    A.s = 0.0f;
    A.c = 0.0f;
}

// Fold a compensated accumulator into a per-thread df64 running sum (FP32 pipe).
__device__ __forceinline__ void dfacc_fold(DfAcc& A, df& run) {
    run = df_add(run, df_make(A.s, A.c));
    A.s = A.c = 0.0f;
}

// Warp butterfly sum of df64 values on the FP32 pipe.  TwoSum is exact and
// symmetric, so both lanes of every exchange form the same sum and all lanes
// end with the same total.
__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, df_make(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)));
    return v;
}

// Warp sums of N df64 values per lane by a reduce-scatter butterfly (FP32
// pipe).  With NP = N rounded up to a power of two (at most 32), each of the
// first log2(NP) exchanges (lane distances 16, 8, ...) has every lane keep
// half of its values and add its partner's copy of that half, so the number
// of values moved halves at every step; the exchanges left are plain
// butterflies on the single value that remains.  Each total passes through
// five additions in a fixed order, as in a butterfly per value, at about a
// third of the operations for 6-8 values.  Accumulator a ends in the lanes
// whose top log2(NP) lane-id bits spell a; the first of them writes its FP64
// conversion to dst[a * stride].
template <int N>
__device__ __forceinline__ void warp_sum_df_to(const df (&v)[N], double* dst, int stride) {
    static_assert(N >= 1 && N <= 32, "at most one value per lane after the scatter");
    constexpr int L = (N <= 1) ? 0 : (N <= 2) ? 1 : (N <= 4) ? 2 : (N <= 8) ? 3 : (N <= 16) ? 4 : 5;
    constexpr int NP = 1 << L;
    const int lane = threadIdx.x & 31;
    df w[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) w[a] = (a < N) ? v[a] : df_make(0.0f, 0.0f);
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const int o = 16 >> l;
        const int H = (NP >> l) / 2;   // values kept after this exchange
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const df send = up ? w[j] : w[j + H];
            const df keep = up ? w[j + H] : w[j];
            const df recv = df_make(__shfl_xor_sync(0xffffffffu, send.h, o), __shfl_xor_sync(0xffffffffu, send.l, o));
            w[j] = df_add(keep, recv);
        }
    }
#pragma unroll
    for (int o = 16 >> L; o > 0; o >>= 1)
        w[0] = df_add(w[0], df_make(__shfl_xor_sync(0xffffffffu, w[0].h, o), __shfl_xor_sync(0xffffffffu, w[0].l, o)));
    const int a = lane >> (5 - L);
    if ((lane & ((1 << (5 - L)) - 1)) == 0 && a < N) dst[a * stride] = df_to_double(w[0]);
}

// Block sum of NACC per-thread df64 values in a fixed order: warp
// reduce-scatter sums in df64, one conversion to FP64 per warp and
// accumulator, then thread a adds accumulator a over the warps in warp order.
// red: shared, NACC * (NT/32) doubles; out: shared, NACC doubles, valid in
// all threads on return.
template <int NACC, int NT>
__device__ __forceinline__ void block_sum_df(const df (&v)[NACC], double* red, double* out) {
    static_assert(NACC <= NT, "one thread per accumulator in the last step");
    constexpr int NW = NT / 32;
    const int wid = threadIdx.x >> 5;
    warp_sum_df_to<NACC>(v, red + wid, NW);
    __syncthreads();
    if (threadIdx.x < NACC) {
        double s = 0.0;
        for (int w = 0; w < NW; ++w) s += red[threadIdx.x * NW + w];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

}  // namespace cg
