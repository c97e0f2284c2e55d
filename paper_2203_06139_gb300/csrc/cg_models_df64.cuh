// cg_models_df64.cuh -- double-float (FP32-pipe) forward + adjoint of the 1-D
// Gaussian-peaks + polynomial model (same accumulators as gp1_elem_fp64 in
// cg_models.cuh, whose epilogue they feed).
#pragma once
#include "cg_df64.cuh"
#include "cg_models.cuh"

namespace cg {

struct GP1Df {
    df A[CG_MAX_PEAKS_1D], mu[CG_MAX_PEAKS_1D], c[CG_MAX_PEAKS_1D];
    df poly[4];
    df lo, h, au, bu;
};

__device__ __forceinline__ void gp1_split(const GP1Consts& c64, double lo, double h, double au, double bu, int K,
                                          GP1Df& c) {
    for (int k = 0; k < K; ++k) {
        c.A[k] = df_from_double(c64.A[k]);
        c.mu[k] = df_from_double(c64.mu[k]);
        c.c[k] = df_from_double(c64.c[k]);
    }
    for (int j = 0; j < 4; ++j) c.poly[j] = df_from_double(c64.poly[j]);
    c.lo = df_from_double(lo);
    c.h = df_from_double(h);
    c.au = df_from_double(au);
    c.bu = df_from_double(bu);
}

// Per-point constants of the 1-D model computed by the 32 lanes of one warp,
// one constant per lane (the FP64 division and the double splits run side by
// side instead of in one thread): FP64 values into c64 and, with SPLIT, their
// df64 splits into cd.  Returns, on every lane, whether the point is valid
// (finite parameters, nonzero widths).  Call from a whole warp; the caller
// synchronises before the constants are read.
template <int K, bool SPLIT>
__device__ __forceinline__ bool gp1_prologue_warp(const double* __restrict__ th, int D, double lo, double h,
                                                  double au, double bu, GP1Consts& c64, GP1Df& cd) {
    static_assert(3 * K + 8 <= 32, "one constant per lane");
    const int lane = threadIdx.x & 31;
    bool ok = true;
    double v = 0.0;
    df* dst = nullptr;
    if (lane < 3 * K) {
        const int k = lane / 3, r = lane - 3 * k;
        const double x = th[lane];
        ok = isfinite(x);
        if (r == 0) {
            v = x;
            c64.A[k] = v;
            dst = &cd.A[k];
        } else if (r == 1) {
            v = x;
            c64.mu[k] = v;
            dst = &cd.mu[k];
        } else {
            v = -0.5 / (x * x);
            ok = ok && x != 0.0;
            c64.c[k] = v;
            dst = &cd.c[k];
        }
    } else if (lane < 3 * K + 4) {
        const int j = lane - 3 * K;
        v = (j <= D) ? th[lane] : 0.0;
        ok = isfinite(v);
        c64.poly[j] = v;
        dst = &cd.poly[j];
    } else if (lane < 3 * K + 8) {
        const int j = lane - 3 * K - 4;
        v = (j == 0) ? lo : (j == 1) ? h : (j == 2) ? au : bu;
        dst = (j == 0) ? &cd.lo : (j == 1) ? &cd.h : (j == 2) ? &cd.au : &cd.bu;
    }
    if (SPLIT && dst) *dst = df_from_double(v);
    return __all_sync(0xffffffffu, ok);
}

// One bin in FP64, out of line (the rare fallback of the df64 bin loops):
// its accumulator terms into out[0..N), *bad set on a domain error.
template <int K, int OBJ>
static __device__ __noinline__ void gp1_elem_fp64_ool(double x, double y, const GP1Consts& cs, GP1Data dd,
                                                      double* out, int* bad) {
    constexpr int N = GP1Acc<K>::N;
    double a[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = 0.0;
    bool b = false;
    gp1_elem_fp64<K, OBJ>(x, y, cs, dd, a, b);
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = a[i];
    *bad = b ? 1 : 0;
}

// Bin centre lo + (i + 0.5) h in df64 (i < 2^24).
__device__ __forceinline__ df gp1_centre_df(const GP1Df& c, float fi) {
    const df t = two_sum(fi, 0.5f);
    return df_add(c.lo, df_mul(c.h, t));
}
__device__ __forceinline__ df gp1_centre_df(const GP1Df& c, int64_t i) { return gp1_centre_df(c, (float)i); }

// One bin at centre X (df64) with count y.  Returns false when the element
// must be recomputed in FP64 (every Gaussian flushed while the model value is
// tiny, or a non-positive model value under a log).
// VO (value only): accumulate T and skip the adjoint part.
// GN: also accumulate the Gauss-Newton diagonal terms h (df/dtheta)^2, with
// h = d2T/df2, into gacc (same slots as the gradient accumulators; slot 0 is
// unused) -- the terms the fitter's initial inverse Hessian is built from.
// GNM: also the Gauss-Newton matrix terms h r_a r_b (a <= b), in FP32, into
// gm (packed upper triangle of the R = 3K + 4 raw Jacobian factors r =
// (e_1, e_1 d_1, e_1 d_1^2, ..., u^0 .. u^3), entries past the degree zero):
// d f/d theta_a = D_a r_a with the per-point scales D applied once after the
// sums (1, A/s^2, A/s^3 per peak, 1 per polynomial term).  Empty bins of the
// Poisson forms add nothing (h = 0).
template <int K>
struct GP1Gnm {
    static constexpr int R = 3 * K + 4;
    static constexpr int NV = R * (R + 1) / 2;
};

template <int K, int OBJ, bool VO = false, bool GN = false, bool GNM = false>
__device__ __forceinline__ bool gp1_elem_df64(df X, double yd, const GP1Df& c, int D, int pm,
                                              DfAcc (&acc)[GP1Acc<K>::N], const DfTables& tab,
                                              DfAcc* gacc = nullptr, float* gm = nullptr) {
    const df u = pm ? df_add(df_mul(X, c.au), c.bu) : X;
    df f = df_make(0.0f, 0.0f);
#pragma unroll
    for (int j = 3; j >= 0; --j) {   // Horner from the leading coefficient
        if (j == D) f = c.poly[j];
        else if (j < D) f = df_add(df_mul(f, u), c.poly[j]);
    }
    df dk[K > 0 ? K : 1], ek[K > 0 ? K : 1];
    bool fl = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dk[k] = df_sub(X, c.mu[k]);
        bool f1 = false;
        ek[k] = df_exp(df_mul(c.c[k], df_sqr(dk[k])), tab, f1);
        fl |= f1;
        f = df_add(f, df_mul_nn(c.A[k], ek[k]));
    }
    const df y = df_split(yd);
    df T, g, hh;
    float gsc = 1.0f;   // GNM: the factors r are taken as r / f for the Poisson forms
    if (OBJ == CG_OBJ_CHI2) {
        const df w = df_rcp(df_make(fmaxf(y.h, 1.0f), y.h >= 1.0f ? y.l : 0.0f));
        const df r = df_sub(y, f);
        const df wr = df_mul(w, r);
        T = df_mul(wr, r);
        g = df_make(-2.0f * wr.h, -2.0f * wr.l);
        if (GN || GNM) hh = df_make(2.0f * w.h, 2.0f * w.l);
    } else {
        if (!(f.h > 1e-30f) || (fl && f.h < 1e-13f)) return false;
        const df rf = df_rcp(f);
        const df yr = df_mul(y, rf);
        if (GNM) gsc = rf.h;
        if (OBJ == CG_OBJ_POISSON) {
            T = (y.h > 0.0f) ? df_sub(f, df_mul(y, df_log(f, tab))) : f;
            g = df_sub(df_make(1.0f, 0.0f), yr);
            if (GN) hh = df_mul(yr, rf);
        } else {
            T = (y.h > 0.0f) ? df_add(df_sub(f, y), df_mul(y, df_log(yr, tab))) : f;
            T = df_make(2.0f * T.h, 2.0f * T.l);
            const df gg = df_sub(df_make(1.0f, 0.0f), yr);
            g = df_make(2.0f * gg.h, 2.0f * gg.l);
            if (GN) {
                hh = df_mul(yr, rf);
                hh = df_make(2.0f * hh.h, 2.0f * hh.l);
            }
        }
    }
    dfacc_add(acc[0], T);
    if (VO) return true;
    if (GNM) {
        constexpr int R = GP1Gnm<K>::R;
        float r[R];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float e = ek[k].h * gsc, ed = e * dk[k].h;
            r[3 * k] = e;
            r[3 * k + 1] = ed;
            r[3 * k + 2] = ed * dk[k].h;
        }
        float up = gsc;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            r[3 * K + j] = (j <= D) ? up : 0.0f;
            up *= u.h;
        }
        // h r_a r_b = 2w r_a r_b (chi2), y (r_a/f)(r_b/f) (Poisson), twice that (Baker-Cousins):
        // no y/f^2 in FP32, whose range it can leave where a peak has no background under it
        const float hf = (OBJ == CG_OBJ_CHI2) ? hh.h : (OBJ == CG_OBJ_POISSON ? y.h : 2.0f * y.h);
        int q = 0;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const float ha = hf * r[a];
#pragma unroll
            for (int b = a; b < R; ++b) {
                gm[q] = fmaf(ha, r[b], gm[q]);
                ++q;
            }
        }
    }
    if (GN) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const df he = df_mul_nn(hh, df_sqr(ek[k]));
            const df d2 = df_sqr(dk[k]);
            const df hd2 = df_mul_nn(he, d2);
            dfacc_add(gacc[1 + 3 * k], he);
            dfacc_add(gacc[2 + 3 * k], hd2);
            dfacc_add(gacc[3 + 3 * k], df_mul_nn(hd2, d2));
        }
        if (D >= 0) dfacc_add(gacc[1 + 3 * K], hh);
        if (D >= 1) {
            const df u2 = df_sqr(u);
            dfacc_add(gacc[2 + 3 * K], df_mul_nn(hh, u2));
            if (D >= 2) {
                const df u4 = df_sqr(u2);
                dfacc_add(gacc[3 + 3 * K], df_mul_nn(hh, u4));
                if (D >= 3) dfacc_add(gacc[4 + 3 * K], df_mul_nn(hh, df_mul(u4, u2)));
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const df t = df_mul_nn(g, ek[k]);
        const df td = df_mul_nn(t, dk[k]);
        dfacc_add(acc[1 + 3 * k], t);
        dfacc_add(acc[2 + 3 * k], td);
        dfacc_add(acc[3 + 3 * k], df_mul_nn(td, dk[k]));
    }
    // polynomial adjoints g u^j, powers only up to the degree
    if (D >= 0) dfacc_add(acc[1 + 3 * K], g);
    if (D >= 1) {
        dfacc_add(acc[2 + 3 * K], df_mul_nn(g, u));
        if (D >= 2) {
            const df u2 = df_sqr(u);
            dfacc_add(acc[3 + 3 * K], df_mul_nn(g, u2));
            if (D >= 3) dfacc_add(acc[4 + 3 * K], df_mul_nn(g, df_mul(u2, u)));
        }
    }
    return true;
}

}  // namespace cg
