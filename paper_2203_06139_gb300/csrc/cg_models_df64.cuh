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
template <int K, int OBJ, bool VO = false, bool GN = false>
__device__ __forceinline__ bool gp1_elem_df64(df X, double yd, const GP1Df& c, int D, int pm,
                                              DfAcc (&acc)[GP1Acc<K>::N], const DfTables& tab,
                                              DfAcc* gacc = nullptr) {
    const df u = pm ? df_add(df_mul(X, c.au), c.bu) : X;
    df f = df_make(0.0f, 0.0f);
#pragma unroll
    for (int j = 3; j >= 0; --j)
        if (j <= D) f = df_add(df_mul(f, u), c.poly[j]);
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
    if (OBJ == CG_OBJ_CHI2) {
        const df w = df_rcp(df_make(fmaxf(y.h, 1.0f), y.h >= 1.0f ? y.l : 0.0f));
        const df r = df_sub(y, f);
        const df wr = df_mul(w, r);
        T = df_mul(wr, r);
        g = df_make(-2.0f * wr.h, -2.0f * wr.l);
        if (GN) hh = df_make(2.0f * w.h, 2.0f * w.l);
    } else {
        if (!(f.h > 1e-30f) || (fl && f.h < 1e-13f)) return false;
        const df rf = df_rcp(f);
        const df yr = df_mul(y, rf);
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
        const df u2 = df_sqr(u);
        df up2 = df_make(1.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j <= D) dfacc_add(gacc[1 + 3 * K + j], df_mul_nn(hh, up2));
            if (j < 3) up2 = df_mul(up2, u2);
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
    df up = df_make(1.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j <= D) dfacc_add(acc[1 + 3 * K + j], df_mul_nn(g, up));
        if (j < 3) up = df_mul(up, u);
    }
    return true;
}

}  // namespace cg
