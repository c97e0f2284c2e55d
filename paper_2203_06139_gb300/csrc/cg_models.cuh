// cg_models.cuh -- per-model prologue, fused per-element forward + adjoint
// (FP64), and epilogue of libcg.
//
// Each model is written as reverse-mode AD by hand (Sec. 1-2 of the paper):
// the forward value of one bin/event term T_i, then the adjoint
// dT_i/df_i, then its propagation into a fixed set of accumulators.  The
// accumulators are the adjoints of theta-only quantities (the prologue
// constants); the epilogue chains them to theta once per parameter point.
#pragma once
#include <math.h>
#include <stdint.h>

#include "cg_internal.cuh"

namespace cg {

constexpr int kMaxAcc = 50;      // 2 + 6 * CG_MAX_PEAKS_2D
constexpr int kMaxParams = CG_MAX_PARAMS;

struct TileGrid {
    int64_t n_elem;   // elements per parameter point
    int64_t chunk;    // elements per tile (even; a multiple of 2 * threads for the df64 kernels)
    int nbx;          // tiles per parameter point
    int n_theta;      // parameter points (groups of pt points for multi-point kernels)
    int n_tiles;      // n_theta * nbx
    const int* gate = nullptr;   // when set, every kernel of the launch returns at once while *gate == 0
    int pt = 1;       // parameter points per tile
    int n_pts = 0;    // multi-point kernels: the number of points (n_theta is then the number of groups)
};

__device__ __forceinline__ bool gated_off(const TileGrid& tg) {
    return tg.gate != nullptr && *(volatile const int*)tg.gate == 0;
}

struct EpiParams {
    int model, P, K, D;
    double lo, hi;
};

// ===========================================================================
// 1-D binned: K Gaussian peaks + polynomial of degree D (runtime, <= 3)
//   f(x) = sum_k A_k exp(c_k (x - mu_k)^2) + sum_j p_j u^j,  c_k = -1/(2 s_k^2)
// accumulators: [ T | (g e_k, g e_k d_k, g e_k d_k^2) for k | g u^j for j<4 ]
// where g = dT/df and d_k = x - mu_k.
// ===========================================================================
template <int K>
struct GP1Acc { static constexpr int N = 1 + 3 * K + 4; };

struct GP1Consts {
    double A[CG_MAX_PEAKS_1D], mu[CG_MAX_PEAKS_1D], c[CG_MAX_PEAKS_1D];
    double poly[4];
};

struct GP1Data {
    const double* y;        // counts
    const double* centres;  // optional explicit centres
    double lo, h;           // uniform centres lo + (i + 0.5) h
    double au, bu;          // t = au x + bu
    int D, pm;
    int vec_ok;             // 16-byte aligned: pairs of bins per 16-byte load
};

template <int K>
__device__ __forceinline__ bool gp1_prologue(const double* __restrict__ th, int D, GP1Consts& cs) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double A = th[3 * k], mu = th[3 * k + 1], s = th[3 * k + 2];
        cs.A[k] = A;
        cs.mu[k] = mu;
        cs.c[k] = -0.5 / (s * s);
        ok = ok && isfinite(A) && isfinite(mu) && isfinite(s) && s != 0.0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double p = (j <= D) ? th[3 * K + j] : 0.0;
        cs.poly[j] = p;
        ok = ok && isfinite(p);
    }
    return ok;
}

template <int K, int OBJ>
__device__ __forceinline__ void gp1_elem_fp64(double x, double y, const GP1Consts& cs, const GP1Data& d,
                                              double (&acc)[GP1Acc<K>::N], bool& bad) {
    const double u = d.pm ? fma(x, d.au, d.bu) : x;
    // forward: polynomial by Horner, then the peaks
    double f = 0.0;
#pragma unroll
    for (int j = 3; j >= 0; --j) {   // Horner from the leading coefficient
        if (j == d.D) f = cs.poly[j];
        else if (j < d.D) f = fma(f, u, cs.poly[j]);
    }
    double dk[K > 0 ? K : 1], ek[K > 0 ? K : 1];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dk[k] = x - cs.mu[k];
        ek[k] = exp(cs.c[k] * dk[k] * dk[k]);
        f = fma(cs.A[k], ek[k], f);
    }
    // objective term and its adjoint g = dT/df
    double T, g;
    if (OBJ == CG_OBJ_CHI2) {
        const double w = 1.0 / fmax(y, 1.0);
        const double r = y - f;
        T = w * r * r;
        g = -2.0 * w * r;
    } else if (OBJ == CG_OBJ_POISSON) {
        const double rf = 1.0 / f;
        T = (y > 0.0) ? f - y * log(f) : f;
        g = (y > 0.0) ? 1.0 - y * rf : 1.0;   // empty bin: T = f, even where f underflows to 0
        bad |= (y > 0.0) && !(f > 0.0);
    } else {  // Baker-Cousins
        const double rf = 1.0 / f;
        T = (y > 0.0) ? 2.0 * (f - y + y * log(y * rf)) : 2.0 * f;
        g = (y > 0.0) ? 2.0 * (1.0 - y * rf) : 2.0;
        bad |= (y > 0.0) && !(f > 0.0);
    }
    bad |= !isfinite(T);
    // adjoint propagation into the accumulators
    acc[0] += T;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double t = g * ek[k];
        const double td = t * dk[k];
        acc[1 + 3 * k] += t;
        acc[2 + 3 * k] += td;
        acc[3 + 3 * k] = fma(td, dk[k], acc[3 + 3 * k]);
    }
    double up = 1.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j <= d.D) acc[1 + 3 * K + j] = fma(g, up, acc[1 + 3 * K + j]);
        if (j < d.D) up *= u;
    }
}

// ===========================================================================
// Unbinned mixture on [lo, hi]: theta = (frac, mu, s, lambda)
//   p(x) = a exp(c (x-mu)^2) + b exp(-lambda (x - lo)),
//   a = frac / (s sqrt(2 pi) Z_G), Z_G = Phi((hi-mu)/s) - Phi((lo-mu)/s),
//   b = (1 - frac) lambda / Z_E,    Z_E = 1 - exp(-lambda (hi - lo)),
//   c = -1/(2 s^2);  T = -w log p.
// accumulators: [ w log p | U | U d | U d^2 | V | V xl ],
//   U = w eG / p, V = w eE / p, d = x - mu, xl = x - lo.
// ===========================================================================
struct MixAcc { static constexpr int N = 6; };

struct MixConsts {
    double mu, c, a, b, lam, lo;
};

struct MixData {
    const double* x;
    const double* w;
    double lo, hi;
    int vec_ok;
    const float2* xs;   // df64 kernels: events split once per call into (hi, lo) float pairs
    const float2* wsp;  // weights split likewise (or nullptr)
    // FP64 kernel: per chunk of the tile grid, sum (x - lo) in [0, nbx), and with
    // weights sum w in [nbx, 2 nbx) and sum w (x - lo) in [2 nbx, 3 nbx)
    const double* csum = nullptr;
};

__device__ __forceinline__ double std_normal_cdf(double z) { return 0.5 * erfc(-z * 0.70710678118654752440); }
__device__ __forceinline__ double std_normal_pdf(double z) { return 0.39894228040143267794 * exp(-0.5 * z * z); }

__device__ __forceinline__ bool mix_prologue(const double* __restrict__ th, double lo, double hi, MixConsts& cs) {
    const double f = th[0], mu = th[1], s = th[2], lam = th[3];
    const double zg = std_normal_cdf((hi - mu) / s) - std_normal_cdf((lo - mu) / s);
    const double ze = -expm1(-lam * (hi - lo));
    cs.mu = mu;
    cs.c = -0.5 / (s * s);
    cs.a = f / (s * 2.50662827463100050242 * zg);
    cs.b = (1.0 - f) * lam / ze;
    cs.lam = lam;
    cs.lo = lo;
    return isfinite(f) && isfinite(mu) && isfinite(s) && isfinite(lam) && s != 0.0 && s * zg > 0.0 &&
           ze > 0.0 && isfinite(cs.a) && isfinite(cs.b);
}

template <bool W>
__device__ __forceinline__ void mix_elem_fp64(double x, double w, const MixConsts& cs, double (&acc)[MixAcc::N],
                                              bool& bad) {
    const double d = x - cs.mu;
    const double eG = exp(cs.c * d * d);
    const double xl = x - cs.lo;
    const double eE = exp(-cs.lam * xl);
    const double p = fma(cs.a, eG, cs.b * eE);
    double r = 1.0 / p;
    double L = log(p);
    bad |= !(p > 0.0);
    if (W) {
        r *= w;
        L *= w;
    }
    const double U = eG * r, V = eE * r;
    const double Ud = U * d;
    acc[0] += L;
    acc[1] += U;
    acc[2] += Ud;
    acc[3] = fma(Ud, d, acc[3]);
    acc[4] += V;
    acc[5] = fma(V, xl, acc[5]);
}

// ===========================================================================
// 2-D binned Poisson NLL: K rotated Gaussians + constant C.
//   u = cos(phi) dx + sin(phi) dy,  v = -sin(phi) dx + cos(phi) dy,
//   q = al u^2 + be v^2 (al = -1/(2 sx^2), be = -1/(2 sy^2)),
//   mu = C + sum_k A_k e^q,  T = mu - n log mu,  g = 1 - n/mu.
// accumulators: [ T | (S, Su, Sv, Suu, Svv, Suv) for k | sum g ],
//   S* = sum g e_k * (1, u, v, u^2, v^2, u v).
// ===========================================================================
template <int K>
struct RG2Acc { static constexpr int N = 2 + 6 * K; };

struct RG2Consts {
    double A[CG_MAX_PEAKS_2D], mx[CG_MAX_PEAKS_2D], my[CG_MAX_PEAKS_2D];
    double cs[CG_MAX_PEAKS_2D], sn[CG_MAX_PEAKS_2D], al[CG_MAX_PEAKS_2D], be[CG_MAX_PEAKS_2D];
    double C;
};

struct RG2Data {
    const double* n;   // counts [ny][nx]
    int64_t nx, ny;
    double lx, ly, hx, hy;
};

// Constants of Gaussian k from its six parameters t; false when one is not
// finite or a width is 0.
__device__ __forceinline__ bool rg2_prologue_one(const double* __restrict__ t, int k, RG2Consts& c) {
    c.A[k] = t[0];
    c.mx[k] = t[1];
    c.my[k] = t[2];
    c.al[k] = -0.5 / (t[3] * t[3]);
    c.be[k] = -0.5 / (t[4] * t[4]);
    sincos(t[5], &c.sn[k], &c.cs[k]);
    bool ok = t[3] != 0.0 && t[4] != 0.0;
    for (int j = 0; j < 6; ++j) ok = ok && isfinite(t[j]);
    return ok;
}

template <int K>
__device__ __forceinline__ bool rg2_prologue(const double* __restrict__ th, RG2Consts& c) {
    bool ok = true;
#pragma unroll
    for (int k = 0; k < K; ++k) ok = rg2_prologue_one(th + 6 * k, k, c) && ok;
    c.C = th[6 * K];
    return ok && isfinite(c.C);
}

// act: bit k set when Gaussian k can contribute in this tile (uniform per block)
template <int K>
__device__ __forceinline__ void rg2_elem_fp64(double x, double y, double n, const RG2Consts& c, unsigned act,
                                              double (&acc)[RG2Acc<K>::N], bool& bad) {
    double u[K], v[K], e[K];
    double mu = c.C;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!(act & (1u << k))) {
            u[k] = v[k] = e[k] = 0.0;
            continue;
        }
        const double dx = x - c.mx[k], dy = y - c.my[k];
        u[k] = fma(c.cs[k], dx, c.sn[k] * dy);
        v[k] = fma(c.cs[k], dy, -c.sn[k] * dx);
        e[k] = exp(fma(c.al[k], u[k] * u[k], c.be[k] * v[k] * v[k]));
        mu = fma(c.A[k], e[k], mu);
    }
    const double rm = 1.0 / mu;
    const double T = (n > 0.0) ? mu - n * log(mu) : mu;
    const double g = (n > 0.0) ? 1.0 - n * rm : 1.0;
    bad |= ((n > 0.0) && !(mu > 0.0)) || !isfinite(T);
    acc[0] += T;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (!(act & (1u << k))) continue;
        const double w = g * e[k];
        const double wu = w * u[k], wv = w * v[k];
        acc[1 + 6 * k] += w;
        acc[2 + 6 * k] += wu;
        acc[3 + 6 * k] += wv;
        acc[4 + 6 * k] = fma(wu, u[k], acc[4 + 6 * k]);
        acc[5 + 6 * k] = fma(wv, v[k], acc[5 + 6 * k]);
        acc[6 + 6 * k] = fma(wu, v[k], acc[6 + 6 * k]);
    }
    acc[1 + 6 * K] += g;
}

// ===========================================================================
// Epilogue: value and gradient from the summed accumulators S.
// ===========================================================================
__device__ inline double epilogue(const EpiParams& ep, const double* __restrict__ th, const double* S, double* g) {
    if (ep.model == CG_MODEL_GAUSS_POLY) {
        const int K = ep.K;
        for (int k = 0; k < K; ++k) {
            const double A = th[3 * k], s = th[3 * k + 2];
            g[3 * k] = S[1 + 3 * k];
            g[3 * k + 1] = A / (s * s) * S[2 + 3 * k];        // df/dmu = A e d / s^2
            g[3 * k + 2] = A / (s * s * s) * S[3 + 3 * k];    // df/ds  = A e d^2 / s^3
        }
        for (int j = 0; j <= ep.D; ++j) g[3 * K + j] = S[1 + 3 * K + j];
        return S[0];
    }
    if (ep.model == CG_MODEL_MIX_GAUSS_EXP) {
        const double f = th[0], mu = th[1], s = th[2], lam = th[3];
        const double lo = ep.lo, hi = ep.hi, L = hi - lo;
        const double al = (lo - mu) / s, be = (hi - mu) / s;
        const double zg = std_normal_cdf(be) - std_normal_cdf(al);
        const double ze = -expm1(-lam * L);
        const double sq = s * 2.50662827463100050242;
        const double a = f / (sq * zg), b = (1.0 - f) * lam / ze;
        const double Ga = -S[1], Gb = -S[4];              // dNLL/da, dNLL/db at fixed shapes
        const double pa = std_normal_pdf(al), pb = std_normal_pdf(be);
        const double dzg_dmu = (pa - pb) / s;
        const double dzg_ds = (al * pa - be * pb) / s;
        const double da_df = 1.0 / (sq * zg);
        const double da_dmu = -a / zg * dzg_dmu;
        const double da_ds = -a / s - a / zg * dzg_ds;
        const double db_df = -lam / ze;
        const double dze_dlam = L * exp(-lam * L);
        const double db_dlam = (1.0 - f) / ze - (1.0 - f) * lam / (ze * ze) * dze_dlam;
        g[0] = Ga * da_df + Gb * db_df;
        g[1] = -(a / (s * s)) * S[2] + Ga * da_dmu;
        g[2] = -(a / (s * s * s)) * S[3] + Ga * da_ds;
        g[3] = b * S[5] + Gb * db_dlam;
        return -S[0];
    }
    // rotated 2-D Gaussians
    const int K = ep.K;
    for (int k = 0; k < K; ++k) {
        const double* t = th + 6 * k;
        const double A = t[0], sx = t[3], sy = t[4];
        double sn, cs;
        sincos(t[5], &sn, &cs);
        const double al = -0.5 / (sx * sx), be = -0.5 / (sy * sy);
        const double* Sk = S + 1 + 6 * k;
        g[6 * k + 0] = Sk[0];
        g[6 * k + 1] = A * (-2.0 * al * cs * Sk[1] + 2.0 * be * sn * Sk[2]);
        g[6 * k + 2] = A * (-2.0 * al * sn * Sk[1] - 2.0 * be * cs * Sk[2]);
        g[6 * k + 3] = A * Sk[3] / (sx * sx * sx);
        g[6 * k + 4] = A * Sk[4] / (sy * sy * sy);
        g[6 * k + 5] = 2.0 * A * (al - be) * Sk[5];
    }
    g[6 * K] = S[1 + 6 * K];
    return S[0];
}

// double-float path (cg_df64.cu)
bool df64_supported(const cg_problem* pb);
size_t df64_split_bytes(const cg_problem* pb);   // workspace for events split into float pairs
cg_status launch_df64(const cg_problem* pb, const double* theta, int64_t n_theta, double* part, WsHeader* hdr,
                      TileGrid* tg, cudaStream_t st, const int* gate, bool value_only, void* split);

}  // namespace cg
