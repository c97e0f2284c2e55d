// cg_df64.cu -- double-float (FP32-pipe) variants of the fused kernels.
//
// Same models, same accumulators and same epilogue as the FP64 kernels
// (cg_models.cuh); only the per-element forward + adjoint arithmetic is
// carried out in df64 (cg_df64.cuh).  Per-thread accumulators are
// compensated float pairs flushed into FP64 sums every kFlush elements, so
// every sum that leaves a thread is FP64.  Elements whose df64 evaluation
// could lose accuracy (an exponential flushed to zero while the model value
// is itself tiny) are recomputed in FP64 in place.
#include <algorithm>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cg_df64.cuh"
#include "cg_internal.cuh"
#include "cg_models.cuh"
#include "cg_models_df64.cuh"
#include "cg_tiles.cuh"

namespace cg {

constexpr int kFlush = 32;   // elements per compensated run before the FP64 flush
constexpr bool kMixPairs = true;   // unbinned kernel: two events per loop iteration

// ===========================================================================
// Unbinned mixture
// ===========================================================================
struct MixDf {
    df mu, c, a, b, mlam, lo;
};

__device__ __forceinline__ void mix_split(const MixConsts& c64, MixDf& c) {
    c.mu = df_from_double(c64.mu);
    c.c = df_from_double(c64.c);
    c.a = df_from_double(c64.a);
    c.b = df_from_double(c64.b);
    c.mlam = df_from_double(-c64.lam);
    c.lo = df_from_double(c64.lo);
}

// FP64 evaluation of one event, added to this thread's FP64 sums (rare path).
template <bool W>
__device__ __noinline__ void mix_elem_fallback(double x, double w, const MixConsts& c64, double* sum, int* bad) {
    double a[MixAcc::N] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool b = false;
    mix_elem_fp64<W>(x, w, c64, a, b);
    for (int k = 0; k < MixAcc::N; ++k) sum[k * 256] += a[k];
    if (b) *bad = 1;
}

// Events (and weights) split into df64 (hi, lo) float pairs once per call,
// so the tiles of every parameter point read them ready to use.
__global__ void k_split_events(const double* __restrict__ x, const double* __restrict__ w, int64_t n,
                               float2* __restrict__ xs, float2* __restrict__ wsp) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const df a = df_split(__ldg(x + i));
        xs[i] = make_float2(a.h, a.l);
        if (w) {
            const df b = df_split(__ldg(w + i));
            wsp[i] = make_float2(b.h, b.l);
        }
    }
}

// One event: forward p(x), adjoint accumulators.  Without weights the log
// terms are gathered as a running product P (one df_log per flush); with
// weights each log is taken and weighted.  X, Wd: the event and its weight
// as df64; i: its index, for the FP64 fallback, which reads the originals.
template <bool W>
__device__ __forceinline__ void mix_elem_df64(df X, df Wd, int64_t i, const MixData& dd, const MixDf& c,
                                              const MixConsts& c64, const DfTables& tab, DfAcc (&acc)[MixAcc::N],
                                              DfProd& P, double* sum, int* bad) {
    const df d = df_sub(X, c.mu);
    const df q = df_mul(c.c, df_sqr(d));
    const df xl = (c.lo.h == 0.0f && c.lo.l == 0.0f) ? X : df_sub(X, c.lo);   // uniform per tile
    const df t = df_mul(c.mlam, xl);
    bool flG = false, flE = false;
    const df eG = df_exp(q, tab, flG);
    const df eE = df_exp(t, tab, flE);
    const df p = df_add(df_mul_nn(c.a, eG), df_mul_nn(c.b, eE));
    // a flushed component (< 1e-30 of its coefficient) is negligible unless p is tiny too
    if ((flG && p.h < 1e-13f * fabsf(c.a.h)) || (flE && p.h < 1e-13f * fabsf(c.b.h)) || !(p.h > 1e-30f)) {
        mix_elem_fallback<W>(dd.x[i], W ? dd.w[i] : 1.0, c64, sum, bad);
        return;
    }
    df r = df_rcp(p);
    if (W) {
        r = df_mul(r, Wd);
        dfacc_add(acc[0], df_mul(df_log(p, tab), Wd));
    } else {
        dfprod_mul(P, p);
    }
    const df U = df_mul_nn(eG, r);
    const df V = df_mul_nn(eE, r);
    const df Ud = df_mul_nn(U, d);
    dfacc_add(acc[1], U);
    dfacc_add(acc[2], Ud);
    dfacc_add(acc[3], df_mul_nn(Ud, d));
    dfacc_add(acc[4], V);
    dfacc_add(acc[5], df_mul_nn(V, xl));
}

template <bool W, int NT>
__global__ void __launch_bounds__(NT, 3) k_mix_df64(MixData d, const double* __restrict__ theta, TileGrid tg,
                                                 double* __restrict__ part, WsHeader* __restrict__ hdr) {
    constexpr int NACC = MixAcc::N;
    __shared__ DfTables tab;
    __shared__ MixConsts cs64;
    __shared__ MixDf cs;
    __shared__ int cs_bad;
    __shared__ double red[NACC * (NT / 32)];
    __shared__ double tot[NACC];
    __shared__ double ssum[NACC * NT];
    static_assert(NT == 256, "fallback sums use a stride of 256");
    if (gated_off(tg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->status = 0;
    df_tables_init(tab);
    for (int t = blockIdx.x; t < tg.n_tiles; t += gridDim.x) {
        const int c = t / tg.n_theta, th = t - c * tg.n_theta;   // chunk-major: a chunk stays in L2 across points
        if (threadIdx.x == 0) {
            cs_bad = mix_prologue(theta + (size_t)th * 4, d.lo, d.hi, cs64) ? 0 : 1;
            mix_split(cs64, cs);
        }
        __syncthreads();
        const MixDf cr = cs;   // per-tile constants in registers
        double* sum = ssum + threadIdx.x;   // this thread's FP64 sums, stride NT
        DfAcc acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            acc[a].s = acc[a].c = 0.0f;
            sum[a * NT] = 0.0;
        }
        DfProd P;
        P.m = df_make(1.0f, 0.0f);
        P.E = 0;
        int bad = 0;
        int cnt = 0;
        const int64_t e0 = (int64_t)c * tg.chunk;
        const int64_t e1 = min(tg.n_elem, e0 + tg.chunk);
        int64_t i = e0 + threadIdx.x;
        const df one = df_make(1.0f, 0.0f);
        auto ev = [&](int64_t k) { const float2 v = __ldg(d.xs + k); return df_make(v.x, v.y); };
        auto wt = [&](int64_t k) {
            if (!W) return one;
            const float2 v = __ldg(d.wsp + k);
            return df_make(v.x, v.y);
        };
        if (kMixPairs) {
            // two independent events per iteration: their dependency chains interleave
            for (; i + NT < e1; i += 2 * NT) {
                const df xa = ev(i), xb = ev(i + NT);
                mix_elem_df64<W>(xa, wt(i), i, d, cr, cs64, tab, acc, P, sum, &bad);
                mix_elem_df64<W>(xb, wt(i + NT), i + NT, d, cr, cs64, tab, acc, P, sum, &bad);
                cnt += 2;
                if (cnt >= kFlush) {
                    if (!W) {
                        dfacc_add(acc[0], dfprod_log(P, tab));
                        P.m = df_make(1.0f, 0.0f);
                        P.E = 0;
                    }
#pragma unroll
                    for (int a = 0; a < NACC; ++a) dfacc_flush(acc[a], sum[a * NT]);
                    cnt = 0;
                }
            }
        }
        df xn = (i < e1) ? ev(i) : one;
        for (; i < e1; i += NT) {
            const df xi = xn;
            if (i + NT < e1) xn = ev(i + NT);   // next event in flight during this one
            mix_elem_df64<W>(xi, wt(i), i, d, cr, cs64, tab, acc, P, sum, &bad);
            if (++cnt == kFlush) {
                if (!W) {
                    dfacc_add(acc[0], dfprod_log(P, tab));
                    P.m = df_make(1.0f, 0.0f);
                    P.E = 0;
                }
#pragma unroll
                for (int a = 0; a < NACC; ++a) dfacc_flush(acc[a], sum[a * NT]);
                cnt = 0;
            }
        }
        if (!W) dfacc_add(acc[0], dfprod_log(P, tab));
#pragma unroll
        for (int a = 0; a < NACC; ++a) dfacc_flush(acc[a], sum[a * NT]);
        double fin[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) fin[a] = sum[a * NT];
        const int any_bad = __syncthreads_or(bad) | cs_bad;
        block_sum<NACC, NT>(fin, red, tot);
        write_partial<NACC>(part, tg, th, c, tot, any_bad);
    }
}

// ===========================================================================
// 1-D Gaussian peaks + polynomial
// ===========================================================================
template <int K, int OBJ, int NT, bool VO>
__global__ void __launch_bounds__(NT, 2) k_gp1_df64(GP1Data d, const double* __restrict__ theta, TileGrid tg,
                                                    double* __restrict__ part, WsHeader* __restrict__ hdr) {
    constexpr int NACC = GP1Acc<K>::N;
    __shared__ DfTables tab;
    __shared__ GP1Consts cs64;
    __shared__ GP1Df cs;
    __shared__ int cs_bad;
    __shared__ double red[NACC * (NT / 32)];
    __shared__ double tot[NACC];
    if (gated_off(tg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->status = 0;
    df_tables_init(tab);
    const int P = 3 * K + d.D + 1;
    for (int t = blockIdx.x; t < tg.n_tiles; t += gridDim.x) {
        const int c = t / tg.n_theta, th = t - c * tg.n_theta;   // chunk-major: a chunk stays in L2 across points
        if (threadIdx.x < 32) {
            const bool ok = gp1_prologue_warp<K, true>(theta + (size_t)th * P, d.D, d.lo, d.h, d.au, d.bu, cs64, cs);
            if (threadIdx.x == 0) cs_bad = ok ? 0 : 1;
        }
        __syncthreads();
        // per-thread sums stay df64 (FP32 pipe) up to the per-warp conversion
        DfAcc acc[NACC];
        df run[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            acc[a].s = acc[a].c = 0.0f;
            run[a] = df_make(0.0f, 0.0f);
        }
        bool bad = false;
        int cnt = 0;
        const int e0 = (int)((int64_t)c * tg.chunk);   // n < 2^24 on this path
        const int e1 = (int)min(tg.n_elem, (int64_t)e0 + tg.chunk);
        float fi = (float)(e0 + (int)threadIdx.x);     // == i exactly
        for (int i = e0 + threadIdx.x; i < e1; i += NT, fi += (float)NT) {
            const double yv = __ldg(d.y + i);
            const df X = d.centres ? df_split(__ldg(d.centres + i)) : gp1_centre_df(cs, fi);
            if (!gp1_elem_df64<K, OBJ, VO>(X, yv, cs, d.D, d.pm, acc, tab)) {
                double tv[NACC];
                int b = 0;
                gp1_elem_fp64_ool<K, OBJ>(d.centres ? d.centres[i] : fma((double)i + 0.5, d.h, d.lo), yv, cs64, d,
                                          tv, &b);
                bad |= (b != 0);
#pragma unroll
                for (int a = 0; a < NACC; ++a) run[a] = df_add(run[a], df_from_double(tv[a]));
            }
            if (++cnt == kFlush) {
#pragma unroll
                for (int a = 0; a < NACC; ++a) dfacc_fold(acc[a], run[a]);
                cnt = 0;
            }
        }
#pragma unroll
        for (int a = 0; a < NACC; ++a) dfacc_fold(acc[a], run[a]);
        const int any_bad = __syncthreads_or(bad ? 1 : 0) | cs_bad;
        block_sum_df<NACC, NT>(run, red, tot);
        write_partial<NACC>(part, tg, th, c, tot, any_bad);
    }
}

template <int K, bool VO>
static cg_status launch_gp1_df64_kv(const cg_problem* pb, const GP1Data& d, const double* theta, int64_t n_theta,
                                    double* part, WsHeader* hdr, TileGrid* tg, cudaStream_t st, const int* gate) {
    constexpr int NT = 256;
    const int64_t n = pb->n_bins[0];
    switch (pb->objective) {
        case CG_OBJ_CHI2:
            return launch_tiles(k_gp1_df64<K, CG_OBJ_CHI2, NT, VO>, NT, d, theta, n, n_theta, part, hdr, tg, st, gate);
        case CG_OBJ_POISSON:
            return launch_tiles(k_gp1_df64<K, CG_OBJ_POISSON, NT, VO>, NT, d, theta, n, n_theta, part, hdr, tg, st,
                                gate);
        case CG_OBJ_POISSON_BC:
            return launch_tiles(k_gp1_df64<K, CG_OBJ_POISSON_BC, NT, VO>, NT, d, theta, n, n_theta, part, hdr, tg,
                                st, gate);
        default: return CG_ERR_UNSUPPORTED;
    }
}

template <int K>
static cg_status launch_gp1_df64_k(const cg_problem* pb, const GP1Data& d, const double* theta, int64_t n_theta,
                                   double* part, WsHeader* hdr, TileGrid* tg, cudaStream_t st, const int* gate,
                                   bool value_only) {
    if (value_only) return launch_gp1_df64_kv<K, true>(pb, d, theta, n_theta, part, hdr, tg, st, gate);
    return launch_gp1_df64_kv<K, false>(pb, d, theta, n_theta, part, hdr, tg, st, gate);
}

// ===========================================================================
// 2-D rotated Gaussians + constant, Poisson (64 x 64-bin tiles, two passes)
// ===========================================================================
constexpr int kR2TX = 64, kR2TY = 64;
constexpr double kR2Cull = 80.0;

struct RG2Df {
    df A[CG_MAX_PEAKS_2D], mx[CG_MAX_PEAKS_2D], my[CG_MAX_PEAKS_2D];
    df cs[CG_MAX_PEAKS_2D], sn[CG_MAX_PEAKS_2D], al[CG_MAX_PEAKS_2D], be[CG_MAX_PEAKS_2D];
    df C, lx, ly, hx, hy;
};

// u, v and e = exp(al u^2 + be v^2) of Gaussian k at centre (X, Y); the same
// code serves both passes, so both see bitwise the same values.
__device__ __forceinline__ df rg2_uve_df(const RG2Df& c, int k, df X, df Y, df& u, df& v, const DfTables& tab,
                                         bool& fl) {
    const df dx = df_sub(X, c.mx[k]), dy = df_sub(Y, c.my[k]);
    u = df_add(df_mul(c.cs[k], dx), df_mul(c.sn[k], dy));
    v = df_sub(df_mul(c.cs[k], dy), df_mul(c.sn[k], dx));
    const df q = df_add(df_mul(c.al[k], df_sqr(u)), df_mul(c.be[k], df_sqr(v)));
    return df_exp(q, tab, fl);
}

template <int K, int NT>
__global__ void __launch_bounds__(NT, 2) k_rg2_df64(RG2Data d, const double* __restrict__ theta, TileGrid tg,
                                                    double* __restrict__ part, WsHeader* __restrict__ hdr) {
    constexpr int NACC = RG2Acc<K>::N;
    __shared__ DfTables tab;
    __shared__ RG2Consts c64;
    __shared__ RG2Df cs;
    __shared__ int cs_bad;
    __shared__ unsigned act_s;
    __shared__ float2 gsm[kR2TX * kR2TY];
    __shared__ double red[6 * (NT / 32)];
    __shared__ double tot[NACC];
    if (gated_off(tg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->status = 0;
    df_tables_init(tab);
    const int P = 6 * K + 1;
    const int ntx = (int)((d.nx + kR2TX - 1) / kR2TX);
    for (int t = blockIdx.x; t < tg.n_tiles; t += gridDim.x) {
        const int c = t / tg.n_theta, th = t - c * tg.n_theta;
        const int ty = c / ntx, tx = c - ty * ntx;
        const int64_t x0 = (int64_t)tx * kR2TX, y0 = (int64_t)ty * kR2TY;
        const int64_t x1 = min(d.nx, x0 + kR2TX), y1 = min(d.ny, y0 + kR2TY);
        if (threadIdx.x == 0) {
            const double* tht = theta + (size_t)th * P;
            cs_bad = rg2_prologue<K>(tht, c64) ? 0 : 1;
            const double bx0 = fma((double)x0 + 0.5, d.hx, d.lx), bx1 = fma((double)(x1 - 1) + 0.5, d.hx, d.lx);
            const double by0 = fma((double)y0 + 0.5, d.hy, d.ly), by1 = fma((double)(y1 - 1) + 0.5, d.hy, d.ly);
            unsigned act = 0;
            for (int k = 0; k < K; ++k) {
                const double mx = tht[6 * k + 1], my = tht[6 * k + 2];
                const double sm = fmax(fabs(tht[6 * k + 3]), fabs(tht[6 * k + 4]));
                const double ddx = fmax(0.0, fmax(bx0 - mx, mx - bx1));
                const double ddy = fmax(0.0, fmax(by0 - my, my - by1));
                if (!(0.5 * (ddx * ddx + ddy * ddy) / (sm * sm) > kR2Cull)) act |= 1u << k;
                cs.A[k] = df_from_double(c64.A[k]);
                cs.mx[k] = df_from_double(c64.mx[k]);
                cs.my[k] = df_from_double(c64.my[k]);
                cs.cs[k] = df_from_double(c64.cs[k]);
                cs.sn[k] = df_from_double(c64.sn[k]);
                cs.al[k] = df_from_double(c64.al[k]);
                cs.be[k] = df_from_double(c64.be[k]);
            }
            cs.C = df_from_double(c64.C);
            cs.lx = df_from_double(d.lx);
            cs.ly = df_from_double(d.ly);
            cs.hx = df_from_double(d.hx);
            cs.hy = df_from_double(d.hy);
            act_s = act;
        }
        __syncthreads();
        const unsigned act = act_s;
        const int w = (int)(x1 - x0);
        const int nbin = w * (int)(y1 - y0);
        bool bad = false;
        // pass 1: model value, objective term and its adjoint g per bin
        DfAcc aT, aG;
        aT.s = aT.c = aG.s = aG.c = 0.0f;
        double sT = 0.0, sG = 0.0;
        int cnt = 0;
        for (int b = threadIdx.x; b < nbin; b += NT) {
            const int r = b / w, col = b - r * w;
            const int64_t ix = x0 + col, iy = y0 + r;
            const df X = df_add(cs.lx, df_mul(cs.hx, two_sum((float)ix, 0.5f)));
            const df Y = df_add(cs.ly, df_mul(cs.hy, two_sum((float)iy, 0.5f)));
            const double nd = __ldg(d.n + iy * d.nx + ix);
            df mu = cs.C;
            bool fl = false;
#pragma unroll 1
            for (int k = 0; k < K; ++k) {
                if (!(act & (1u << k))) continue;
                df u, v;
                const df e = rg2_uve_df(cs, k, X, Y, u, v, tab, fl);
                mu = df_add(mu, df_mul_nn(cs.A[k], e));
            }
            df T, g;
            if (!(mu.h > 1e-30f) || (fl && mu.h < 1e-13f)) {
                // FP64 for this bin's model value (all Gaussians that can contribute)
                const double xc = fma((double)ix + 0.5, d.hx, d.lx), yc = fma((double)iy + 0.5, d.hy, d.ly);
                double m = c64.C;
                for (int k = 0; k < K; ++k) {
                    if (!(act & (1u << k))) continue;
                    const double dx = xc - c64.mx[k], dy = yc - c64.my[k];
                    const double uu = fma(c64.cs[k], dx, c64.sn[k] * dy), vv = fma(c64.cs[k], dy, -c64.sn[k] * dx);
                    m = fma(c64.A[k], exp(fma(c64.al[k], uu * uu, c64.be[k] * vv * vv)), m);
                }
                const double T64 = (nd > 0.0) ? m - nd * log(m) : m;
                const double g64 = 1.0 - nd / m;
                bad |= ((nd > 0.0) && !(m > 0.0)) || !isfinite(T64);
                sT += T64;
                sG += g64;
                g = df_from_double(g64);
            } else {
                const df y = df_split(nd);
                const df rm = df_rcp(mu);
                T = (y.h > 0.0f) ? df_sub(mu, df_mul(y, df_log(mu, tab))) : mu;
                g = df_sub(df_make(1.0f, 0.0f), df_mul(y, rm));
                dfacc_add(aT, T);
                dfacc_add(aG, g);
            }
            gsm[b] = make_float2(g.h, g.l);
            if (++cnt == 32) {
                dfacc_flush(aT, sT);
                dfacc_flush(aG, sG);
                cnt = 0;
            }
        }
        dfacc_flush(aT, sT);
        dfacc_flush(aG, sG);
        const int any_bad = __syncthreads_or(bad ? 1 : 0) | cs_bad;
        // pass 2: the six adjoint sums of each Gaussian that can contribute
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            if (!(act & (1u << k))) {
                if (threadIdx.x < 6) tot[1 + 6 * k + threadIdx.x] = 0.0;
                continue;
            }
            DfAcc a6[6];
            double s6[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                a6[q].s = a6[q].c = 0.0f;
                s6[q] = 0.0;
            }
            cnt = 0;
            for (int b = threadIdx.x; b < nbin; b += NT) {
                const int r = b / w, col = b - r * w;
                const int64_t ix = x0 + col, iy = y0 + r;
                const df X = df_add(cs.lx, df_mul(cs.hx, two_sum((float)ix, 0.5f)));
                const df Y = df_add(cs.ly, df_mul(cs.hy, two_sum((float)iy, 0.5f)));
                df u, v;
                bool fl = false;
                const df e = rg2_uve_df(cs, k, X, Y, u, v, tab, fl);
                const float2 gg = gsm[b];
                const df wgt = df_mul_nn(df_make(gg.x, gg.y), e);
                const df wu = df_mul_nn(wgt, u), wv = df_mul_nn(wgt, v);
                dfacc_add(a6[0], wgt);
                dfacc_add(a6[1], wu);
                dfacc_add(a6[2], wv);
                dfacc_add(a6[3], df_mul_nn(wu, u));
                dfacc_add(a6[4], df_mul_nn(wv, v));
                dfacc_add(a6[5], df_mul_nn(wu, v));
                if (++cnt == 32) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) dfacc_flush(a6[q], s6[q]);
                    cnt = 0;
                }
            }
#pragma unroll
            for (int q = 0; q < 6; ++q) dfacc_flush(a6[q], s6[q]);
            block_sum<6, NT>(s6, red, tot + 1 + 6 * k);
        }
        double s2[2] = {sT, sG};
        __shared__ double tot2[2];
        block_sum<2, NT>(s2, red, tot2);
        if (threadIdx.x == 0) {
            tot[0] = tot2[0];
            tot[1 + 6 * K] = tot2[1];
        }
        __syncthreads();
        write_partial<NACC>(part, tg, th, c, tot, any_bad);
        __syncthreads();
    }
}

template <int K>
static cg_status launch_rg2_df64_k(const RG2Data& d, const double* theta, int64_t n, int64_t n_theta, double* part,
                                   WsHeader* hdr, TileGrid* tg, cudaStream_t st, const int* gate) {
    constexpr int NT = 256;
    auto kern = k_rg2_df64<K, NT>;
    const int R = resident_blocks((const void*)kern, NT, 0);
    const int G = device_sm_count() * R;
    TileGrid g;
    g.n_elem = n;
    g.chunk = 0;
    g.nbx = (int)(((d.nx + kR2TX - 1) / kR2TX) * ((d.ny + kR2TY - 1) / kR2TY));
    g.n_theta = (int)n_theta;
    g.n_tiles = (int)(n_theta * g.nbx);
    g.gate = gate;
    const int grid = g.n_tiles < G ? g.n_tiles : G;
    prof_begin(st);
    kern<<<grid, NT, 0, st>>>(d, theta, g, part, hdr);
    prof_end(st);
    *tg = g;
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

bool df64_supported(const cg_problem* pb) {
    return pb->model == CG_MODEL_MIX_GAUSS_EXP || (pb->model == CG_MODEL_GAUSS_POLY && pb->n_bins[0] < (1 << 24)) ||
           (pb->model == CG_MODEL_ROTGAUSS2D && pb->n_bins[0] < (1 << 24) && pb->n_bins[1] < (1 << 24));
}

size_t df64_split_bytes(const cg_problem* pb) {
    if (pb->model != CG_MODEL_MIX_GAUSS_EXP || pb->precision != CG_PREC_DF64) return 0;
    return align_up((size_t)pb->n_events * sizeof(float2) * (pb->weights ? 2 : 1), 256);
}

cg_status launch_df64(const cg_problem* pb, const double* theta, int64_t n_theta, double* part, WsHeader* hdr,
                      TileGrid* tg, cudaStream_t st, const int* gate, bool value_only, void* split) {
    if (pb->model == CG_MODEL_MIX_GAUSS_EXP) {
        MixData d;
        d.x = pb->data;
        d.w = pb->weights;
        d.lo = pb->lo[0];
        d.hi = pb->hi[0];
        d.vec_ok = 0;
        float2* xs = reinterpret_cast<float2*>(split);
        float2* wsp = pb->weights ? xs + pb->n_events : nullptr;
        d.xs = xs;
        d.wsp = wsp;
        {
            const int64_t blocks = std::min<int64_t>((pb->n_events + 255) / 256, 8 * (int64_t)device_sm_count());
            k_split_events<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(pb->data, pb->weights,
                                                                                  pb->n_events, xs, wsp);
        }
        constexpr int NT = 256;
        if (pb->weights)
            return launch_tiles(k_mix_df64<true, NT>, NT, d, theta, pb->n_events, n_theta, part, hdr, tg, st, gate);
        return launch_tiles(k_mix_df64<false, NT>, NT, d, theta, pb->n_events, n_theta, part, hdr, tg, st, gate);
    }
    if (pb->model == CG_MODEL_GAUSS_POLY) {
        GP1Data d;
        d.y = pb->data;
        d.centres = pb->centres;
        d.lo = pb->lo[0];
        d.h = (pb->hi[0] - pb->lo[0]) / (double)pb->n_bins[0];
        d.au = 2.0 / (pb->hi[0] - pb->lo[0]);
        d.bu = -(pb->lo[0] + pb->hi[0]) / (pb->hi[0] - pb->lo[0]);
        d.D = pb->poly_degree;
        d.pm = pb->poly_mode;
        d.vec_ok = 0;
        switch (pb->n_peaks) {
            case 0: return launch_gp1_df64_k<0>(pb, d, theta, n_theta, part, hdr, tg, st, gate, value_only);
            case 1: return launch_gp1_df64_k<1>(pb, d, theta, n_theta, part, hdr, tg, st, gate, value_only);
            case 2: return launch_gp1_df64_k<2>(pb, d, theta, n_theta, part, hdr, tg, st, gate, value_only);
            case 3: return launch_gp1_df64_k<3>(pb, d, theta, n_theta, part, hdr, tg, st, gate, value_only);
            case 4: return launch_gp1_df64_k<4>(pb, d, theta, n_theta, part, hdr, tg, st, gate, value_only);
            default: return CG_ERR_INVALID_ARG;
        }
    }
    if (pb->model == CG_MODEL_ROTGAUSS2D) {
        RG2Data d;
        d.n = pb->data;
        d.nx = pb->n_bins[0];
        d.ny = pb->n_bins[1];
        d.lx = pb->lo[0];
        d.ly = pb->lo[1];
        d.hx = (pb->hi[0] - pb->lo[0]) / (double)pb->n_bins[0];
        d.hy = (pb->hi[1] - pb->lo[1]) / (double)pb->n_bins[1];
        const int64_t n = d.nx * d.ny;
        switch (pb->n_peaks) {
            case 1: return launch_rg2_df64_k<1>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            case 2: return launch_rg2_df64_k<2>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            case 3: return launch_rg2_df64_k<3>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            case 4: return launch_rg2_df64_k<4>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            case 5: return launch_rg2_df64_k<5>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            case 6: return launch_rg2_df64_k<6>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            case 7: return launch_rg2_df64_k<7>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            case 8: return launch_rg2_df64_k<8>(d, theta, n, n_theta, part, hdr, tg, st, gate);
            default: return CG_ERR_INVALID_ARG;
        }
    }
    return CG_ERR_UNSUPPORTED;
}

}  // namespace cg
