// cg_df64.cu -- double-float (FP32-pipe) variants of the fused kernels.
//
// Same models, same accumulators and same epilogue as the FP64 kernels
// (cg_models.cuh); only the per-element forward + adjoint arithmetic is
// carried out in df64 (cg_df64.cuh).  Per-thread accumulators are
// compensated float pairs flushed into FP64 sums every kFlush elements, so
// every sum that leaves a thread is FP64.  Elements whose df64 evaluation
// could lose accuracy (an exponential flushed to zero while the model value
// is itself tiny) are recomputed in FP64 in place.
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

// One event: forward p(x), adjoint accumulators.  Without weights the log
// terms are gathered as a running product P (one df_log per flush); with
// weights each log is taken and weighted.
template <bool W>
__device__ __forceinline__ void mix_elem_df64(double x, double w, const MixDf& c, const MixConsts& c64,
                                              const DfTables& tab, DfAcc (&acc)[MixAcc::N], DfProd& P,
                                              double* sum, int* bad) {
    const df X = df_split(x);
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
        mix_elem_fallback<W>(x, w, c64, sum, bad);
        return;
    }
    df r = df_rcp(p);
    if (W) {
        const df wd = df_split(w);
        r = df_mul(r, wd);
        dfacc_add(acc[0], df_mul(df_log(p, tab), wd));
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
        double xn = (e0 + threadIdx.x < e1) ? __ldg(d.x + e0 + threadIdx.x) : 0.0;
        for (int64_t i = e0 + threadIdx.x; i < e1; i += NT) {
            const double xi = xn;
            if (i + NT < e1) xn = __ldg(d.x + i + NT);   // next event in flight during this one
            mix_elem_df64<W>(xi, W ? __ldg(d.w + i) : 1.0, cr, cs64, tab, acc, P, sum, &bad);
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
template <int K, int OBJ, int NT>
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
        if (threadIdx.x == 0) {
            cs_bad = gp1_prologue<K>(theta + (size_t)th * P, d.D, cs64) ? 0 : 1;
            gp1_split(cs64, d.lo, d.h, d.au, d.bu, K, cs);
        }
        __syncthreads();
        DfAcc acc[NACC];
        double sum[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) {
            acc[a].s = acc[a].c = 0.0f;
            sum[a] = 0.0;
        }
        bool bad = false;
        int cnt = 0;
        const int64_t e0 = (int64_t)c * tg.chunk;
        const int64_t e1 = min(tg.n_elem, e0 + tg.chunk);
        for (int64_t i = e0 + threadIdx.x; i < e1; i += NT) {
            const double yv = __ldg(d.y + i);
            const df X = d.centres ? df_split(__ldg(d.centres + i)) : gp1_centre_df(cs, i);
            if (!gp1_elem_df64<K, OBJ>(X, yv, cs, d.D, d.pm, acc, tab)) {
                const double x = d.centres ? d.centres[i] : fma((double)i + 0.5, d.h, d.lo);
                gp1_elem_fp64<K, OBJ>(x, yv, cs64, d, sum, bad);
            }
            if (++cnt == kFlush) {
#pragma unroll
                for (int a = 0; a < NACC; ++a) dfacc_flush(acc[a], sum[a]);
                cnt = 0;
            }
        }
#pragma unroll
        for (int a = 0; a < NACC; ++a) dfacc_flush(acc[a], sum[a]);
        const int any_bad = __syncthreads_or(bad ? 1 : 0) | cs_bad;
        block_sum<NACC, NT>(sum, red, tot);
        write_partial<NACC>(part, tg, th, c, tot, any_bad);
    }
}

template <int K>
static cg_status launch_gp1_df64_k(const cg_problem* pb, const GP1Data& d, const double* theta, int64_t n_theta,
                                   double* part, WsHeader* hdr, TileGrid* tg, cudaStream_t st, const int* gate) {
    constexpr int NT = 256;
    const int64_t n = pb->n_bins[0];
    switch (pb->objective) {
        case CG_OBJ_CHI2:
            return launch_tiles(k_gp1_df64<K, CG_OBJ_CHI2, NT>, NT, d, theta, n, n_theta, part, hdr, tg, st, gate);
        case CG_OBJ_POISSON:
            return launch_tiles(k_gp1_df64<K, CG_OBJ_POISSON, NT>, NT, d, theta, n, n_theta, part, hdr, tg, st, gate);
        case CG_OBJ_POISSON_BC:
            return launch_tiles(k_gp1_df64<K, CG_OBJ_POISSON_BC, NT>, NT, d, theta, n, n_theta, part, hdr, tg, st,
                                gate);
        default: return CG_ERR_UNSUPPORTED;
    }
}

bool df64_supported(const cg_problem* pb) {
    return pb->model == CG_MODEL_MIX_GAUSS_EXP || (pb->model == CG_MODEL_GAUSS_POLY && pb->n_bins[0] < (1 << 24));
}

cg_status launch_df64(const cg_problem* pb, const double* theta, int64_t n_theta, double* part, WsHeader* hdr,
                      TileGrid* tg, cudaStream_t st, const int* gate) {
    if (pb->model == CG_MODEL_MIX_GAUSS_EXP) {
        MixData d;
        d.x = pb->data;
        d.w = pb->weights;
        d.lo = pb->lo[0];
        d.hi = pb->hi[0];
        d.vec_ok = 0;
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
            case 0: return launch_gp1_df64_k<0>(pb, d, theta, n_theta, part, hdr, tg, st, gate);
            case 1: return launch_gp1_df64_k<1>(pb, d, theta, n_theta, part, hdr, tg, st, gate);
            case 2: return launch_gp1_df64_k<2>(pb, d, theta, n_theta, part, hdr, tg, st, gate);
            case 3: return launch_gp1_df64_k<3>(pb, d, theta, n_theta, part, hdr, tg, st, gate);
            case 4: return launch_gp1_df64_k<4>(pb, d, theta, n_theta, part, hdr, tg, st, gate);
            default: return CG_ERR_INVALID_ARG;
        }
    }
    return CG_ERR_UNSUPPORTED;
}

}  // namespace cg
