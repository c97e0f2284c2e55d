// cg_fit.cu -- histogram batches and the BFGS fitters of libcg.
//
// The paper uses AD gradients inside the histogram fitter, whose minimiser
// takes the gradient from AD and no second derivatives (Sec. 4).  The
// gradient-only minimiser here is BFGS with a backtracking Armijo line
// search (steps in cg.h, cg_fit_step).  Every objective evaluation is the
// fused forward + adjoint of cg_models.cuh over one histogram's bins.
//
// Batched fitter: ONE persistent launch fits thousands of histograms of
// uneven size.  Three granularities share the launch, chosen per histogram
// by the plan (cg_fit_plan): a cluster of CTAs (largest histograms; the
// per-CTA partial sums are combined through distributed shared memory), one
// CTA, or one warp (smallest).  Each granularity pops histograms from its
// own size-sorted queue with an integer atomic; no unit ever waits for
// another.  Inside a unit the data-parallel part (the bins) is spread over
// all its threads and reduced in a fixed order; the control part (search
// direction, line search, BFGS update) is done by one warp, lane i owning
// row i of the inverse-Hessian approximation.  In a cluster every CTA runs
// the control part on the same broadcast sums, so all CTAs take the same
// branches and reach the same cluster barriers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "cg_internal.cuh"
#include "cg_models.cuh"
#include "cg_models_df64.cuh"
#include "cg_models_fp64.cuh"
#include "cg_tiles.cuh"

namespace cgx = cooperative_groups;

namespace cg {
size_t grad_workspace_bytes(const cg_problem* pb, int64_t n_theta);
cg_status grad_points(const cg_problem* pb, const double* theta, int64_t n_theta, double* value, double* grad,
                      void* ws, size_t ws_bytes, cudaStream_t st, const int* gate);

namespace {

constexpr int FP = CG_FIT_MAX_PARAMS;
constexpr int kMaxTrials = 20;
constexpr double kArmijo = 1e-4;
constexpr int kMaxWarpsPerCta = 16;

enum { UNIT_WARP = 0, UNIT_CTA = 1, UNIT_CLUSTER = 2 };

// Per-unit fit state in shared memory.
struct FitSm {
    double th[FP], g[FP], d[FP], tt[FP], gt[FP], h0[FP], sv[FP], yv[FP], hy[FP];
    double H[FP * FP];
    double f, ft, gd, alpha, edm;
    double fdata;   // the value's data-only part (cg_fit_state::fdata)
    int P, iter, n_eval, status, ntrial, go, upd, bad;
};

struct Geom {   // one histogram
    const double* y;
    int64_t n;
    double lo, hw;
};

// Arguments of the fit kernels.
struct FitArgs {
    cg_fit_state* st;
    const double* data;
    const int64_t* offsets;
    const double* lo;
    const double* hi;
    const double* theta;   // grad mode: [H][P]; init mode: theta0 [H][P]
    double* value;         // grad mode
    double* grad;          // grad mode
    double* gn;            // mode 4: Gauss-Newton matrices [H][P][P]
    const int* queue[3];   // histogram ids per unit kind (cluster, cta, warp), sorted by size
    const int* n_items;    // device [3]: queue lengths (written by the plan)
    int* counters;         // 3 ints, zeroed before each persistent launch
    const int* order;      // k_fit_eval: histograms by decreasing size (NULL: index order, grid-stride)
    int* ectr;             // k_fit_eval / k_lm_tiles: queue position, zero at launch
    const void* lm_hdr;    // LM: plan header (tile count, magic)
    const int2* tiles;     // LM: (histogram, chunk) per tile, histograms by decreasing size
    const int2* hspan;     // LM: (first tile, tile count) per histogram
    size_t ws_bytes;       // LM: workspace size (bounds the tile count read from the header)
    int64_t H;
    int P, D, pm, n_steps;
    double tol;
};

__device__ __forceinline__ Geom geom_of(const FitArgs& a, int64_t h) {
    Geom g;
    const int64_t b0 = a.offsets[h], b1 = a.offsets[h + 1];
    g.y = a.data + b0;
    g.n = b1 - b0;
    g.lo = a.lo[h];
    g.hw = (a.hi[h] - a.lo[h]) / (double)(g.n > 0 ? g.n : 1);
    return g;
}

// ---------------------------------------------------------------------------
// Data-parallel part: accumulate one histogram's bins (thread t0 of T).
// ---------------------------------------------------------------------------
template <int K, int OBJ>
__device__ __forceinline__ void acc_bins(const Geom& G, const GP1Consts& cs, const GP1Data& dd, int t0, int T,
                                         double (&acc)[GP1Acc<K>::N], bool& bad) {
    for (int64_t i = t0; i < G.n; i += T) {
        const double x = fma((double)i + 0.5, G.hw, G.lo);
        gp1_elem_fp64<K, OBJ>(x, __ldg(G.y + i), cs, dd, acc, bad);
    }
}

// The same on the table-driven FP64 functions (FP64 batches): the thread's
// sums leave with the objective's factors applied (gp1_tile_scale), and a
// non-finite value sum sets bad.  acc must start at zero.  DATA = false
// leaves out the part of the value that depends on the counts alone
// (data_part_f64; the fit adds it from its state).
template <int K, int OBJ, bool DATA = true>
__device__ __forceinline__ void acc_bins_f64(const Geom& G, const GP1Consts& cs, const GP1Data& dd,
                                             const Fp64Tab& tab, int t0, int T, double (&acc)[GP1Acc<K>::N],
                                             bool& bad) {
    GP1C2 c2;
    gp1_c2(cs, K, c2);
    const double hh = 0.5 * G.hw;   // centre (2i + 1) (h/2) + lo, correctly rounded
    gp1_dispatch(dd.D, dd.pm, [&](auto dd_, auto pm_) {
        constexpr int DD = decltype(dd_)::value, PM = decltype(pm_)::value;
        for (int64_t i = t0; i < G.n; i += T) {
            const GP1Bin b = gp1_bin<OBJ, PM, DATA>(fma((double)(2 * i + 1), hh, G.lo), __ldg(G.y + i), dd, tab);
            gp1_elem_f64<K, OBJ, DD, DATA>(b, cs, c2, tab, acc, bad);
        }
    });
    gp1_tile_scale<K, OBJ>(acc);
    bad |= nonfinite(acc[0]);
}

// This thread's share of the value's part that depends on the counts alone:
// Baker-Cousins 2 sum (y log y - y) over y > 0 (the terms gp1_bin leaves out
// with DATA = false, in the same arithmetic); 0 for chi2 and Poisson.
template <int OBJ>
__device__ __forceinline__ double data_part_f64(const Geom& G, const Fp64Tab& tab, int t0, int T) {
    double s = 0.0;
    if (OBJ == CG_OBJ_POISSON_BC)
        for (int64_t i = t0; i < G.n; i += T) {
            const double y = __ldg(G.y + i);
            if (__double_as_longlong(y) > 0) s += fma(y, flog(y, tab), -y);
        }
    return 2.0 * s;
}

// Gauss-Newton diagonal terms of one bin: h (df/dtheta_k)^2 with h = d2T/df2.
template <int K, int OBJ>
__device__ __forceinline__ void gn_elem_fp64(double x, double y, const GP1Consts& cs, const GP1Data& dd,
                                             double (&acc)[GP1Acc<K>::N]) {
    const double u = dd.pm ? fma(x, dd.au, dd.bu) : x;
    double f = 0.0;
#pragma unroll
    for (int j = 3; j >= 0; --j) {
        if (j == dd.D) f = cs.poly[j];
        else if (j < dd.D) f = fma(f, u, cs.poly[j]);
    }
    double dk[K], ek[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        dk[k] = x - cs.mu[k];
        ek[k] = exp(cs.c[k] * dk[k] * dk[k]);
        f = fma(cs.A[k], ek[k], f);
    }
    double h;   // an empty bin's Poisson term is linear in f: curvature 0
    if (OBJ == CG_OBJ_CHI2) h = 2.0 / fmax(y, 1.0);
    else if (OBJ == CG_OBJ_POISSON) h = (y > 0.0) ? y / (f * f) : 0.0;
    else h = (y > 0.0) ? 2.0 * y / (f * f) : 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double he = h * ek[k] * ek[k];
        const double d2 = dk[k] * dk[k];
        acc[1 + 3 * k] += he;
        acc[2 + 3 * k] = fma(he, d2, acc[2 + 3 * k]);
        acc[3 + 3 * k] = fma(he * d2, d2, acc[3 + 3 * k]);
    }
    double up = 1.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (j <= dd.D) acc[1 + 3 * K + j] = fma(h, up * up, acc[1 + 3 * K + j]);
        if (j < dd.D) up *= u;
    }
}

template <int K, int OBJ>
__device__ __forceinline__ void gn_bins(const Geom& G, const GP1Consts& cs, const GP1Data& dd, int t0, int T,
                                        double (&acc)[GP1Acc<K>::N]) {
    for (int64_t i = t0; i < G.n; i += T)
        gn_elem_fp64<K, OBJ>(fma((double)i + 0.5, G.hw, G.lo), __ldg(G.y + i), cs, dd, acc);
}

// The df64 bin centres are exact below this many bins; longer histograms are
// evaluated in FP64 whatever the batch precision.
constexpr int64_t kDfMaxBins = (int64_t)1 << 24;
constexpr int kFitFlush = 32;

// FP64 terms of one bin that the df64 path hands back (rare).  Kept out of
// line so that the bin loop keeps no FP64 state: out[0..N) gradient
// accumulators, out[N..2N) Gauss-Newton terms (GN only).
template <int K, int OBJ, bool GN>
static __device__ __noinline__ void gp1_fallback_fp64(double x, double y, const GP1Consts& cs, GP1Data dd,
                                                      double* out, int* bad) {
    constexpr int N = GP1Acc<K>::N;
    double a[N], g[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = g[i] = 0.0;
    bool b = false;
    gp1_elem_fp64<K, OBJ>(x, y, cs, dd, a, b);
    if (GN) gn_elem_fp64<K, OBJ>(x, y, cs, dd, g);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        out[i] = a[i];
        out[N + i] = g[i];
    }
    *bad = b ? 1 : 0;
}

// Gauss-Newton matrix factors of one bin in FP64, for the bins the df64
// element hands to the FP64 fallback: q = the raw factors r (as in the df64
// element) divided by f for the Poisson forms, and hs with h r_a r_b =
// hs q_a q_b (2w for chi2, y for Poisson, 2y for Baker-Cousins; 0 for an empty
// Poisson bin).
template <int K, int OBJ>
static __device__ __noinline__ void gnm_fallback_fp64(double x, double y, const GP1Consts& cs, GP1Data dd,
                                                      double* q, double* hs) {
    constexpr int R = GP1Gnm<K>::R;
    const double u = dd.pm ? fma(x, dd.au, dd.bu) : x;
    double f = 0.0;
    for (int j = 3; j >= 0; --j) {
        if (j == dd.D) f = cs.poly[j];
        else if (j < dd.D) f = fma(f, u, cs.poly[j]);
    }
    double dk[K], ek[K];
    for (int k = 0; k < K; ++k) {
        dk[k] = x - cs.mu[k];
        ek[k] = exp(cs.c[k] * dk[k] * dk[k]);
        f = fma(cs.A[k], ek[k], f);
    }
    double sc = 1.0;
    if (OBJ == CG_OBJ_CHI2) {
        *hs = 2.0 / fmax(y, 1.0);
    } else {
        *hs = (y > 0.0) ? (OBJ == CG_OBJ_POISSON ? y : 2.0 * y) : 0.0;
        sc = (y > 0.0) ? 1.0 / f : 0.0;
    }
    for (int k = 0; k < K; ++k) {
        const double e = ek[k] * sc;
        q[3 * k] = e;
        q[3 * k + 1] = e * dk[k];
        q[3 * k + 2] = e * dk[k] * dk[k];
    }
    double up = sc;
    for (int j = 0; j < 4; ++j) {
        q[3 * K + j] = (j <= dd.D) ? up : 0.0;
        up *= u;
    }
    (void)R;
}

// The same in double-float arithmetic (FP32 pipe): every kFitFlush bins the
// compensated accumulators are folded into the df64 running sums run[]
// (zeroed here), which leave the thread as df64 and are converted to FP64
// once per warp by the reductions; elements that need it are evaluated in
// FP64 and folded into the same running sums.  GN: also the Gauss-Newton
// diagonal terms, into grun[].  VO: the value term only (run[0]).  GNM: the
// Gauss-Newton matrix terms in FP32 into gm (elements that fall back to FP64
// take their terms in FP64 and add them rounded to FP32).
// Requires G.n < kDfMaxBins (bin index and centre exact in FP32 / df64).
template <int K, int OBJ, bool GN, bool VO = false, bool GNM = false>
__device__ __forceinline__ void acc_bins_df64(const Geom& G, const GP1Consts& cs, const GP1Df& cd,
                                              const GP1Data& dd, const DfTables& tab, int t0, int T,
                                              df (&run)[GP1Acc<K>::N], df (&grun)[GP1Acc<K>::N], bool& bad,
                                              float* gm = nullptr) {
    constexpr int N = GP1Acc<K>::N;
    constexpr int NG = GN ? N : 1;
    DfAcc da[N], ga[NG];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        da[a].s = da[a].c = 0.0f;
        run[a] = df_make(0.0f, 0.0f);
    }
#pragma unroll
    for (int a = 0; a < NG; ++a) {
        ga[a].s = ga[a].c = 0.0f;
        grun[a] = df_make(0.0f, 0.0f);
    }
    const int n = (int)G.n;
    const float fT = (float)T;
    float fi = (float)t0;   // == i exactly (i < 2^24)
    int cnt = 0;
    for (int i = t0; i < n; i += T, fi += fT) {
        const double y = __ldg(G.y + i);
        if (!gp1_elem_df64<K, OBJ, VO, GN, GNM>(gp1_centre_df(cd, fi), y, cd, dd.D, dd.pm, da, tab, ga, gm)) {
            double t[2 * N];
            int b = 0;
            gp1_fallback_fp64<K, OBJ, GN>(fma((double)i + 0.5, G.hw, G.lo), y, cs, dd, t, &b);
            bad |= (b != 0);
#pragma unroll
            for (int a = 0; a < N; ++a) run[a] = df_add(run[a], df_from_double(t[a]));
            if (GN) {
#pragma unroll
                for (int a = 1; a < NG; ++a) grun[a] = df_add(grun[a], df_from_double(t[N + a]));
            }
            if constexpr (GNM) {
                constexpr int R = GP1Gnm<K>::R;
                double q[R], hs;
                gnm_fallback_fp64<K, OBJ>(fma((double)i + 0.5, G.hw, G.lo), y, cs, dd, q, &hs);
                int p = 0;
#pragma unroll
                for (int a2 = 0; a2 < R; ++a2) {
                    const double ha = hs * q[a2];
#pragma unroll
                    for (int b2 = a2; b2 < R; ++b2) {
                        gm[p] += (float)(ha * q[b2]);
                        ++p;
                    }
                }
            }
        }
        if (++cnt == kFitFlush) {
#pragma unroll
            for (int a = 0; a < N; ++a) dfacc_fold(da[a], run[a]);
            if (GN) {
#pragma unroll
                for (int a = 1; a < NG; ++a) dfacc_fold(ga[a], grun[a]);
            }
            cnt = 0;
        }
    }
#pragma unroll
    for (int a = 0; a < N; ++a) dfacc_fold(da[a], run[a]);
    if (GN) {
#pragma unroll
        for (int a = 1; a < NG; ++a) dfacc_fold(ga[a], grun[a]);
    }
}

// ---------------------------------------------------------------------------
// Reductions of the accumulators over one unit; result in tot[] (shared).
// ---------------------------------------------------------------------------
// Warp totals of N accumulators into dst[a * stride]: FP64 butterflies for
// FP64 values; for df64 values the reduce-scatter sum on the FP32 pipe with
// one conversion per accumulator.
template <int N>
__device__ __forceinline__ void warp_totals(const double (&acc)[N], double* dst, int stride) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < N; ++a) {
        const double v = warp_sum(acc[a]);
        if (lane == 0) dst[a * stride] = v;
    }
}
template <int N>
__device__ __forceinline__ void warp_totals(const df (&acc)[N], double* dst, int stride) {
    warp_sum_df_to<N>(acc, dst, stride);
}

// Warp totals of NV FP32 accumulators (chunks of 32 values through the df64
// reduce-scatter; exact FP32 inputs), one FP64 value per accumulator.
template <int NV>
__device__ __forceinline__ void warp_totals_f(const float (&v)[NV], double* dst, int stride) {
    constexpr int NC = (NV + 31) / 32;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        constexpr int W = 32;
        df w[W];
#pragma unroll
        for (int i = 0; i < W; ++i) w[i] = df_make((c * W + i < NV) ? v[(c * W + i < NV) ? c * W + i : 0] : 0.0f, 0.0f);
        warp_sum_df_to<W>(w, dst + (size_t)c * W * stride, stride);
    }
}

template <int N, typename T>
__device__ __forceinline__ void reduce_warp(const T (&acc)[N], double* tot) {
    warp_totals<N>(acc, tot, 1);
    __syncwarp();
}
template <int N, typename T>
__device__ __forceinline__ void reduce_cta(const T (&acc)[N], double* red, double* tot) {
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_totals<N>(acc, red + wid, kMaxWarpsPerCta);
    __syncthreads();
    if (threadIdx.x < N) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[threadIdx.x * kMaxWarpsPerCta + w];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
}
template <int N, typename T>
__device__ __forceinline__ void reduce_cluster(const T (&acc)[N], double* red, double* part, double* tot) {
    cgx::cluster_group cl = cgx::this_cluster();
    reduce_cta<N, T>(acc, red, part);
    cl.sync();
    const unsigned nr = cl.num_blocks();
    if (cl.block_rank() == 0 && threadIdx.x < N) {
        double s = 0.0;
        for (unsigned r = 0; r < nr; ++r) s += cl.map_shared_rank(part, r)[threadIdx.x];
        tot[threadIdx.x] = s;
    }
    cl.sync();
    if (cl.block_rank() != 0 && threadIdx.x < N) tot[threadIdx.x] = cl.map_shared_rank(tot, 0)[threadIdx.x];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Control part, executed by one full warp on the unit's FitSm.  Lane i < P
// owns parameter i (and row i of the inverse-Hessian approximation); dot
// products are lane products summed by a warp butterfly, and the P x P
// update is spread over all 32 lanes.  An FP64 warp instruction occupies the
// FP64 pipe for the whole warp whatever the number of active lanes, so the
// control issues as few FP64 instructions as it can, none of them serial
// over the parameters.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ctl_direction(FitSm& s, int lane) {
    const int P = s.P;
    const bool own = lane < P;
    double dl = 0.0;
    if (own) {
        double acc = 0.0;
        for (int j = 0; j < P; ++j) acc = fma(s.H[lane * FP + j], s.g[j], acc);
        dl = -acc;
    }
    double gd = warp_sum(own ? s.g[lane] * dl : 0.0);
    if (!(gd < 0.0)) {  // not a descent direction: restart from the initial diagonal
        if (own) {
            for (int j = 0; j < P; ++j) s.H[lane * FP + j] = (j == lane) ? s.h0[lane] : 0.0;
            dl = -s.h0[lane] * s.g[lane];
        }
        gd = warp_sum(own ? s.g[lane] * dl : 0.0);
    }
    if (own) {
        s.d[lane] = dl;
        s.tt[lane] = s.th[lane] + dl;
    }
    if (lane == 0) {
        s.gd = gd;
        s.alpha = 1.0;
        s.ntrial = 0;
    }
    __syncwarp();
}

// After an evaluation at tt: go = 1 accepted (BFGS update done), 0 retry
// with a new tt, 2 stop (line search failed).
__device__ __forceinline__ void ctl_after_eval(FitSm& s, int lane, double tol) {
    const int P = s.P;
    const bool own = lane < P;
    if (lane == 0) {
        s.n_eval += 1;
        const double ft = s.bad ? __longlong_as_double(0x7ff0000000000000LL) : s.ft;
        const bool ok = isfinite(ft) && ft <= s.f + kArmijo * s.alpha * s.gd;
        if (ok) {
            s.go = 1;
        } else {
            s.ntrial += 1;
            if (s.ntrial >= kMaxTrials) {
                s.go = 2;
                s.status = CG_FIT_LINESEARCH_FAILED;
            } else {
                const double a = s.alpha;
                double an;
                if (isfinite(ft)) {
                    const double den = 2.0 * (ft - s.f - s.gd * a);
                    an = (den > 0.0) ? -s.gd * a * a / den : 0.5 * a;
                    an = fmin(fmax(an, 0.1 * a), 0.5 * a);
                } else {
                    an = 0.1 * a;
                }
                s.alpha = an;
                s.go = 0;
            }
        }
    }
    __syncwarp();
    if (s.go == 0) {
        if (own) s.tt[lane] = fma(s.alpha, s.d[lane], s.th[lane]);
        __syncwarp();
        return;
    }
    if (s.go == 2) return;
    // accepted: BFGS update with step sv and gradient change yv
    double sv = 0.0, yv = 0.0;
    if (own) {
        sv = s.tt[lane] - s.th[lane];
        yv = s.gt[lane] - s.g[lane];
        s.sv[lane] = sv;
        s.yv[lane] = yv;
    }
    __syncwarp();
    double hy = 0.0;
    if (own) {
        for (int j = 0; j < P; ++j) hy = fma(s.H[lane * FP + j], s.yv[j], hy);
        s.hy[lane] = hy;
    }
    const double sy = warp_sum(sv * yv), yhy = warp_sum(yv * hy);
    const double ss = warp_sum(sv * sv), yy = warp_sum(yv * yv);
    const double rq = sqrt(lane == 0 ? ss : yy);   // both roots in one instruction sequence
    const double rs = __shfl_sync(0xffffffffu, rq, 0), ry = __shfl_sync(0xffffffffu, rq, 1);
    __syncwarp();
    if (sy > 1e-12 * rs * ry) {   // the same decision in every lane
        const double r = 1.0 / sy;
        const double c = (1.0 + r * yhy) * r;
        for (int e = lane; e < P * P; e += 32) {
            const int i = e / P, j = e - i * P;
            s.H[i * FP + j] += -r * (s.sv[i] * s.hy[j] + s.hy[i] * s.sv[j]) + c * s.sv[i] * s.sv[j];
        }
    }
    __syncwarp();
    if (own) {
        s.th[lane] = s.tt[lane];
        s.g[lane] = s.gt[lane];
    }
    __syncwarp();
    // EDM with the updated approximation
    double hg = 0.0;
    if (own) {
        for (int j = 0; j < P; ++j) hg = fma(s.H[lane * FP + j], s.g[j], hg);
    }
    const double e = warp_sum(own ? s.g[lane] * hg : 0.0);
    if (lane == 0) {
        s.f = s.ft;
        s.iter += 1;
        s.edm = 0.5 * e;
        if (s.edm < tol * fmax(1.0, fabs(s.f))) s.status = CG_FIT_CONVERGED;
    }
    __syncwarp();
}

// Gradient component k of the 1-D model from its summed accumulators S (the
// chain rule of the epilogue in cg_models.cuh, one parameter per lane).
template <int K>
__device__ __forceinline__ double gp1_grad_component(int k, const double* th, const double* S) {
    if (k < 3 * K) {
        const int p = k / 3, role = k - 3 * p;
        const double A = th[3 * p], sg = th[3 * p + 2];
        if (role == 0) return S[1 + 3 * p];
        if (role == 1) return A / (sg * sg) * S[2 + 3 * p];
        return A / (sg * sg * sg) * S[3 + 3 * p];
    }
    return S[1 + k];
}

// Sum one unit's accumulators into tot[] (shared) and OR its domain flags.
__device__ __forceinline__ void set_flag(double& x, bool b) { x = b ? 1.0 : 0.0; }
__device__ __forceinline__ void set_flag(df& x, bool b) { x = df_make(b ? 1.0f : 0.0f, 0.0f); }

template <int UNIT, int N, typename T>
__device__ __forceinline__ int unit_reduce(const T (&v)[N], bool bad, double* red, double* part, double* tot) {
    if (UNIT == UNIT_WARP) {
        const int any_bad = __any_sync(0xffffffffu, bad);
        reduce_warp<N, T>(v, tot);
        return any_bad;
    }
    if (UNIT == UNIT_CTA) {
        const int any_bad = __syncthreads_or(bad);
        reduce_cta<N, T>(v, red, tot);
        return any_bad;
    }
    // the flag travels as one more accumulator through the cluster sum
    T v2[N + 1];
#pragma unroll
    for (int a = 0; a < N; ++a) v2[a] = v[a];
    set_flag(v2[N], bad);
    reduce_cluster<N + 1, T>(v2, red, part, tot);
    return tot[N] != 0.0;
}

// ---------------------------------------------------------------------------
// One objective evaluation of histogram G at s.tt by a unit (all threads).
// ---------------------------------------------------------------------------
template <int UNIT, int K, int OBJ, int PREC>
__device__ __forceinline__ void unit_eval(FitSm& s, GP1Consts& cs, GP1Df& cd, const DfTables& tab,
                                          const Fp64Tab* t64, const Geom& G, const GP1Data& dd, int D, double* red,
                                          double* part, double* tot, int t0, int T) {
    constexpr int N = GP1Acc<K>::N;
    const int lane = threadIdx.x & 31;
    if (UNIT == UNIT_WARP || threadIdx.x < 32) {   // the constants, one per lane of the control warp
        const bool ok = gp1_prologue_warp<K, PREC == CG_PREC_DF64>(s.tt, D, G.lo, G.hw, dd.au, dd.bu, cs, cd);
        if (lane == 0) s.bad = ok ? 0 : 1;
    }
    if (UNIT == UNIT_WARP) __syncwarp(); else __syncthreads();
    bool bad = false;
    int any_bad;
    if (PREC == CG_PREC_DF64 && G.n < kDfMaxBins) {
        df v[N], unused[N];
        acc_bins_df64<K, OBJ, false>(G, cs, cd, dd, tab, t0, T, v, unused, bad);
        any_bad = unit_reduce<UNIT, N>(v, bad, red, part, tot);
    } else {
        double acc[N];
#pragma unroll
        for (int a = 0; a < N; ++a) acc[a] = 0.0;
        // FP64: the counts-only part of the value comes from the state (s.fdata)
        if (PREC == CG_PREC_FP64) acc_bins_f64<K, OBJ, false>(G, cs, dd, *t64, t0, T, acc, bad);
        else acc_bins<K, OBJ>(G, cs, dd, t0, T, acc, bad);   // df64 batches: histograms of 2^24 bins or more
        any_bad = unit_reduce<UNIT, N>(acc, bad, red, part, tot);
    }
    if (UNIT == UNIT_WARP || threadIdx.x < 32) {   // value and gradient, one parameter per lane
        if (lane < s.P) s.gt[lane] = gp1_grad_component<K>(lane, s.tt, tot);
        if (lane == 0) {
            s.ft = tot[0] + s.fdata;
            s.bad |= any_bad ? 1 : 0;
        }
    }
    if (UNIT == UNIT_WARP) __syncwarp(); else __syncthreads();
}

// Load / store the per-histogram state.
__device__ __forceinline__ void state_load(FitSm& s, const cg_fit_state* st, int lane_or_tid, int nthr) {
    for (int k = lane_or_tid; k < FP; k += nthr) {
        s.th[k] = st->theta[k];
        s.g[k] = st->grad[k];
        s.h0[k] = st->h0[k];
    }
    for (int k = lane_or_tid; k < FP * FP; k += nthr) s.H[k] = st->hinv[k];
    if (lane_or_tid == 0) {
        s.f = st->f;
        s.edm = st->edm;
        s.fdata = st->fdata;
        s.iter = st->iter;
        s.n_eval = st->n_eval;
        s.status = st->status;
        s.P = st->n_params;
    }
}

__device__ __forceinline__ void state_store(const FitSm& s, cg_fit_state* st, int lane_or_tid, int nthr) {
    for (int k = lane_or_tid; k < FP; k += nthr) {
        st->theta[k] = s.th[k];
        st->grad[k] = s.g[k];
    }
    for (int k = lane_or_tid; k < FP * FP; k += nthr) st->hinv[k] = s.H[k];
    if (lane_or_tid == 0) {
        st->f = s.f;
        st->edm = s.edm;
        st->iter = s.iter;
        st->n_eval = s.n_eval;
        st->status = s.status;
    }
}

// Fit one histogram with one unit for up to a.n_steps iterations.
template <int UNIT, int K, int OBJ, int PREC>
__device__ void unit_fit(const FitArgs& a, int64_t h, FitSm& s, GP1Consts& cs, GP1Df& cd, const DfTables& tab,
                         const Fp64Tab* t64, double* red, double* part, double* tot, int t0, int T) {
    const int lane = threadIdx.x & 31;
    const bool ctl = (UNIT == UNIT_WARP) || (threadIdx.x < 32);
    const int ld_id = (UNIT == UNIT_WARP) ? lane : threadIdx.x;
    const int ld_n = (UNIT == UNIT_WARP) ? 32 : blockDim.x;
    state_load(s, a.st + h, ld_id, ld_n);
    if (UNIT == UNIT_WARP) __syncwarp(); else __syncthreads();
    const Geom G = geom_of(a, h);
    GP1Data dd;
    dd.y = G.y;
    dd.centres = nullptr;
    dd.lo = G.lo;
    dd.h = G.hw;
    dd.au = 2.0 / (a.hi[h] - a.lo[h]);
    dd.bu = -(a.lo[h] + a.hi[h]) / (a.hi[h] - a.lo[h]);
    dd.D = a.D;
    dd.pm = a.pm;
    dd.vec_ok = 0;
    if (ctl && lane == 0 && s.status == CG_FIT_RUNNING && s.edm < a.tol * fmax(1.0, fabs(s.f)))
        s.status = CG_FIT_CONVERGED;
    if (UNIT == UNIT_WARP) __syncwarp(); else __syncthreads();
    const int it_end = s.iter + a.n_steps;
    while (s.status == CG_FIT_RUNNING && s.iter < it_end) {
        if (ctl) ctl_direction(s, lane);
        if (UNIT != UNIT_WARP) __syncthreads();
        for (;;) {
            unit_eval<UNIT, K, OBJ, PREC>(s, cs, cd, tab, t64, G, dd, a.D, red, part, tot, t0, T);
            if (ctl) ctl_after_eval(s, lane, a.tol);
            if (UNIT == UNIT_WARP) __syncwarp(); else __syncthreads();
            if (s.go != 0) break;
        }
        if (UNIT == UNIT_WARP) __syncwarp(); else __syncthreads();
    }
    const bool writer = (UNIT != UNIT_CLUSTER) || cgx::this_cluster().block_rank() == 0;
    if (writer) state_store(s, a.st + h, ld_id, ld_n);
    if (UNIT == UNIT_WARP) __syncwarp(); else __syncthreads();
}

// Shared-memory layout of the persistent kernel (dynamic).
struct SmLayout {
    size_t cta_sm, warp_sm, cta_cs, warp_cs, cta_cd, warp_cd, tab, tab64, red, part, tot, warp_tot, item, total;
};

// fp64: room for the tables of the FP64 functions (FP64 batches only).
__host__ __device__ inline SmLayout sm_layout(int nwarps, int nacc, bool fp64) {
    SmLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 15) / 16 * 16; return r; };
    L.cta_sm = take(sizeof(FitSm));
    L.warp_sm = take(sizeof(FitSm) * nwarps);
    L.cta_cs = take(sizeof(GP1Consts));
    L.warp_cs = take(sizeof(GP1Consts) * nwarps);
    L.cta_cd = take(sizeof(GP1Df));
    L.warp_cd = take(sizeof(GP1Df) * nwarps);
    L.tab = take(sizeof(DfTables));
    L.tab64 = take(fp64 ? sizeof(Fp64Tab) : 0);
    L.red = take(sizeof(double) * (nacc + 1) * kMaxWarpsPerCta);
    L.part = take(sizeof(double) * (nacc + 1));
    L.tot = take(sizeof(double) * (nacc + 1));
    L.warp_tot = take(sizeof(double) * (nacc + 1) * nwarps);
    L.item = take(16);
    L.total = o;
    return L;
}

// Persistent batched fit: clusters, then CTAs, then warps pop histograms.
template <int K, int OBJ, bool CLUSTERS, int PREC>
__global__ void __launch_bounds__(512) k_fit_persistent(FitArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int N = GP1Acc<K>::N;
    const int nw = blockDim.x >> 5;
    const SmLayout L = sm_layout(nw, N, PREC == CG_PREC_FP64);
    FitSm& cta_s = *reinterpret_cast<FitSm*>(smem + L.cta_sm);
    GP1Consts& cta_cs = *reinterpret_cast<GP1Consts*>(smem + L.cta_cs);
    double* red = reinterpret_cast<double*>(smem + L.red);
    double* part = reinterpret_cast<double*>(smem + L.part);
    double* tot = reinterpret_cast<double*>(smem + L.tot);
    int* item = reinterpret_cast<int*>(smem + L.item);
    GP1Df& cta_cd = *reinterpret_cast<GP1Df*>(smem + L.cta_cd);
    DfTables& tab = *reinterpret_cast<DfTables*>(smem + L.tab);
    const Fp64Tab* t64 = reinterpret_cast<const Fp64Tab*>(smem + L.tab64);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (PREC == CG_PREC_DF64) {
        df_tables_init(tab);
        __syncthreads();
    } else {
        fp64_tab_load(*reinterpret_cast<Fp64Tab*>(smem + L.tab64));
        __syncthreads();
    }

    const int n0 = a.n_items[0], n1 = a.n_items[1], n2 = a.n_items[2];
    if (CLUSTERS) {
        cgx::cluster_group cl = cgx::this_cluster();
        const int rank = (int)cl.block_rank();
        const int csz = (int)cl.num_blocks();
        for (;;) {
            if (rank == 0 && threadIdx.x == 0) *item = atomicAdd(&a.counters[0], 1);
            cl.sync();
            const int it = *cl.map_shared_rank(item, 0);
            cl.sync();
            if (it >= n0) break;
            unit_fit<UNIT_CLUSTER, K, OBJ, PREC>(a, a.queue[0][it], cta_s, cta_cs, cta_cd, tab, t64, red, part, tot,
                                                 rank * blockDim.x + threadIdx.x, csz * blockDim.x);
        }
    }
    for (;;) {
        if (threadIdx.x == 0) *item = atomicAdd(&a.counters[1], 1);
        __syncthreads();
        const int it = *item;
        __syncthreads();
        if (it >= n1) break;
        unit_fit<UNIT_CTA, K, OBJ, PREC>(a, a.queue[1][it], cta_s, cta_cs, cta_cd, tab, t64, red, part, tot, threadIdx.x,
                                         blockDim.x);
    }
    FitSm& ws_ = reinterpret_cast<FitSm*>(smem + L.warp_sm)[wid];
    GP1Consts& wcs = reinterpret_cast<GP1Consts*>(smem + L.warp_cs)[wid];
    GP1Df& wcd = reinterpret_cast<GP1Df*>(smem + L.warp_cd)[wid];
    double* wtot = reinterpret_cast<double*>(smem + L.warp_tot) + wid * (N + 1);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(&a.counters[2], 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n2) break;
        unit_fit<UNIT_WARP, K, OBJ, PREC>(a, a.queue[2][it], ws_, wcs, wcd, tab, t64, nullptr, nullptr, wtot, lane, 32);
    }
}

// Gauss-Newton matrix out[i * ld + j] (i, j < P) from the packed sums raw of
// h r_a r_b over the raw factors r: GN_ij = D_i D_j raw_ij, with the per-point
// scales D = (1, A/s^2, A/s^3) per peak and 1 per polynomial term.
template <int K>
__device__ void gn_scaled(const double* th, int P, const double* raw, double* out, int ld) {
    constexpr int R = GP1Gnm<K>::R;
    double dsc[FP];
    for (int k = 0; k < P; ++k) {
        dsc[k] = 1.0;
        if (k < 3 * K) {
            const int pk = k / 3, role = k - 3 * pk;
            const double A = th[3 * pk], sg = th[3 * pk + 2];
            if (role == 1) dsc[k] = A / (sg * sg);
            if (role == 2) dsc[k] = A / (sg * sg * sg);
        }
    }
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) {
            const int lo = i < j ? i : j, hi = i < j ? j : i;
            out[i * ld + j] = dsc[i] * dsc[j] * raw[lo * R - lo * (lo - 1) / 2 + (hi - lo)];
        }
}

// Init (GN + first evaluation) and plain evaluation: one CTA per histogram,
// taken from a.order through the counter a.ectr (largest first) or, without
// an order, grid-stride in index order.  mode 0: value/grad at a.theta; mode 1: init;
// mode 2: value only; mode 4: value, gradient and the full Gauss-Newton
// matrix [H][P][P] (df64 only).
template <int K, int OBJ, int PREC, int MODE>
__global__ void __launch_bounds__(256) k_fit_eval(FitArgs a) {
    constexpr int mode = MODE;
    constexpr int N = GP1Acc<K>::N;
    constexpr int NV = GP1Gnm<K>::NV;
    // warp_totals_f writes whole chunks of 32 accumulators (the tail past NV is zero)
    __shared__ double gmred[(MODE == 4 ? (NV + 31) / 32 * 32 : 1) * kMaxWarpsPerCta];
    __shared__ double gmtot[MODE == 4 ? NV : 1];
    __shared__ GP1Consts cs;
    __shared__ GP1Df cd;
    __shared__ DfTables tab;
    __shared__ int cs_bad;
    __shared__ typename std::conditional<PREC == CG_PREC_FP64, Fp64Tab, int>::type t64;
    if (PREC == CG_PREC_DF64) {
        df_tables_init(tab);
        __syncthreads();
    } else {
        if constexpr (PREC == CG_PREC_FP64) fp64_tab_load(t64);
        __syncthreads();
    }
    __shared__ double red[(N + 1) * kMaxWarpsPerCta];
    __shared__ double tot[N + 1];
    __shared__ double gn[N + 1];
    __shared__ double fdt[1];   // init, FP64: the value's counts-only part
    __shared__ int q_sh;
    for (int64_t it = blockIdx.x;; it += gridDim.x) {
        int64_t h;
        if (a.order) {   // dynamic queue, largest histograms first
            if (threadIdx.x == 0) q_sh = atomicAdd(a.ectr, 1);
            __syncthreads();
            const int q = q_sh;
            __syncthreads();
            if (q >= a.H) break;
            h = a.order[q];
            if (h < 0 || h >= a.H) continue;   // an order not written by a plan: skip, never index past H
        } else {
            if (it >= a.H) break;
            h = it;
        }
        const double* th = a.theta + h * (int64_t)a.P;
        const Geom G = geom_of(a, h);
        GP1Data dd;
        dd.y = G.y;
        dd.centres = nullptr;
        dd.lo = G.lo;
        dd.h = G.hw;
        dd.au = 2.0 / (a.hi[h] - a.lo[h]);
        dd.bu = -(a.lo[h] + a.hi[h]) / (a.hi[h] - a.lo[h]);
        dd.D = a.D;
        dd.pm = a.pm;
        dd.vec_ok = 0;
        if (threadIdx.x < 32) {
            const bool ok = gp1_prologue_warp<K, PREC == CG_PREC_DF64>(th, a.D, G.lo, G.hw, dd.au, dd.bu, cs, cd);
            if (threadIdx.x == 0) cs_bad = ok ? 0 : 1;
        }
        __syncthreads();
        bool bad = false;
        int any_bad;
        if (MODE == 4 && !(PREC == CG_PREC_DF64 && G.n < kDfMaxBins)) {
            // the Gauss-Newton matrix is taken on the df64 path only
            if (threadIdx.x == 0) a.value[h] = __longlong_as_double(0x7ff8000000000000LL);
            __syncthreads();
            continue;
        }
        if (PREC == CG_PREC_DF64 && G.n < kDfMaxBins) {
            // mode 1: gradient and Gauss-Newton terms in one sweep over the bins
            df v[N], gv[N];
            float gm[MODE == 4 ? NV : 1];
#pragma unroll
            for (int i = 0; i < (MODE == 4 ? NV : 1); ++i) gm[i] = 0.0f;
            acc_bins_df64<K, OBJ, MODE == 1, MODE == 2, MODE == 4>(G, cs, cd, dd, tab, threadIdx.x, blockDim.x, v,
                                                                  gv, bad, gm);
            any_bad = __syncthreads_or(bad) | cs_bad;
            if constexpr (MODE == 4) {
                warp_totals_f<NV>(gm, gmred + (threadIdx.x >> 5), kMaxWarpsPerCta);
                __syncthreads();
                for (int i = threadIdx.x; i < NV; i += blockDim.x) {
                    double sum = 0.0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += gmred[i * kMaxWarpsPerCta + w];
                    gmtot[i] = sum;
                }
                __syncthreads();
            }
            if constexpr (MODE == 2) {
                const df v0[1] = {v[0]};
                reduce_cta<1, df>(v0, red, tot);
            } else {
                reduce_cta<N, df>(v, red, tot);
            }
            if constexpr (MODE == 1) reduce_cta<N, df>(gv, red, gn);
        } else {
            double acc[N], gacc[N];
#pragma unroll
            for (int i = 0; i < N; ++i) acc[i] = gacc[i] = 0.0;
            if constexpr (PREC == CG_PREC_FP64) {
                if constexpr (MODE == 1) {   // init: the counts-only part once, into the fit state
                    acc_bins_f64<K, OBJ, false>(G, cs, dd, t64, threadIdx.x, blockDim.x, acc, bad);
                    const double fd[1] = {data_part_f64<OBJ>(G, t64, threadIdx.x, blockDim.x)};
                    reduce_cta<1, double>(fd, red, fdt);
                } else {
                    acc_bins_f64<K, OBJ>(G, cs, dd, t64, threadIdx.x, blockDim.x, acc, bad);
                }
            } else {
                acc_bins<K, OBJ>(G, cs, dd, threadIdx.x, blockDim.x, acc, bad);
            }
            if constexpr (MODE == 1) gn_bins<K, OBJ>(G, cs, dd, threadIdx.x, blockDim.x, gacc);
            any_bad = __syncthreads_or(bad) | cs_bad;
            if constexpr (MODE == 2) {
                const double v0[1] = {acc[0]};
                reduce_cta<1, double>(v0, red, tot);
            } else {
                reduce_cta<N, double>(acc, red, tot);
            }
            if constexpr (MODE == 1) reduce_cta<N, double>(gacc, red, gn);
        }
        if (threadIdx.x == 0) {
            EpiParams ep;
            ep.model = CG_MODEL_GAUSS_POLY;
            ep.K = K;
            ep.D = a.D;
            ep.P = a.P;
            ep.lo = ep.hi = 0.0;
            double g[kMaxParams];
            if (mode == 2) {
                a.value[h] = any_bad ? __longlong_as_double(0x7ff8000000000000LL) : tot[0];
            } else if (mode == 4) {
                // value, gradient and GN = D (sum h r r^T) D with the per-point scales D
                const double v = epilogue(ep, th, tot, g);
                a.value[h] = any_bad ? __longlong_as_double(0x7ff8000000000000LL) : v;
                const int P = a.P;
                for (int k = 0; k < P; ++k) a.grad[h * P + k] = g[k];
                gn_scaled<K>(th, P, gmtot, a.gn + h * P * P, P);
            } else if (mode == 0) {
                const double v = epilogue(ep, th, tot, g);
                a.value[h] = v;
                for (int k = 0; k < a.P; ++k) a.grad[h * a.P + k] = g[k];
                if (any_bad) a.value[h] = __longlong_as_double(0x7ff8000000000000LL);
            } else {
                const double v = epilogue(ep, th, tot, g);
                cg_fit_state* st = a.st + h;
                // GN diagonal from its accumulators
                double gd[FP];
                for (int k = 0; k < K; ++k) {
                    const double A = th[3 * k], s = th[3 * k + 2];
                    gd[3 * k] = gn[1 + 3 * k];
                    gd[3 * k + 1] = (A / (s * s)) * (A / (s * s)) * gn[2 + 3 * k];
                    gd[3 * k + 2] = (A / (s * s * s)) * (A / (s * s * s)) * gn[3 + 3 * k];
                }
                for (int j = 0; j <= a.D; ++j) gd[3 * K + j] = gn[1 + 3 * K + j];
                double edm = 0.0;
                for (int k = 0; k < FP; ++k) {
                    const bool in = k < a.P;
                    const double h0 = in ? ((gd[k] > 0.0) ? 1.0 / gd[k] : 1.0) : 0.0;
                    st->theta[k] = in ? th[k] : 0.0;
                    st->grad[k] = in ? g[k] : 0.0;
                    st->h0[k] = h0;
                    for (int j = 0; j < FP; ++j) st->hinv[k * FP + j] = (j == k) ? h0 : 0.0;
                    if (in) edm = fma(g[k] * h0, g[k], edm);
                }
                const double fdata = (PREC == CG_PREC_FP64) ? fdt[0] : 0.0;
                st->f = v + fdata;
                st->fdata = fdata;
                st->edm = 0.5 * edm;
                st->iter = 0;
                st->n_eval = 1;
                st->n_params = a.P;
                st->status = (any_bad || !isfinite(v)) ? CG_FIT_DOMAIN : CG_FIT_RUNNING;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Levenberg-Marquardt fits.  The plan cuts every histogram into tiles of at
// most kLmTile bins (histograms by decreasing size, a histogram's tiles
// consecutive).  One step is two launches:
//  k_lm_tiles: resident CTAs take tiles from a counter; for a tile of a
//    RUNNING fit, the df64 value / gradient accumulators, a domain flag and
//    the FP32 Gauss-Newton products of its bins at the trial point, summed
//    over the CTA into one partial row;
//  k_lm_finish: one warp per histogram sums its tiles' rows in tile order
//    (deterministic, no atomics on values), applies the epilogue (value,
//    gradient, GN with the per-point scales) and runs the control on lane 0.
// Control: accept the trial when F(trial) < F (theta, F, g, GN move there,
// lambda / 10 down to 1e-12, iteration + 1, EDM = g^T GN^-1 g / 2 with the
// undamped matrix; converged when EDM < tol max(1, |F|)); otherwise
// lambda x 10 (CG_FIT_LINESEARCH_FAILED past 1e16); then the next trial
// theta + delta, (GN + lambda diag(GN)) delta = -g by Cholesky (diag(GN)
// entries <= 0 count as 1; a scaled gradient step where the damped matrix is
// not positive definite).  State reuse: hinv holds GN at theta, h0[0] lambda.
// ---------------------------------------------------------------------------
constexpr int kLmTile = 16384;
constexpr int kLmMagic = 0x4c4d5431;

struct LmHdr {
    int ectr;      // tile queue position (zeroed by the plan, init and every k_lm_finish)
    int n_tiles;
    int magic;     // kLmMagic once a plan has been written
    int pad;
};

template <int K>
struct LmRow {
    static constexpr int N = GP1Acc<K>::N, NV = GP1Gnm<K>::NV, NP = N + 1 + NV;
};

__host__ __device__ inline size_t lm_align(size_t x) { return (x + 255) & ~(size_t)255; }

// Partial rows follow the tile list: the address depends on the tile count.
__device__ inline double* lm_part(const FitArgs& a, int n_tiles) {
    return (double*)((char*)a.tiles + lm_align(sizeof(int2) * (size_t)n_tiles));
}

// Tile count from the plan header, or -1 when no plan of this size is there.
template <int K>
__device__ inline int lm_tiles_checked(const FitArgs& a) {
    const LmHdr* hd = (const LmHdr*)a.lm_hdr;
    const int T = hd->n_tiles;
    if (hd->magic != kLmMagic || T < 1) return -1;
    const size_t end = (size_t)((const char*)lm_part(a, T) - (const char*)a.lm_hdr) +
                       sizeof(double) * (size_t)T * LmRow<K>::NP;
    return end <= a.ws_bytes ? T : -1;
}

// Warp-parallel dense algebra for the control: lane i < P holds row i of a
// P x P matrix (or component i of a vector) in registers; loops run over the
// compile-time bound FP so that every register index is static.
__device__ __forceinline__ double lane_bcast(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Cholesky factorisation in place: on success lane i holds row i of L
// (m[0..i]).  The result is the same on every lane (false: not positive
// definite).
__device__ __forceinline__ bool chol_warp(double (&m)[FP], int P, int lane) {
#pragma unroll
    for (int j = 0; j < FP; ++j) {
        if (j >= P) break;
        const double ajj = lane_bcast(m[j], j);
        if (!(ajj > 0.0)) return false;
        const double ljj = sqrt(ajj);
        if (lane == j) m[j] = ljj;
        else if (lane > j) m[j] = m[j] / ljj;
#pragma unroll
        for (int k = j + 1; k < FP; ++k) {
            if (k >= P) break;
            const double lkj = lane_bcast(m[j], k);
            if (lane >= k) m[k] = fma(-m[j], lkj, m[k]);
        }
    }
    return true;
}

// x = (L L^T)^-1 b with L from chol_warp; b and x one component per lane.
__device__ __forceinline__ double chol_solve_warp(const double (&l)[FP], double b, int P, int lane) {
    double r = b, y = 0.0;
#pragma unroll
    for (int j = 0; j < FP; ++j) {   // L y = b, column by column
        if (j >= P) break;
        const double yj = lane_bcast(r / l[j], j);
        if (lane == j) y = yj;
        if (lane > j) r = fma(-l[j], yj, r);
    }
    double x = 0.0;
#pragma unroll
    for (int j = FP - 1; j >= 0; --j) {   // L^T x = y, row j from the lanes below it
        if (j >= P) continue;
        const double sj = warp_sum((lane > j && lane < P) ? l[j] * x : 0.0);
        if (lane == j) x = (y - sj) / l[j];
    }
    return x;
}

// Row i of the Gauss-Newton matrix from the packed sums raw (per-point
// scales D = 1, A/s^2, A/s^3 per peak, 1 per polynomial term); zero past P.
template <int K>
__device__ __forceinline__ void gn_row(const double* th, int P, const double* raw, int i, double (&row)[FP]) {
    constexpr int R = GP1Gnm<K>::R;
    auto dsc = [&](int k) -> double {
        if (k < 3 * K) {
            const int pk = k / 3, role = k - 3 * pk;
            const double A = th[3 * pk], sg = th[3 * pk + 2];
            return role == 0 ? 1.0 : (role == 1 ? A / (sg * sg) : A / (sg * sg * sg));
        }
        return 1.0;
    };
    const double di = i < P ? dsc(i) : 0.0;
#pragma unroll
    for (int j = 0; j < FP; ++j) {
        if (i < P && j < P) {
            const int lo = i < j ? i : j, hi = i < j ? j : i;
            row[j] = di * dsc(j) * raw[lo * R - lo * (lo - 1) / 2 + (hi - lo)];
        } else {
            row[j] = 0.0;
        }
    }
}

// The control of one fit, all 32 lanes of a warp, after the evaluation of
// its trial point tt (value ft, uniform; gradient component g_l and GN row G
// of this lane); writes the next trial point into tt.
__device__ void lm_control_warp(cg_fit_state& s, double* tt, double ft, double g_l, const double (&G)[FP], int P,
                                double tol, bool first, int lane) {
    const bool own = lane < P;
    double lam = first ? 1e-3 : s.h0[0];
    const double f_old = first ? 0.0 : s.f;
    int status = first ? CG_FIT_RUNNING : s.status;
    const int iter = first ? 0 : s.iter;
    const int n_eval = first ? 1 : s.n_eval + 1;
    bool accept;
    if (first) {
        accept = isfinite(ft);
        if (!accept) status = CG_FIT_DOMAIN;
    } else {
        accept = isfinite(ft) && ft < f_old;
        if (accept) {
            lam = fmax(lam * 0.1, 1e-12);
        } else {
            lam *= 10.0;
            if (lam > 1e16) status = CG_FIT_LINESEARCH_FAILED;
        }
    }
    // the Gauss-Newton matrix and gradient at theta (this lane's row / component);
    // the start point is kept also when its value is not finite
    const bool use_trial = accept || first;
    double row[FP], gth, th_l;
    const double tt_l = lane < FP ? tt[lane] : 0.0;
    if (use_trial) {
#pragma unroll
        for (int j = 0; j < FP; ++j) row[j] = G[j];
        gth = own ? g_l : 0.0;
        th_l = own ? tt_l : 0.0;
    } else {
#pragma unroll
        for (int j = 0; j < FP; ++j) row[j] = (own && j < P) ? s.hinv[lane * FP + j] : 0.0;
        gth = own ? s.grad[lane] : 0.0;
        th_l = own ? s.theta[lane] : 0.0;
    }
    double dg = 0.0;
#pragma unroll
    for (int j = 0; j < FP; ++j)
        if (j == lane) dg = row[j];
    const double dpos = dg > 0.0 ? dg : 1.0;
    double edm = first ? 0.0 : s.edm;
    if (accept) {
        double m[FP];
#pragma unroll
        for (int j = 0; j < FP; ++j) m[j] = row[j];
        double e;
        if (chol_warp(m, P, lane)) {
            const double z = chol_solve_warp(m, gth, P, lane);
            e = warp_sum(own ? gth * z : 0.0);
        } else {
            e = warp_sum(own ? gth * gth / dpos : 0.0);
        }
        edm = 0.5 * e;
        if (status == CG_FIT_RUNNING && edm < tol * fmax(1.0, fabs(ft))) status = CG_FIT_CONVERGED;
    }
    __syncwarp();   // every lane has read the old state
    if (use_trial && lane < FP) {
        s.theta[lane] = th_l;
        s.grad[lane] = gth;
#pragma unroll
        for (int j = 0; j < FP; ++j) s.hinv[lane * FP + j] = row[j];
        s.h0[lane] = 0.0;
    }
    __syncwarp();
    if (lane == 0) {
        if (use_trial) s.f = ft;
        s.h0[0] = lam;
        s.edm = edm;
        s.iter = iter + ((accept && !first) ? 1 : 0);
        s.n_eval = n_eval;
        s.n_params = P;
        s.status = status;
    }
    if (status != CG_FIT_RUNNING) return;
    // next trial: (GN + lambda diag(GN)) delta = -g, diagonal entries <= 0 counting as 1
    double m[FP];
#pragma unroll
    for (int j = 0; j < FP; ++j) m[j] = row[j] + ((j == lane) ? lam * dpos : 0.0);
    double d;
    if (chol_warp(m, P, lane)) d = chol_solve_warp(m, -gth, P, lane);
    else d = -gth / ((1.0 + lam) * dpos);
    if (lane < FP) tt[lane] = own ? th_l + d : 0.0;
}

__global__ void k_lm_reset(cg_fit_state* st, int64_t H, int P) {
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    st[h].status = CG_FIT_RUNNING;
    st[h].n_params = P;
    st[h].fdata = 0.0;   // the Levenberg-Marquardt evaluations include the counts-only part
}

template <int K, int OBJ>
__global__ void __launch_bounds__(256) k_lm_tiles(FitArgs a) {
    constexpr int N = LmRow<K>::N, NV = LmRow<K>::NV, NP = LmRow<K>::NP;
    __shared__ double gmred[(NV + 31) / 32 * 32 * kMaxWarpsPerCta];
    __shared__ double red[(N + 1) * kMaxWarpsPerCta];
    __shared__ double tot[N + 1];
    __shared__ GP1Consts cs;
    __shared__ GP1Df cd;
    __shared__ DfTables tab;
    __shared__ int cs_bad, q_sh;
    const int T = lm_tiles_checked<K>(a);
    if (T < 0) return;   // no plan in this workspace: nothing is read or written
    double* part = lm_part(a, T);
    df_tables_init(tab);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) q_sh = atomicAdd(a.ectr, 1);
        __syncthreads();
        const int q = q_sh;
        __syncthreads();
        if (q >= T) break;
        const int2 tl = a.tiles[q];
        const int64_t h = tl.x;
        if (h < 0 || h >= a.H || a.st[h].status != CG_FIT_RUNNING) continue;   // uniform per block
        double* out = part + (size_t)q * NP;
        const Geom G = geom_of(a, h);
        const int64_t b0 = (int64_t)tl.y * kLmTile;
        if (G.n >= kDfMaxBins || tl.y < 0 || (b0 >= G.n && b0 > 0)) {
            // the df64 bin loop needs exact float bin indices: no value for this fit
            for (int v = threadIdx.x; v < NP; v += blockDim.x) out[v] = (v == N) ? 1.0 : 0.0;
            continue;
        }
        const double* th = a.theta + h * FP;
        GP1Data dd;
        dd.y = G.y;
        dd.centres = nullptr;
        dd.lo = G.lo;
        dd.h = G.hw;
        dd.au = 2.0 / (a.hi[h] - a.lo[h]);
        dd.bu = -(a.lo[h] + a.hi[h]) / (a.hi[h] - a.lo[h]);
        dd.D = a.D;
        dd.pm = a.pm;
        dd.vec_ok = 0;
        if (threadIdx.x < 32) {
            const bool ok = gp1_prologue_warp<K, true>(th, a.D, G.lo, G.hw, dd.au, dd.bu, cs, cd);
            if (threadIdx.x == 0) cs_bad = ok ? 0 : 1;
        }
        __syncthreads();
        Geom Gt = G;
        Gt.n = G.n < b0 + kLmTile ? G.n : b0 + kLmTile;
        df v[N], gv[N];
        float gm[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) gm[i] = 0.0f;
        bool bad = false;
        acc_bins_df64<K, OBJ, false, false, true>(Gt, cs, cd, dd, tab, (int)b0 + threadIdx.x, blockDim.x, v, gv,
                                                  bad, gm);
        const int any_bad = __syncthreads_or(bad) | cs_bad;
        warp_totals_f<NV>(gm, gmred + (threadIdx.x >> 5), kMaxWarpsPerCta);
        reduce_cta<N, df>(v, red, tot);   // its barriers also order the gmred writes
        const int nw = blockDim.x >> 5;
        for (int i = threadIdx.x; i < NV; i += blockDim.x) {
            double sum = 0.0;
            for (int w = 0; w < nw; ++w) sum += gmred[i * kMaxWarpsPerCta + w];
            out[N + 1 + i] = sum;
        }
        for (int i = threadIdx.x; i < N; i += blockDim.x) out[i] = tot[i];
        if (threadIdx.x == 0) out[N] = any_bad ? 1.0 : 0.0;
        __syncthreads();
    }
}

template <int K, int OBJ>
__global__ void __launch_bounds__(128) k_lm_finish(FitArgs a, int first) {
    constexpr int N = LmRow<K>::N, NP = LmRow<K>::NP;
    __shared__ double sums[4][NP];
    __shared__ double gsh[4][FP];
    __shared__ double fsh[4];
    if (blockIdx.x == 0 && threadIdx.x == 0) ((LmHdr*)a.lm_hdr)->ectr = 0;   // for the next tile launch
    const int T = lm_tiles_checked<K>(a);
    if (T < 0) return;
    const double* part = lm_part(a, T);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t h = (int64_t)blockIdx.x * 4 + w;
    if (h >= a.H) return;
    cg_fit_state& s = a.st[h];
    if (s.status != CG_FIT_RUNNING) return;
    const int2 span = a.hspan[h];
    if (span.x < 0 || span.y < 1 || span.x + span.y > T) return;
    double* sm = sums[w];
    for (int v = lane; v < NP; v += 32) {
        double acc = 0.0;
        for (int t = 0; t < span.y; ++t) acc += part[(size_t)(span.x + t) * NP + v];
        sm[v] = acc;
    }
    __syncwarp();
    double* tt = (double*)a.theta + h * FP;
    if (lane == 0) {
        EpiParams ep;
        ep.model = CG_MODEL_GAUSS_POLY;
        ep.K = K;
        ep.D = a.D;
        ep.P = a.P;
        ep.lo = ep.hi = 0.0;
        double g[kMaxParams];
        const double v = epilogue(ep, tt, sm, g);
        fsh[w] = (sm[N] != 0.0) ? __longlong_as_double(0x7ff8000000000000LL) : v;
        for (int k = 0; k < a.P; ++k) gsh[w][k] = g[k];
    }
    __syncwarp();
    double G[FP];
    gn_row<K>(tt, a.P, sm + N + 1, lane, G);
    lm_control_warp(s, tt, fsh[w], lane < a.P ? gsh[w][lane] : 0.0, G, a.P, a.tol, first != 0, lane);
}

template <int K, int OBJ>
static cg_status lm_launch_k(const FitArgs& a, int first, bool tiles, cudaStream_t st) {
    if (tiles) {
        const int occ = resident_blocks((const void*)k_lm_tiles<K, OBJ>, 256, 0);
        k_lm_tiles<K, OBJ><<<device_sm_count() * occ, 256, 0, st>>>(a);
    } else {
        k_lm_finish<K, OBJ><<<(unsigned)((a.H + 3) / 4), 128, 0, st>>>(a, first);
    }
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

static cg_status lm_launch(const cg_batch* b, const FitArgs& a, int first, bool tiles, cudaStream_t st) {
    const int K = b->tmpl.n_peaks, O = b->tmpl.objective;
#define CG_LM_CASE(KK, OO) if (K == KK && O == OO) return lm_launch_k<KK, OO>(a, first, tiles, st);
    CG_LM_CASE(1, CG_OBJ_CHI2) CG_LM_CASE(1, CG_OBJ_POISSON) CG_LM_CASE(1, CG_OBJ_POISSON_BC)
    CG_LM_CASE(2, CG_OBJ_CHI2) CG_LM_CASE(2, CG_OBJ_POISSON) CG_LM_CASE(2, CG_OBJ_POISSON_BC)
    CG_LM_CASE(3, CG_OBJ_CHI2) CG_LM_CASE(3, CG_OBJ_POISSON) CG_LM_CASE(3, CG_OBJ_POISSON_BC)
#undef CG_LM_CASE
    return CG_ERR_UNSUPPORTED;
}

// ---------------------------------------------------------------------------
// Plain per-histogram path: control kernel around full-GPU evaluations.
// ---------------------------------------------------------------------------
struct SingleWs {        // lives in the workspace
    FitSm s;
    double ft;           // written by the gradient launch
    double gt[FP];
    int need_eval;       // gate of the gradient launch
    int pending;         // an evaluation at s.tt has been requested
    int fresh;           // set by init: load the fit state on the next control step
    int64_t offsets[2];
    double lo, hi;
};

// One warp: consume the pending evaluation (if any), then request the next one.
__global__ void k_single_ctl(SingleWs* w, cg_fit_state* st, double tol) {
    __shared__ FitSm s;
    const int lane = threadIdx.x;
    const int fresh = w->fresh;
    const int pending = fresh ? 0 : w->pending;
    if (fresh) {
        state_load(s, st, lane, 32);
        __syncwarp();
        if (lane == 0 && s.status == CG_FIT_RUNNING && s.edm < tol * fmax(1.0, fabs(s.f)))
            s.status = CG_FIT_CONVERGED;
    } else {
        const double* src = reinterpret_cast<const double*>(&w->s);
        double* dst = reinterpret_cast<double*>(&s);
        for (int k = lane; k < (int)(sizeof(FitSm) / sizeof(double)); k += 32) dst[k] = src[k];
    }
    __syncwarp();
    bool need_dir = true;
    if (pending && s.status == CG_FIT_RUNNING) {
        if (lane < s.P) s.gt[lane] = w->gt[lane];
        if (lane == 0) {
            s.ft = w->ft;
            s.bad = !isfinite(w->ft);
        }
        __syncwarp();
        ctl_after_eval(s, lane, tol);
        need_dir = (s.go != 0);
    }
    __syncwarp();
    if (need_dir && s.status == CG_FIT_RUNNING) ctl_direction(s, lane);
    __syncwarp();
    if (lane == 0) {
        w->fresh = 0;
        w->pending = (s.status == CG_FIT_RUNNING) ? 1 : 0;
        w->need_eval = w->pending;
    }
    const double* src = reinterpret_cast<const double*>(&s);
    double* dst = reinterpret_cast<double*>(&w->s);
    for (int k = lane; k < (int)(sizeof(FitSm) / sizeof(double)); k += 32) dst[k] = src[k];
    state_store(s, st, lane, 32);
}

__global__ void k_single_setup(SingleWs* w, int64_t n, double lo, double hi) {
    w->offsets[0] = 0;
    w->offsets[1] = n;
    w->lo = lo;
    w->hi = hi;
    w->pending = 0;
    w->need_eval = 0;
    w->fresh = 1;
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
struct FitWsLayout {
    size_t hdr, counters, qmeta, queues, order, total;
};

FitWsLayout fit_ws_layout(int64_t H) {
    FitWsLayout L;
    L.hdr = 0;
    L.counters = 256;
    L.qmeta = 512;
    L.queues = 768;
    L.order = L.queues + align_up((size_t)3 * H * sizeof(int), 256);
    L.total = L.order + align_up((size_t)H * sizeof(int), 256);
    return L;
}

bool fit_supported(const cg_problem* t) {
    return t->model == CG_MODEL_GAUSS_POLY && t->n_peaks >= 1 && t->n_peaks <= 3 && t->poly_degree >= -1 &&
           t->poly_degree <= 3 && 3 * t->n_peaks + t->poly_degree + 1 <= FP &&
           (t->objective == CG_OBJ_CHI2 || t->objective == CG_OBJ_POISSON || t->objective == CG_OBJ_POISSON_BC);
}

bool map_ok(const cg_tile_map* m) {
    return m && m->cta_threads >= 64 && m->cta_threads <= 512 && (m->cta_threads % 32) == 0 &&
           (m->cluster_size == 1 || m->cluster_size == 2 || m->cluster_size == 4 || m->cluster_size == 8) &&
           m->warp_max_bins >= 0 && m->cta_max_bins >= m->warp_max_bins;
}

FitArgs base_args(const cg_batch* b) {
    FitArgs a;
    memset(&a, 0, sizeof(a));
    a.data = b->tmpl.data;
    a.offsets = b->offsets;
    a.lo = b->lo;
    a.hi = b->hi;
    a.H = b->n_hist;
    a.D = b->tmpl.poly_degree;
    a.pm = b->tmpl.poly_mode;
    a.P = 3 * b->tmpl.n_peaks + b->tmpl.poly_degree + 1;
    return a;
}

template <int K, int OBJ>
cg_status launch_eval_k(const FitArgs& a, int mode, int prec, cudaStream_t st) {
    int G = device_sm_count() * 4;
    const bool df = prec == CG_PREC_DF64;
    if (a.order && df) {   // one wave of resident CTAs pulling from the queue
        // resident CTAs of 256 threads per SM (per device, cached)
        int occ = 4;
        if (mode == 1) occ = resident_blocks((const void*)k_fit_eval<K, OBJ, CG_PREC_DF64, 1>, 256, 0);
        else if (mode == 4) occ = resident_blocks((const void*)k_fit_eval<K, OBJ, CG_PREC_DF64, 4>, 256, 0);
        G = device_sm_count() * occ;
    }
    const int grid = (int)(a.H < G ? a.H : G);
    if (mode == 0) {
        if (df) k_fit_eval<K, OBJ, CG_PREC_DF64, 0><<<grid, 256, 0, st>>>(a);
        else k_fit_eval<K, OBJ, CG_PREC_FP64, 0><<<grid, 256, 0, st>>>(a);
    } else if (mode == 2) {
        if (df) k_fit_eval<K, OBJ, CG_PREC_DF64, 2><<<grid, 256, 0, st>>>(a);
        else k_fit_eval<K, OBJ, CG_PREC_FP64, 2><<<grid, 256, 0, st>>>(a);
    } else if (mode == 4) {
        if (!df) return CG_ERR_UNSUPPORTED;
        k_fit_eval<K, OBJ, CG_PREC_DF64, 4><<<grid, 256, 0, st>>>(a);
    } else {
        if (df) k_fit_eval<K, OBJ, CG_PREC_DF64, 1><<<grid, 256, 0, st>>>(a);
        else k_fit_eval<K, OBJ, CG_PREC_FP64, 1><<<grid, 256, 0, st>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status launch_eval(const cg_problem* t, const FitArgs& a, int mode, cudaStream_t st) {
    const int K = t->n_peaks, O = t->objective;
#define CG_EVAL_CASE(KK, OO) if (K == KK && O == OO) return launch_eval_k<KK, OO>(a, mode, t->precision, st);
    CG_EVAL_CASE(1, CG_OBJ_CHI2) CG_EVAL_CASE(1, CG_OBJ_POISSON) CG_EVAL_CASE(1, CG_OBJ_POISSON_BC)
    CG_EVAL_CASE(2, CG_OBJ_CHI2) CG_EVAL_CASE(2, CG_OBJ_POISSON) CG_EVAL_CASE(2, CG_OBJ_POISSON_BC)
    CG_EVAL_CASE(3, CG_OBJ_CHI2) CG_EVAL_CASE(3, CG_OBJ_POISSON) CG_EVAL_CASE(3, CG_OBJ_POISSON_BC)
#undef CG_EVAL_CASE
    return CG_ERR_UNSUPPORTED;
}

template <int K, int OBJ, bool CL, int PREC>
cg_status launch_persistent_k(const FitArgs& a, const cg_tile_map* m, cudaStream_t st) {
    constexpr int N = GP1Acc<K>::N;
    const int nt = m->cta_threads;
    const SmLayout L = sm_layout(nt / 32, N, PREC == CG_PREC_FP64);
    auto kern = k_fit_persistent<K, OBJ, CL, PREC>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total) != cudaSuccess)
        return CG_ERR_CUDA;
    const int csz = CL ? m->cluster_size : 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    int nattr = 0;
    if (CL) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = csz;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        nattr = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = nattr;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, L.total) != cudaSuccess || per_sm < 1)
        return CG_ERR_UNSUPPORTED;
    int grid = device_sm_count() * per_sm;
    if (CL) {
        cfg.gridDim = dim3(csz);
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) return CG_ERR_UNSUPPORTED;
        grid = ncl * csz;
    }
    cfg.gridDim = dim3(grid);
    prof_begin(st);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
    prof_end(st);
    return e == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status launch_persistent(const cg_problem* t, const FitArgs& a, const cg_tile_map* m, cudaStream_t st) {
    const int K = t->n_peaks, O = t->objective;
    const bool CL = m->cluster_size > 1;
    const bool DF = t->precision == CG_PREC_DF64;
#define CG_P_CASE(KK, OO)                                                                                  \
    if (K == KK && O == OO) {                                                                              \
        if (DF) return CL ? launch_persistent_k<KK, OO, true, CG_PREC_DF64>(a, m, st)                      \
                          : launch_persistent_k<KK, OO, false, CG_PREC_DF64>(a, m, st);                     \
        return CL ? launch_persistent_k<KK, OO, true, CG_PREC_FP64>(a, m, st)                              \
                  : launch_persistent_k<KK, OO, false, CG_PREC_FP64>(a, m, st);                             \
    }
    CG_P_CASE(1, CG_OBJ_CHI2) CG_P_CASE(1, CG_OBJ_POISSON) CG_P_CASE(1, CG_OBJ_POISSON_BC)
    CG_P_CASE(2, CG_OBJ_CHI2) CG_P_CASE(2, CG_OBJ_POISSON) CG_P_CASE(2, CG_OBJ_POISSON_BC)
    CG_P_CASE(3, CG_OBJ_CHI2) CG_P_CASE(3, CG_OBJ_POISSON) CG_P_CASE(3, CG_OBJ_POISSON_BC)
#undef CG_P_CASE
    return CG_ERR_UNSUPPORTED;
}

struct QueueMeta {
    int n_items[3];
    int cluster_size;
};
static_assert(sizeof(FitSm) % sizeof(double) == 0, "FitSm is copied as doubles");

cg_status batch_checks(const cg_batch* b, void* ws, size_t ws_bytes) {
    if (!b || b->n_hist < 1 || !b->offsets || !b->lo || !b->hi || !b->tmpl.data) return CG_ERR_INVALID_ARG;
    if (b->n_hist > (int64_t)1 << 30) return CG_ERR_INVALID_ARG;
    if (!fit_supported(&b->tmpl)) return CG_ERR_UNSUPPORTED;
    if (b->tmpl.precision != CG_PREC_FP64 && b->tmpl.precision != CG_PREC_DF64) return CG_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < fit_ws_layout(b->n_hist).total) return CG_ERR_WORKSPACE;
    return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" {

size_t cg_batch_workspace_size(const cg_batch* b) {
    if (!b || b->n_hist < 1) return 0;
    if (!b->offsets) return grad_workspace_bytes(&b->tmpl, b->n_hist);
    if (!fit_supported(&b->tmpl)) return 0;
    return 256;
}

cg_status cg_batch_gradient(const cg_batch* b, const double* theta, double* value, double* grad, void* ws,
                            size_t ws_bytes, void* stream) {
    if (!b || b->n_hist < 1) return CG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->offsets) return grad_points(&b->tmpl, theta, b->n_hist, value, grad, ws, ws_bytes, st, nullptr);
    if (!theta || !value || !b->lo || !b->hi || !b->tmpl.data) return CG_ERR_INVALID_ARG;
    if (!fit_supported(&b->tmpl)) return CG_ERR_UNSUPPORTED;
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < 256) return CG_ERR_WORKSPACE;
    FitArgs a = base_args(b);
    a.theta = theta;
    a.value = value;
    a.grad = grad;
    return launch_eval(&b->tmpl, a, grad ? 0 : 2, st);   // grad == NULL: values only
}

// Levenberg-Marquardt workspace: plan header, trial points [H][FP], tile
// spans [H], then the tile list [T] and the partial rows [T][NP].
struct LmWs {
    size_t hdr, th, hspan, tiles, total;
};
static int lm_row_doubles(int K) { return (1 + 3 * K + 4) + 1 + (3 * K + 4) * (3 * K + 5) / 2; }
static LmWs lm_ws_layout(int64_t H, int64_t T, int K) {
    LmWs L;
    L.hdr = 0;
    L.th = 256;
    L.hspan = L.th + lm_align(sizeof(double) * (size_t)H * FP);
    L.tiles = L.hspan + lm_align(sizeof(int2) * (size_t)H);
    L.total = L.tiles + lm_align(sizeof(int2) * (size_t)T) + sizeof(double) * (size_t)T * lm_row_doubles(K);
    return L;
}
// Tiles of a batch (-1 when an offset is decreasing or the count leaves int).
static int64_t lm_tile_count(const int64_t* ho, int64_t H) {
    int64_t T = 0;
    for (int64_t h = 0; h < H; ++h) {
        const int64_t n = ho[h + 1] - ho[h];
        if (n < 0) return -1;
        T += n > 0 ? (n + kLmTile - 1) / kLmTile : 1;
    }
    return T < INT32_MAX ? T : -1;
}
static bool lm_batch_ok(const cg_batch* b) {
    return b && b->n_hist >= 1 && b->n_hist <= ((int64_t)1 << 30) && b->offsets && b->lo && b->hi &&
           b->tmpl.data && fit_supported(&b->tmpl) && b->tmpl.precision == CG_PREC_DF64;
}

size_t cg_fit_lm_workspace_size(const cg_batch* b, const int64_t* host_offsets) {
    if (!lm_batch_ok(b) || !host_offsets) return 0;
    const int64_t T = lm_tile_count(host_offsets, b->n_hist);
    if (T < 1) return 0;
    return lm_ws_layout(b->n_hist, T, b->tmpl.n_peaks).total;
}

cg_status cg_fit_lm_plan(const cg_batch* b, const int64_t* host_offsets, void* ws, size_t ws_bytes, void* stream) {
    if (!b || !host_offsets) return CG_ERR_INVALID_ARG;
    if (!lm_batch_ok(b)) return fit_supported(&b->tmpl) ? CG_ERR_UNSUPPORTED : CG_ERR_INVALID_ARG;
    const int64_t H = b->n_hist;
    const int64_t T = lm_tile_count(host_offsets, H);
    if (T < 1) return CG_ERR_INVALID_ARG;
    const LmWs L = lm_ws_layout(H, T, b->tmpl.n_peaks);
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < L.total) return CG_ERR_WORKSPACE;
    std::vector<std::pair<int64_t, int>> by_size((size_t)H);
    for (int64_t h = 0; h < H; ++h) by_size[(size_t)h] = {host_offsets[h + 1] - host_offsets[h], (int)h};
    std::stable_sort(by_size.begin(), by_size.end(),
                     [](const std::pair<int64_t, int>& x, const std::pair<int64_t, int>& y) { return x.first > y.first; });
    std::vector<int2> tiles;
    tiles.reserve((size_t)T);
    std::vector<int2> span((size_t)H);
    for (auto& e : by_size) {
        const int nt = e.first > 0 ? (int)((e.first + kLmTile - 1) / kLmTile) : 1;
        span[(size_t)e.second] = make_int2((int)tiles.size(), nt);
        for (int j = 0; j < nt; ++j) tiles.push_back(make_int2(e.second, j));
    }
    LmHdr hd;
    hd.ectr = 0;
    hd.n_tiles = (int)T;
    hd.magic = kLmMagic;
    hd.pad = 0;
    char* base = (char*)ws;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(base + L.tiles, tiles.data(), tiles.size() * sizeof(int2), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.hspan, span.data(), span.size() * sizeof(int2), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.hdr, &hd, sizeof(hd), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return CG_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_batch_gn(const cg_batch* b, const double* theta, double* value, double* grad, double* gn, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!b || b->n_hist < 1 || !b->offsets || !theta || !value || !grad || !gn || !b->lo || !b->hi ||
        !b->tmpl.data)
        return CG_ERR_INVALID_ARG;
    if (!fit_supported(&b->tmpl)) return CG_ERR_UNSUPPORTED;
    if (b->tmpl.precision != CG_PREC_DF64) return CG_ERR_UNSUPPORTED;
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < 256) return CG_ERR_WORKSPACE;
    FitArgs a = base_args(b);
    a.theta = theta;
    a.value = value;
    a.grad = grad;
    a.gn = gn;
    return launch_eval(&b->tmpl, a, 4, (cudaStream_t)stream);
}

static FitArgs lm_args(const cg_batch* b, cg_fit_state* state, double tol, void* ws, size_t ws_bytes) {
    const LmWs L = lm_ws_layout(b->n_hist, 0, b->tmpl.n_peaks);
    char* base = (char*)ws;
    FitArgs a = base_args(b);
    a.st = state;
    a.tol = tol;
    a.theta = (const double*)(base + L.th);
    a.lm_hdr = base + L.hdr;
    a.ectr = (int*)(base + L.hdr);   // LmHdr::ectr
    a.hspan = (const int2*)(base + L.hspan);
    a.tiles = (const int2*)(base + L.tiles);
    a.ws_bytes = ws_bytes;
    return a;
}

static cg_status lm_checks(const cg_batch* b, cg_fit_state* state, double tol, void* ws, size_t ws_bytes) {
    if (!b || !state || !(tol >= 0.0)) return CG_ERR_INVALID_ARG;
    if (!lm_batch_ok(b)) return fit_supported(&b->tmpl) ? CG_ERR_UNSUPPORTED : CG_ERR_INVALID_ARG;
    // the tile part's size is known to the plan only; the kernels check it against ws_bytes
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < lm_ws_layout(b->n_hist, 1, b->tmpl.n_peaks).total)
        return CG_ERR_WORKSPACE;
    return CG_OK;
}

cg_status cg_fit_lm_init(const cg_batch* b, const double* theta0, cg_fit_state* state, double tol, void* ws,
                         size_t ws_bytes, void* stream) {
    cg_status s = lm_checks(b, state, tol, ws, ws_bytes);
    if (s != CG_OK) return s;
    if (!theta0) return CG_ERR_INVALID_ARG;
    const FitArgs a = lm_args(b, state, tol, ws, ws_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    const int P = a.P;
    double* th = (double*)a.theta;
    if (cudaMemsetAsync(th, 0, sizeof(double) * (size_t)b->n_hist * FP, st) != cudaSuccess ||
        cudaMemcpy2DAsync(th, sizeof(double) * FP, theta0, sizeof(double) * P, sizeof(double) * P,
                          (size_t)b->n_hist, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(a.ectr, 0, sizeof(int), st) != cudaSuccess)
        return CG_ERR_CUDA;
    k_lm_reset<<<(unsigned)((b->n_hist + 255) / 256), 256, 0, st>>>(state, b->n_hist, P);
    if (cudaGetLastError() != cudaSuccess) return CG_ERR_CUDA;
    s = lm_launch(b, a, 1, true, st);
    if (s != CG_OK) return s;
    return lm_launch(b, a, 1, false, st);
}

cg_status cg_fit_lm_step(const cg_batch* b, cg_fit_state* state, int n_steps, double tol, void* ws, size_t ws_bytes,
                         void* stream) {
    cg_status s = lm_checks(b, state, tol, ws, ws_bytes);
    if (s != CG_OK) return s;
    if (n_steps < 0) return CG_ERR_INVALID_ARG;
    const FitArgs a = lm_args(b, state, tol, ws, ws_bytes);
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n_steps; ++i) {
        s = lm_launch(b, a, 0, true, st);
        if (s != CG_OK) return s;
        s = lm_launch(b, a, 0, false, st);
        if (s != CG_OK) return s;
    }
    return CG_OK;
}

size_t cg_fit_workspace_size(const cg_batch* b) {
    if (!b || b->n_hist < 1 || !b->offsets || !fit_supported(&b->tmpl)) return 0;
    return fit_ws_layout(b->n_hist).total;
}

cg_status cg_fit_plan(const cg_batch* b, const int64_t* host_offsets, const cg_tile_map* map, void* ws,
                      size_t ws_bytes, void* stream) {
    cg_status s = batch_checks(b, ws, ws_bytes);
    if (s != CG_OK) return s;
    if (!host_offsets || !map_ok(map)) return CG_ERR_INVALID_ARG;
    const int64_t H = b->n_hist;
    std::vector<std::pair<int64_t, int>> by_size((size_t)H);
    for (int64_t h = 0; h < H; ++h) {
        const int64_t n = host_offsets[h + 1] - host_offsets[h];
        if (n < 0) return CG_ERR_INVALID_ARG;
        by_size[(size_t)h] = {n, (int)h};
    }
    std::stable_sort(by_size.begin(), by_size.end(),
                     [](const std::pair<int64_t, int>& x, const std::pair<int64_t, int>& y) { return x.first > y.first; });
    std::vector<int> q[3];
    for (auto& e : by_size) {
        int kind;
        if (e.first > map->cta_max_bins && map->cluster_size > 1) kind = 0;
        else if (e.first > map->warp_max_bins) kind = 1;
        else kind = 2;
        q[kind].push_back(e.second);
    }
    const FitWsLayout L = fit_ws_layout(H);
    std::vector<int> flat((size_t)3 * H, 0);
    for (int k = 0; k < 3; ++k) std::copy(q[k].begin(), q[k].end(), flat.begin() + (size_t)k * H);
    QueueMeta meta;
    for (int k = 0; k < 3; ++k) meta.n_items[k] = (int)q[k].size();
    meta.cluster_size = map->cluster_size;
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)ws;
    std::vector<int> order((size_t)H);
    for (int64_t h = 0; h < H; ++h) order[(size_t)h] = by_size[(size_t)h].second;
    if (cudaMemcpyAsync(base + L.queues, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(base + L.qmeta, &meta, sizeof(meta), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(base, 0, 512, st) != cudaSuccess)
        return CG_ERR_CUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_fit_init(const cg_batch* b, const cg_tile_map* map, const double* theta0, cg_fit_state* state,
                      void* ws, size_t ws_bytes, void* stream) {
    cg_status s = batch_checks(b, ws, ws_bytes);
    if (s != CG_OK) return s;
    if (!theta0 || !state || !map_ok(map)) return CG_ERR_INVALID_ARG;
    FitArgs a = base_args(b);
    a.theta = theta0;
    a.st = state;
    const FitWsLayout L = fit_ws_layout(b->n_hist);
    char* base = (char*)ws;
    a.order = (const int*)(base + L.order);
    a.ectr = (int*)(base + L.counters) + 4;
    if (cudaMemsetAsync(a.ectr, 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess) return CG_ERR_CUDA;
    return launch_eval(&b->tmpl, a, 1, (cudaStream_t)stream);
}

cg_status cg_fit_step(const cg_batch* b, const cg_tile_map* map, cg_fit_state* state, int n_steps, double tol,
                      void* ws, size_t ws_bytes, void* stream) {
    cg_status s = batch_checks(b, ws, ws_bytes);
    if (s != CG_OK) return s;
    if (!state || !map_ok(map) || n_steps < 0 || !(tol >= 0.0)) return CG_ERR_INVALID_ARG;
    if (n_steps == 0) return CG_OK;
    const FitWsLayout L = fit_ws_layout(b->n_hist);
    char* base = (char*)ws;
    FitArgs a = base_args(b);
    a.st = state;
    a.n_steps = n_steps;
    a.tol = tol;
    a.counters = (int*)(base + L.counters);
    a.n_items = (const int*)(base + L.qmeta);
    for (int k = 0; k < 3; ++k) a.queue[k] = (const int*)(base + L.queues) + (size_t)k * b->n_hist;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(a.counters, 0, 16, st) != cudaSuccess) return CG_ERR_CUDA;
    return launch_persistent(&b->tmpl, a, map, st);
}

// ---- plain per-histogram path ----------------------------------------------
size_t cg_fit_single_workspace_size(const cg_problem* pb) {
    if (!pb || !fit_supported(pb)) return 0;
    const size_t g = grad_workspace_bytes(pb, 1);
    if (g == 0) return 0;
    return g + align_up(sizeof(SingleWs), 256);
}

static cg_status single_checks(const cg_problem* pb, void* ws, size_t ws_bytes) {
    if (!pb || !fit_supported(pb) || pb->centres || pb->n_bins[0] < 1 || !pb->data) return CG_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < cg_fit_single_workspace_size(pb)) return CG_ERR_WORKSPACE;
    return CG_OK;
}

cg_status cg_fit_single_init(const cg_problem* pb, const double* theta0, cg_fit_state* state, void* ws,
                             size_t ws_bytes, void* stream) {
    cg_status s = single_checks(pb, ws, ws_bytes);
    if (s != CG_OK) return s;
    if (!theta0 || !state) return CG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    SingleWs* w = (SingleWs*)((char*)ws + grad_workspace_bytes(pb, 1));
    k_single_setup<<<1, 1, 0, st>>>(w, pb->n_bins[0], pb->lo[0], pb->hi[0]);
    FitArgs a;
    memset(&a, 0, sizeof(a));
    a.data = pb->data;
    a.offsets = w->offsets;
    a.lo = &w->lo;
    a.hi = &w->hi;
    a.H = 1;
    a.D = pb->poly_degree;
    a.pm = pb->poly_mode;
    a.P = 3 * pb->n_peaks + pb->poly_degree + 1;
    a.theta = theta0;
    a.st = state;
    return launch_eval(pb, a, 1, st);
}

cg_status cg_fit_single_step(const cg_problem* pb, cg_fit_state* state, int n_evals, double tol, void* ws,
                             size_t ws_bytes, void* stream) {
    cg_status s = single_checks(pb, ws, ws_bytes);
    if (s != CG_OK) return s;
    if (!state || n_evals < 0 || !(tol >= 0.0)) return CG_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t gbytes = grad_workspace_bytes(pb, 1);
    SingleWs* w = (SingleWs*)((char*)ws + gbytes);
    for (int e = 0; e < n_evals; ++e) {
        k_single_ctl<<<1, 32, 0, st>>>(w, state, tol);
        s = grad_points(pb, w->s.tt, 1, &w->ft, w->gt, ws, gbytes, st, &w->need_eval);
        if (s != CG_OK) return s;
    }
    if (n_evals > 0) k_single_ctl<<<1, 32, 0, st>>>(w, state, tol);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

}  // extern "C"
