// cg_grad.cu -- fused forward + adjoint kernels (FP64) and the C-ABI entry
// points cg_objective / cg_gradient / cg_batch_gradient (parameter-point
// batches) of libcg.
//
// The method (Sec. 1-2 of the paper): reverse-mode AD of F(theta) =
// sum_i T_i(theta).  Per element i one thread evaluates the model and the
// term T_i (forward), seeds the term's adjoint dT_i/df_i and propagates it to
// per-thread FP64 adjoint accumulators (reverse); no tape is kept, every
// intermediate lives in registers.  Quantities that depend on theta alone
// (1/(2 s^2), normalisation integrals, cos/sin of angles) are computed once
// per tile in a prologue, and their adjoints are chained back to theta once
// per parameter point in the epilogue, so the per-element adjoint is a small
// set of sums (the model's "accumulators").  Summing the per-element
// adjoints is the "parallel reads become parallel writes" step of Sec. 3:
// here a deterministic warp-butterfly -> block -> fixed-order tile sum, with
// no floating-point atomics.
//
// Work decomposition: a tile is (parameter point, contiguous chunk of
// elements).  A persistent grid of (#SMs x resident CTAs) blocks walks the
// tiles round-robin; each tile writes one partial vector; a finalize kernel
// (one block per parameter point) sums the partials of a point in chunk
// order and applies the epilogue.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <unordered_map>

#include "cg_internal.cuh"
#include "cg_models.cuh"
#include "cg_models_fp64.cuh"
#include "cg_tiles.cuh"

namespace cg {

cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

int device_sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return kNumSMsFallback;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        return kNumSMsFallback;
    return n;
}

// ---------------------------------------------------------------------------
// Tile accumulation kernels
// ---------------------------------------------------------------------------

// 1-D Gaussian peaks + polynomial, FP64.  A tile is (PT consecutive
// parameter points, one chunk of bins); every bin's point-independent part
// is taken once and reused for the PT points.  In a ragged last group the
// missing points repeat the group's first point and are not written.
template <int K, int OBJ, int PT, int NT>
__global__ void __launch_bounds__(NT) k_gp1_fp64(GP1Data d, const double* __restrict__ theta,
                                                 TileGrid tg, double* __restrict__ part,
                                                 WsHeader* __restrict__ hdr) {
    constexpr int N = GP1Acc<K>::N;
    __shared__ Fp64Tab tab;
    __shared__ GP1Consts cs[PT];
    __shared__ GP1C2 cq[PT];
    __shared__ int s_badm;
    __shared__ double red[N * PT * (NT / 32)];
    __shared__ double tot[N * PT];
    if (gated_off(tg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->status = 0;
    fp64_tab_load<OBJ != CG_OBJ_CHI2>(tab);
    const int P = 3 * K + d.D + 1;
    for (int t = blockIdx.x; t < tg.n_tiles; t += gridDim.x) {
        const int c = t / tg.n_theta, grp = t - c * tg.n_theta;   // chunk-major: a chunk stays in L2 across points
        const int th0 = grp * PT;
        const int np = min(PT, tg.n_pts - th0);
        if (threadIdx.x == 0) s_badm = 0;
        __syncthreads();
        if (threadIdx.x < PT) {
            const int pt = threadIdx.x;
            const bool ok = gp1_prologue<K>(theta + (size_t)(th0 + (pt < np ? pt : 0)) * P, d.D, cs[pt]);
            gp1_c2(cs[pt], K, cq[pt]);
            if (!ok && pt < np) atomicOr(&s_badm, 1 << pt);
        }
        __syncthreads();
        double acc[PT][N];
#pragma unroll
        for (int p = 0; p < PT; ++p)
#pragma unroll
            for (int a = 0; a < N; ++a) acc[p][a] = 0.0;
        bool bad[PT];
#pragma unroll
        for (int p = 0; p < PT; ++p) bad[p] = false;
        // centre lo + (i + 1/2) h as (2i + 1) (h/2) + lo: one conversion and one FMA
        // (2i + 1 and h/2 are exact, so this is the correctly rounded centre)
        const double hh = 0.5 * d.h;
        auto centre = [&](int64_t i) { return fma((double)(2 * i + 1), hh, d.lo); };
        const int64_t e0 = (int64_t)c * tg.chunk;
        const int64_t e1 = min(tg.n_elem, e0 + tg.chunk);
        gp1_dispatch(d.D, d.pm, [&](auto dd_, auto pm_) {
            constexpr int DD = decltype(dd_)::value, PM = decltype(pm_)::value;
            auto bin = [&](double x, double y) {
                const GP1Bin b = gp1_bin<OBJ, PM>(x, y, d, tab);
#pragma unroll
                for (int p = 0; p < PT; ++p) gp1_elem_f64<K, OBJ, DD>(b, cs[p], cq[p], tab, acc[p], bad[p]);
            };
            if (d.vec_ok) {
                // two consecutive bins per thread with one 16-byte load of the counts (e0 is even)
                for (int64_t i = e0 + 2 * threadIdx.x; i < e1; i += 2 * NT) {
                    if (i + 1 < e1) {
                        const double2 y2 = __ldg(reinterpret_cast<const double2*>(d.y + i));
                        double2 x2;
                        if (d.centres) x2 = __ldg(reinterpret_cast<const double2*>(d.centres + i));
                        else { x2.x = centre(i); x2.y = centre(i + 1); }
                        bin(x2.x, y2.x);
                        bin(x2.y, y2.y);
                    } else {
                        bin(d.centres ? d.centres[i] : centre(i), d.y[i]);
                    }
                }
            } else {
                for (int64_t i = e0 + threadIdx.x; i < e1; i += NT)
                    bin(d.centres ? d.centres[i] : centre(i), d.y[i]);
            }
        });
        int bm = 0;
#pragma unroll
        for (int p = 0; p < PT; ++p)
            if (bad[p] || nonfinite(acc[p][0])) bm |= 1 << p;
        if (bm) atomicOr(&s_badm, bm);
        __syncthreads();
        const int badm = s_badm;
        block_sum_rs<N * PT, NT>(reinterpret_cast<const double(&)[N * PT]>(acc), red, tot);
        // the objective's constant factors once per tile, on the block's sums
        for (int k = threadIdx.x; k < np * (N + 1); k += NT) {
            const int pt = k / (N + 1), a = k - pt * (N + 1);
            part[((size_t)(th0 + pt) * (N + 1) + a) * tg.nbx + c] =
                (a < N) ? tot[pt * N + a] * gp1_acc_factor<OBJ>(a) : (((badm >> pt) & 1) ? 1.0 : 0.0);
        }
    }
}

// The events [e0, e1) of one tile through one form of the mixture element
// (FORM 0: mix_elem_f64, 1: mix_elem_ratio, 2: mix_elem_lean); pairs of
// events per load when the arrays are 16-byte aligned.
template <bool W, int NT, int FORM>
__device__ __forceinline__ void mix_events(const MixData& d, int64_t e0, int64_t e1, const MixConsts& cs,
                                           const MixC2& cq, const MixR2& cr, const Fp64Tab& tab,
                                           double (&acc)[MixAcc::N], LogProd& lp, bool& bad) {
    auto elem = [&](double x, double w) {
        if constexpr (FORM == 2) mix_elem_lean<W>(x, w, cs, cr, tab, acc, lp, bad);
        else if constexpr (FORM == 1) mix_elem_ratio<W>(x, w, cs, cr, tab, acc, lp, bad);
        else mix_elem_f64<W>(x, w, cs, cq, tab, acc, lp, bad);
    };
    if (d.vec_ok) {
        for (int64_t i = e0 + 2 * threadIdx.x; i < e1; i += 2 * NT) {
            if (i + 1 < e1) {
                const double2 x2 = __ldg(reinterpret_cast<const double2*>(d.x + i));
                double2 w2 = make_double2(1.0, 1.0);
                if (W) w2 = __ldg(reinterpret_cast<const double2*>(d.w + i));
                elem(x2.x, w2.x);
                elem(x2.y, w2.y);
            } else {
                elem(d.x[i], W ? d.w[i] : 1.0);
            }
        }
    } else {
        for (int64_t i = e0 + threadIdx.x; i < e1; i += NT) elem(d.x[i], W ? d.w[i] : 1.0);
    }
}

// One tile's block sums in one form (see mix_events), the thread sums
// finished by mix_tile_finish; returns the tile's domain flag.
template <bool W, int NT, int FORM>
__device__ __forceinline__ int mix_tile_sums(const MixData& d, int64_t e0, int64_t e1, const MixConsts& cs,
                                             const MixC2& cq, const MixR2& cr, const Fp64Tab& tab, double* red,
                                             double* tot) {
    double acc[MixAcc::N];
#pragma unroll
    for (int a = 0; a < MixAcc::N; ++a) acc[a] = 0.0;
    LogProd lp;
    logprod_init(lp);
    bool bad = false;
    mix_events<W, NT, FORM>(d, e0, e1, cs, cq, cr, tab, acc, lp, bad);
    mix_tile_finish<W>(cs, tab, acc, lp);
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    block_sum_rs<MixAcc::N, NT>(acc, red, tot);
    return any_bad;
}

// Per chunk of the mixture's tile grid: sum (x - lo), and with weights sum w
// and sum w (x - lo) (MixData::csum), one block per chunk in a fixed order.
template <bool W, int NT>
__global__ void __launch_bounds__(NT) k_mix_chunk_sums(MixData d, TileGrid tg, double* __restrict__ csum) {
    __shared__ double red[3 * (NT / 32)];
    __shared__ double tot[3];
    if (gated_off(tg)) return;
    for (int c = blockIdx.x; c < tg.nbx; c += gridDim.x) {
        const int64_t e0 = (int64_t)c * tg.chunk, e1 = min(tg.n_elem, e0 + tg.chunk);
        double a[3] = {0.0, 0.0, 0.0};
        auto add = [&](double x, double w) {
            const double xl = x - d.lo;
            a[0] += xl;
            if (W) {
                a[1] += w;
                a[2] = fma(w, xl, a[2]);
            }
        };
        if (d.vec_ok) {   // 8 events per thread and step, four 16-byte loads in flight (chunk starts are even)
            for (int64_t i = e0 + 8 * threadIdx.x; i < e1; i += 8 * NT) {
                if (i + 7 < e1) {
                    double2 x2[4], w2[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        x2[q] = __ldg(reinterpret_cast<const double2*>(d.x + i) + q);
                        w2[q] = W ? __ldg(reinterpret_cast<const double2*>(d.w + i) + q) : make_double2(1.0, 1.0);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        add(x2[q].x, w2[q].x);
                        add(x2[q].y, w2[q].y);
                    }
                } else {
                    for (int64_t j = i; j < e1; ++j) add(d.x[j], W ? d.w[j] : 1.0);
                }
            }
        } else {
            for (int64_t i = e0 + threadIdx.x; i < e1; i += NT) add(d.x[i], W ? d.w[i] : 1.0);
        }
        block_sum_rs<3, NT>(a, red, tot);
        if (threadIdx.x == 0) {
            csum[c] = tot[0];
            if (W) {
                csum[tg.nbx + c] = tot[1];
                csum[2 * tg.nbx + c] = tot[2];
            }
        }
        __syncthreads();
    }
}

// Unbinned Gaussian + exponential mixture, FP64: one point per tile.  A tile
// whose point has both coefficients a, b > 0 (every point inside the
// parameter space) takes the lean ratio form, one exponential and the
// Gaussian's three sums per event; where the exponential's sums taken as
// differences would cancel (mix_lean_sums), the tile is summed again in the
// full ratio form.  Other points (a = 0 at f = 0, b <= 0 at f >= 1) take the
// two-exponential form.  All three give the same accumulators.
template <bool W, int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_mix_fp64(MixData d, const double* __restrict__ theta,
                                                          TileGrid tg, double* __restrict__ part,
                                                          WsHeader* __restrict__ hdr) {
    constexpr int NACC = MixAcc::N;
    __shared__ Fp64Tab tab;
    __shared__ MixConsts cs;
    __shared__ MixC2 cq;
    __shared__ MixR2 cr;
    __shared__ int cs_bad, lean_ok;
    __shared__ double red[NACC * (NT / 32)];
    __shared__ double tot[NACC];
    if (gated_off(tg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->status = 0;
    fp64_tab_load(tab);
    for (int t = blockIdx.x; t < tg.n_tiles; t += gridDim.x) {
        const int c = t / tg.n_theta, th = t - c * tg.n_theta;   // chunk-major: a chunk stays in L2 across points
        if (threadIdx.x == 0) {
            cs_bad = mix_prologue(theta + (size_t)th * 4, d.lo, d.hi, cs) ? 0 : 1;
            mix_c2(cs, cq);
            mix_r2(cs, cr);
        }
        __syncthreads();
        const bool ratio = cr.ok != 0;
        const int64_t e0 = (int64_t)c * tg.chunk;
        const int64_t e1 = min(tg.n_elem, e0 + tg.chunk);
        int any_bad;
        if (ratio) {
            const double n_w = W ? d.csum[tg.nbx + c] : (double)(e1 - e0);
            const double sxl = W ? d.csum[2 * tg.nbx + c] : d.csum[c];
            any_bad = mix_tile_sums<W, NT, 2>(d, e0, e1, cs, cq, cr, tab, red, tot);
            if (threadIdx.x == 0) lean_ok = mix_lean_sums(cs, cr, n_w, sxl, tot) ? 1 : 0;
            __syncthreads();
            if (!lean_ok) {
                any_bad = mix_tile_sums<W, NT, 1>(d, e0, e1, cs, cq, cr, tab, red, tot);
                if (threadIdx.x == 0) mix_ratio_sums(cs, cr, n_w, sxl, tot);
                __syncthreads();
            }
        } else {
            any_bad = mix_tile_sums<W, NT, 0>(d, e0, e1, cs, cq, cr, tab, red, tot);
        }
        write_partial<NACC>(part, tg, th, c, tot, any_bad | cs_bad);
    }
}

// The mixture's FP64 launch: the tile grid, the chunk sums, the tile kernel.
template <bool W, int NT>
static cg_status launch_mix_fp64(MixData d, double* csum, const double* theta, int64_t n, int64_t n_theta,
                                 double* part, WsHeader* hdr, TileGrid* tg_out, cudaStream_t st, const int* gate) {
    const int nsm = device_sm_count();
    const int R = resident_blocks((const void*)k_mix_fp64<W, NT>, NT, 0);
    TileGrid tg = make_tiles_balanced(n, n_theta, 1, NT, nsm, R);
    tg.gate = gate;
    k_mix_chunk_sums<W, 512><<<tg.nbx, 512, 0, st>>>(d, tg, csum);
    d.csum = csum;
    const int G = nsm * R;
    const int grid = tg.n_tiles < G ? tg.n_tiles : G;
    prof_begin(st);
    k_mix_fp64<W, NT><<<grid, NT, 0, st>>>(d, theta, tg, part, hdr);
    prof_end(st);
    *tg_out = tg;
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

// 2-D tiles of kRgTX x kRgTY bins.  Per tile, a Gaussian whose exponent
// -q = -(u^2/sx^2 + v^2/sy^2)/2 stays below -kRgCull everywhere in the tile's
// box of bin centres is skipped (the exact maximum of the exponent over the
// box, rg2_box_max_exponent).  The dropped term is below e^-80 A = 1.8e-35 A
// at every bin of the tile, under the FP64 resolution of the model value
// wherever that value exceeds 1.8e-19 A (a constant C > 0 or another
// Gaussian within reach).
constexpr int kRgTX = 64, kRgTY = 64;
constexpr double kRgCull = 80.0;
constexpr int kRgRecMaxKept = 5;   // more kept Gaussians per tile: the direct form (register pressure)

// The rows of one tile for the NA Gaussians kept by its culling: thread ->
// one column (consecutive threads, consecutive bins of a row), rows r0,
// r0 + NT / kRgTX, ...; the block's sums of the (dx, dy) moments over the
// kept Gaussians land in totc[0 .. 2 + 6 NA).
template <int NA, int NT>
__device__ __forceinline__ void rg2_tile_rows(const RG2Data& d, int64_t x0, int64_t y0, int w, int h, double C,
                                              const RG2Act& a, const Fp64Tab& tab, double* red, double* totc,
                                              bool& bad) {
    constexpr int NM = 2 + 6 * NA;
    constexpr int S = NT / kRgTX;   // rows between a thread's bins
    constexpr int KA = NA > 0 ? NA : 1;
    double m[NM];
#pragma unroll
    for (int i = 0; i < NM; ++i) m[i] = 0.0;
    const int col_i = threadIdx.x % kRgTX, r0 = threadIdx.x / kRgTX;
    const bool mine = col_i < w;
    // centres lo + (i + 1/2) h as (2i + 1) (h/2) + lo (correctly rounded, one FMA each)
    const double hhy = 0.5 * d.hy;
    const int64_t ix = x0 + col_i;
    const int nr = r0 < h ? (h - 1 - r0) / S + 1 : 0;   // this thread's rows
    const double xc = fma((double)(2 * ix + 1), 0.5 * d.hx, d.lx);
    double cacc[2 + 3 * NA];
#pragma unroll
    for (int i = 0; i < 2 + 3 * NA; ++i) cacc[i] = 0.0;
    // the row recurrence (rg2_act_rec) where every kept Gaussian allows it at
    // both ends of every thread's run, else the direct form for the whole tile
    // (the column's constants are taken where they are used, so that the
    // recurrence loop holds only E, R and the sums); compiled for up to
    // kRgRecMaxKept kept Gaussians (more: the direct form, register pressure)
    bool rec = false;
    if constexpr (NA > 0 && NA <= kRgRecMaxKept) {
        double E[KA], R[KA];
        bool fail = h < 3 * S;   // h is the block's: short tiles take the direct form
        if (mine && !fail) {
            RG2Col<NA> col;
            rg2_col<NA>(xc, a, col);
            const double yf = fma((double)(2 * (y0 + r0) + 1), hhy, d.ly);
            const double yl = fma((double)(2 * (y0 + r0 + (int64_t)(nr - 1) * S) + 1), hhy, d.ly);
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                double up, vp, ul, vl;
                const double e0 = rg2_col_exponent<NA>(a, col, j, yf - a.my[j], up, vp);
                const double el = rg2_col_exponent<NA>(a, col, j, yl - a.my[j], ul, vl);
                const double lr = -fma(up, a.a2[j], fma(vp, a.b2[j], a.kk[j]));
                fail |= !(e0 > -1000.0 && el > -1000.0 && fabs(lr) < 1000.0 && fabs(a.qm[j]) < kRgRecQMax);
                E[j] = exp2_core(e0, tab);   // table index masked: in bounds for any argument
                R[j] = exp2_core(lr, tab);
            }
        }
        rec = __syncthreads_or(fail ? 1 : 0) == 0;
        if (rec && mine) {
            int64_t iy = y0 + r0;
            for (int r = 0; r < nr; ++r, iy += S) {
                const double y = fma((double)(2 * iy + 1), hhy, d.ly);
                double dy[KA], e[KA];
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    dy[j] = y - a.my[j];
                    e[j] = E[j];
                    E[j] *= R[j];
                    R[j] = fma(R[j], a.qm[j], R[j]);
                }
                rg2_elem_col_de<NA>(__ldg(d.n + iy * d.nx + ix), C, a, dy, e, tab, cacc, bad);
            }
        }
    }
    if (mine) {
        if (!rec) {
            RG2Col<NA> col;
            rg2_col<NA>(xc, a, col);
            for (int r = r0; r < h; r += S) {
                const int64_t iy = y0 + r;
                rg2_elem_col<NA>(fma((double)(2 * iy + 1), hhy, d.ly), __ldg(d.n + iy * d.nx + ix), C, a, col,
                                 tab, cacc, bad);
            }
        }
        RG2Col<NA> col;
        rg2_col<NA>(xc, a, col);
        rg2_col_moments<NA>(col, cacc, m);
    }
    bad |= nonfinite(m[0]);
    block_sum_rs<NM, NT>(m, red, totc);
}

// rg2_tile_rows compiled for each count 0 .. NA of kept Gaussians; n selects
// one (uniform over the block).
template <int NA, int NT>
__device__ __forceinline__ void rg2_rows_upto(int n, const RG2Data& d, int64_t x0, int64_t y0, int w, int h,
                                              double C, const RG2Act& a, const Fp64Tab& tab, double* red,
                                              double* totc, bool& bad) {
    if (n == NA) rg2_tile_rows<NA, NT>(d, x0, y0, w, h, C, a, tab, red, totc, bad);
    else if constexpr (NA > 0) rg2_rows_upto<NA - 1, NT>(n, d, x0, y0, w, h, C, a, tab, red, totc, bad);
}

template <int K, int NT>
__global__ void __launch_bounds__(NT, 3) k_rg2_fp64(RG2Data d, const double* __restrict__ theta,
                                                 TileGrid tg, double* __restrict__ part,
                                                 WsHeader* __restrict__ hdr) {
    constexpr int NACC = RG2Acc<K>::N;
    static_assert(NT % kRgTX == 0, "whole columns per block");
    __shared__ Fp64Tab tab;
    __shared__ RG2Consts cs;
    __shared__ RG2Q cq;
    __shared__ RG2Act ka;
    __shared__ int cs_bad;
    __shared__ unsigned act_s;
    __shared__ double red[NACC * (NT / 32)];
    __shared__ double totc[NACC];   // block sums over the kept Gaussians
    __shared__ double tot[NACC];    // the same in accumulator order
    if (gated_off(tg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) hdr->status = 0;
    fp64_tab_load(tab);
    const int P = 6 * K + 1;
    const int ntx = (int)((d.nx + kRgTX - 1) / kRgTX);
    for (int t = blockIdx.x; t < tg.n_tiles; t += gridDim.x) {
        const int c = t / tg.n_theta, th = t - c * tg.n_theta;
        const int ty = c / ntx, tx = c - ty * ntx;
        const int64_t x0 = (int64_t)tx * kRgTX, y0 = (int64_t)ty * kRgTY;
        const int64_t x1 = min(d.nx, x0 + kRgTX), y1 = min(d.ny, y0 + kRgTY);
        if (threadIdx.x < 32) {   // one Gaussian per lane: constants, culling, the kept set
            const int k = threadIdx.x;
            const double* tht = theta + (size_t)th * P;
            bool ok = true, keep = false;
            if (k < K) {
                ok = rg2_prologue_one(tht + 6 * k, k, cs);
                rg2_q_one(cs, k, cq);
                // the box of bin centres of this tile, as offsets from the Gaussian's centre
                const double bx0 = fma((double)x0 + 0.5, d.hx, d.lx), bx1 = fma((double)(x1 - 1) + 0.5, d.hx, d.lx);
                const double by0 = fma((double)y0 + 0.5, d.hy, d.ly), by1 = fma((double)(y1 - 1) + 0.5, d.hy, d.ly);
                const double mx = cs.mx[k], my = cs.my[k];
                const double emax = rg2_box_max_exponent(cq, k, bx0 - mx, bx1 - mx, by0 - my, by1 - my);
                keep = !(emax < -kRgCull * kLog2e);   // NaN keeps the Gaussian
            }
            const unsigned act = __ballot_sync(0xffffffffu, keep);
            const bool all_ok = __all_sync(0xffffffffu, ok);
            if (keep) {
                const int slot = __popc(act & ((1u << k) - 1u));
                rg2_act_one(cs, k, slot, ka);
                rg2_act_rec(slot, (double)(NT / kRgTX) * d.hy, ka);
            }
            if (k == 0) {
                cs.C = tht[6 * K];
                cs_bad = (all_ok && isfinite(cs.C)) ? 0 : 1;
                act_s = act;
                ka.n = __popc(act);
            }
        }
        __syncthreads();
        const unsigned act = act_s;
        const int nact = ka.n;
        bool bad = false;
        rg2_rows_upto<K, NT>(nact, d, x0, y0, (int)(x1 - x0), (int)(y1 - y0), cs.C, ka, tab, red, totc, bad);
        const int any_bad = __syncthreads_or(bad ? 1 : 0) | cs_bad;
        // the kept Gaussians' moments rotated to (u, v) and put in accumulator order (0 for the culled)
        if (threadIdx.x < nact) {
            const int k = ka.k[threadIdx.x];
            rg2_rotate_moments(totc + 1 + 6 * threadIdx.x, cs.cs[k], cs.sn[k]);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NACC; i += NT) {
            double v;
            if (i == 0) {
                v = totc[0];
            } else if (i == NACC - 1) {
                v = totc[1 + 6 * nact];
            } else {
                const int k = (i - 1) / 6, comp = i - 1 - 6 * k;
                v = ((act >> k) & 1u) ? totc[1 + 6 * __popc(act & ((1u << k) - 1u)) + comp] : 0.0;
            }
            tot[i] = v;
        }
        __syncthreads();
        write_partial<NACC>(part, tg, th, c, tot, any_bad);
    }
}

// ---------------------------------------------------------------------------
// Finalize: fixed-order sum of the tile partials of one parameter point and
// the epilogue (adjoints of the prologue constants chained back to theta).
// Warp w sums accumulators w, w + NT/32, ...: lane l adds chunks l, l + 32,
// ... in order, then a butterfly (the same sum on every lane).  Launched as a
// programmatic dependent of the tile kernel: its blocks may be scheduled
// while the tile kernel's last blocks run, and wait here until the tile
// kernel has completed and its partials are visible.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT) k_finalize(const double* __restrict__ part, int nacc, TileGrid tg,
                                                 EpiParams ep, const double* __restrict__ theta,
                                                 double* __restrict__ value, double* __restrict__ grad,
                                                 WsHeader* __restrict__ hdr) {
    __shared__ double tot[kMaxAcc + 1];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (gated_off(tg)) return;
    const int th = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int a = wid; a <= nacc; a += NT / 32) {
        const double* p = part + ((size_t)th * (nacc + 1) + a) * tg.nbx;
        double s = 0.0;
        for (int c = lane; c < tg.nbx; c += 32) s += p[c];
        s = warp_sum(s);
        if (lane == 0) tot[a] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double* tht = theta + (size_t)th * ep.P;
        double g[kMaxParams];
        double v = epilogue(ep, tht, tot, g);
        if (value) value[th] = v;
        if (grad)
            for (int k = 0; k < ep.P; ++k) grad[(size_t)th * ep.P + k] = g[k];
        if (tot[nacc] != 0.0) atomicOr(&hdr->status, (int)DEV_DOMAIN);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int acc_count(const cg_problem* pb) {
    switch (pb->model) {
        case CG_MODEL_GAUSS_POLY: return 1 + 3 * pb->n_peaks + 4;
        case CG_MODEL_MIX_GAUSS_EXP: return MixAcc::N;
        case CG_MODEL_ROTGAUSS2D: return 2 + 6 * pb->n_peaks;
        default: return -1;
    }
}

static int64_t n_elements(const cg_problem* pb) {
    switch (pb->model) {
        case CG_MODEL_GAUSS_POLY: return pb->n_bins[0];
        case CG_MODEL_MIX_GAUSS_EXP: return pb->n_events;
        case CG_MODEL_ROTGAUSS2D: return pb->n_bins[0] * pb->n_bins[1];
        default: return -1;
    }
}

static cg_status validate(const cg_problem* pb) {
    if (!pb) return CG_ERR_INVALID_ARG;
    if (pb->precision != CG_PREC_FP64 && pb->precision != CG_PREC_DF64) return CG_ERR_INVALID_ARG;
    switch (pb->model) {
        case CG_MODEL_GAUSS_POLY:
            if (pb->n_peaks < 0 || pb->n_peaks > CG_MAX_PEAKS_1D) return CG_ERR_INVALID_ARG;
            if (pb->poly_degree < -1 || pb->poly_degree > CG_MAX_POLY_DEGREE) return CG_ERR_INVALID_ARG;
            if (pb->n_peaks == 0 && pb->poly_degree < 0) return CG_ERR_INVALID_ARG;
            if (pb->poly_mode != 0 && pb->poly_mode != 1) return CG_ERR_INVALID_ARG;
            if (pb->objective != CG_OBJ_CHI2 && pb->objective != CG_OBJ_POISSON &&
                pb->objective != CG_OBJ_POISSON_BC)
                return CG_ERR_INVALID_ARG;
            if (pb->n_bins[0] < 0) return CG_ERR_INVALID_ARG;
            if (pb->n_bins[0] > 0 && !pb->data) return CG_ERR_INVALID_ARG;
            if (!pb->centres && !(pb->hi[0] > pb->lo[0])) return CG_ERR_INVALID_ARG;
            return CG_OK;
        case CG_MODEL_MIX_GAUSS_EXP:
            if (pb->objective != CG_OBJ_UNBINNED_NLL) return CG_ERR_INVALID_ARG;
            if (pb->n_events < 0 || (pb->n_events > 0 && !pb->data)) return CG_ERR_INVALID_ARG;
            if (!(pb->hi[0] > pb->lo[0])) return CG_ERR_INVALID_ARG;
            return CG_OK;
        case CG_MODEL_ROTGAUSS2D:
            if (pb->n_peaks < 1 || pb->n_peaks > CG_MAX_PEAKS_2D) return CG_ERR_INVALID_ARG;
            if (pb->objective != CG_OBJ_POISSON) return CG_ERR_INVALID_ARG;
            if (pb->n_bins[0] < 0 || pb->n_bins[1] < 0) return CG_ERR_INVALID_ARG;
            if (pb->n_bins[0] * pb->n_bins[1] > 0 && !pb->data) return CG_ERR_INVALID_ARG;
            if (!(pb->hi[0] > pb->lo[0]) || !(pb->hi[1] > pb->lo[1])) return CG_ERR_INVALID_ARG;
            return CG_OK;
        default:
            return CG_ERR_INVALID_ARG;
    }
}

static int num_params(const cg_problem* pb) {
    switch (pb->model) {
        case CG_MODEL_GAUSS_POLY: return 3 * pb->n_peaks + pb->poly_degree + 1;
        case CG_MODEL_MIX_GAUSS_EXP: return 4;
        case CG_MODEL_ROTGAUSS2D: return 6 * pb->n_peaks + 1;
        default: return -1;
    }
}

size_t grad_workspace_bytes(const cg_problem* pb, int64_t n_theta) {
    if (validate(pb) != CG_OK || n_theta < 1) return 0;
    const int nacc = acc_count(pb);
    // then the df64 kernels' split events, or the FP64 mixture's three sums per chunk
    const size_t mix_csum = (pb->model == CG_MODEL_MIX_GAUSS_EXP && pb->precision == CG_PREC_FP64)
                                ? align_up((size_t)3 * max_nbx(n_theta) * sizeof(double), 256)
                                : 0;
    return sizeof(WsHeader) + align_up((size_t)n_theta * (nacc + 1) * max_nbx(n_theta) * sizeof(double), 256) +
           df64_split_bytes(pb) + mix_csum;
}

// Points per tile of the 1-D FP64 kernel: 4 for models of at most one peak
// (their per-thread sums stay in registers), else 1.
template <int K>
static cg_status launch_gp1_k(const cg_problem* pb, const GP1Data& d, const double* theta, int64_t n_theta,
                              double* part, WsHeader* hdr, TileGrid* tg, cudaStream_t st, const int* gate) {
    constexpr int NT = 128;   // 157 registers at 4 points per tile: three CTAs per SM
    const int64_t n = pb->n_bins[0];
#ifndef CG_GP1_POINTS_PER_TILE
#define CG_GP1_POINTS_PER_TILE 4
#endif
    constexpr int PTM = (K <= 1) ? CG_GP1_POINTS_PER_TILE : 1;
    const bool multi = PTM > 1 && n_theta >= PTM;
#define CG_GP1_LAUNCH(OO)                                                                                        \
    return multi ? launch_tiles_balanced(k_gp1_fp64<K, OO, PTM, NT>, NT, PTM, d, theta, n, n_theta, part, hdr, tg, \
                                         st, gate)                                                               \
                 : launch_tiles_balanced(k_gp1_fp64<K, OO, 1, NT>, NT, 1, d, theta, n, n_theta, part, hdr, tg, st, \
                                         gate);
    switch (pb->objective) {
        case CG_OBJ_CHI2: CG_GP1_LAUNCH(CG_OBJ_CHI2)
        case CG_OBJ_POISSON: CG_GP1_LAUNCH(CG_OBJ_POISSON)
        case CG_OBJ_POISSON_BC: CG_GP1_LAUNCH(CG_OBJ_POISSON_BC)
        default: return CG_ERR_UNSUPPORTED;
    }
#undef CG_GP1_LAUNCH
}

template <int K>
static cg_status launch_rg2_k(const RG2Data& d, const double* theta, int64_t n, int64_t n_theta, double* part,
                              WsHeader* hdr, TileGrid* tg, cudaStream_t st, const int* gate) {
    constexpr int NT = 128;
    auto kern = k_rg2_fp64<K, NT>;
    const int R = resident_blocks((const void*)kern, NT, 0);
    const int G = device_sm_count() * R;
    TileGrid g;
    g.n_elem = n;
    g.chunk = 0;
    g.nbx = (int)(((d.nx + kRgTX - 1) / kRgTX) * ((d.ny + kRgTY - 1) / kRgTY));
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

cg_status grad_points(const cg_problem* pb, const double* theta, int64_t n_theta, double* value, double* grad,
                      void* ws, size_t ws_bytes, cudaStream_t st, const int* gate) {
    cg_status s = validate(pb);
    if (s != CG_OK) return s;
    if (n_theta < 1 || !theta || (!value && !grad)) return CG_ERR_INVALID_ARG;
    if (n_theta > (int64_t)kMaxTiles * 64) return CG_ERR_INVALID_ARG;
    const size_t need = grad_workspace_bytes(pb, n_theta);
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < need) return CG_ERR_WORKSPACE;
    if (pb->precision != CG_PREC_FP64 && !df64_supported(pb)) return CG_ERR_UNSUPPORTED;
    WsHeader* hdr = (WsHeader*)ws;
    double* part = (double*)((char*)ws + sizeof(WsHeader));
    const int64_t n = n_elements(pb);
    const int nacc = acc_count(pb);
    TileGrid tg;
    EpiParams ep;
    memset(&ep, 0, sizeof(ep));
    ep.model = pb->model;
    ep.P = num_params(pb);
    ep.K = pb->n_peaks;
    ep.D = pb->poly_degree;
    ep.lo = pb->lo[0];
    ep.hi = pb->hi[0];
    if (n == 0 && gate) return CG_ERR_UNSUPPORTED;
    if (n == 0) {
        // empty data: every sum is zero; still produce value/grad and a clean status
        cudaMemsetAsync(hdr, 0, sizeof(WsHeader), st);
        tg.n_elem = 0; tg.chunk = 1; tg.nbx = 1; tg.n_theta = (int)n_theta; tg.n_tiles = (int)n_theta;
        tg.gate = nullptr;
        cudaMemsetAsync(part, 0, (size_t)n_theta * (nacc + 1) * sizeof(double), st);
        s = CG_OK;
    } else if (pb->precision == CG_PREC_DF64) {
        const int nacc_ = acc_count(pb);
        void* split = (char*)ws + sizeof(WsHeader) +
                      align_up((size_t)n_theta * (nacc_ + 1) * max_nbx(n_theta) * sizeof(double), 256);
        s = launch_df64(pb, theta, n_theta, part, hdr, &tg, st, gate, grad == nullptr, split);
    } else if (pb->model == CG_MODEL_GAUSS_POLY) {
        GP1Data d;
        d.y = pb->data;
        d.centres = pb->centres;
        d.lo = pb->lo[0];
        d.h = (pb->hi[0] - pb->lo[0]) / (double)pb->n_bins[0];
        d.au = 2.0 / (pb->hi[0] - pb->lo[0]);
        d.bu = -(pb->lo[0] + pb->hi[0]) / (pb->hi[0] - pb->lo[0]);
        d.D = pb->poly_degree;
        d.pm = pb->poly_mode;
        d.vec_ok = (((uintptr_t)pb->data & 15) == 0) && (!pb->centres || (((uintptr_t)pb->centres & 15) == 0));
        switch (pb->n_peaks) {
            case 0: s = launch_gp1_k<0>(pb, d, theta, n_theta, part, hdr, &tg, st, gate); break;
            case 1: s = launch_gp1_k<1>(pb, d, theta, n_theta, part, hdr, &tg, st, gate); break;
            case 2: s = launch_gp1_k<2>(pb, d, theta, n_theta, part, hdr, &tg, st, gate); break;
            case 3: s = launch_gp1_k<3>(pb, d, theta, n_theta, part, hdr, &tg, st, gate); break;
            case 4: s = launch_gp1_k<4>(pb, d, theta, n_theta, part, hdr, &tg, st, gate); break;
            default: return CG_ERR_INVALID_ARG;
        }
    } else if (pb->model == CG_MODEL_MIX_GAUSS_EXP) {
        MixData d;
        d.x = pb->data;
        d.w = pb->weights;
        d.lo = pb->lo[0];
        d.hi = pb->hi[0];
        d.vec_ok = (((uintptr_t)pb->data & 15) == 0) && (!pb->weights || (((uintptr_t)pb->weights & 15) == 0));
        constexpr int NT = 256;
        double* csum = (double*)((char*)ws + sizeof(WsHeader) +
                                 align_up((size_t)n_theta * (nacc + 1) * max_nbx(n_theta) * sizeof(double), 256));
        s = pb->weights ? launch_mix_fp64<true, NT>(d, csum, theta, n, n_theta, part, hdr, &tg, st, gate)
                        : launch_mix_fp64<false, NT>(d, csum, theta, n, n_theta, part, hdr, &tg, st, gate);
    } else {
        RG2Data d;
        d.n = pb->data;
        d.nx = pb->n_bins[0];
        d.ny = pb->n_bins[1];
        d.lx = pb->lo[0];
        d.ly = pb->lo[1];
        d.hx = (pb->hi[0] - pb->lo[0]) / (double)pb->n_bins[0];
        d.hy = (pb->hi[1] - pb->lo[1]) / (double)pb->n_bins[1];
        switch (pb->n_peaks) {
            case 1: s = launch_rg2_k<1>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            case 2: s = launch_rg2_k<2>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            case 3: s = launch_rg2_k<3>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            case 4: s = launch_rg2_k<4>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            case 5: s = launch_rg2_k<5>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            case 6: s = launch_rg2_k<6>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            case 7: s = launch_rg2_k<7>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            case 8: s = launch_rg2_k<8>(d, theta, n, n_theta, part, hdr, &tg, st, gate); break;
            default: return CG_ERR_INVALID_ARG;
        }
    }
    if (s != CG_OK) return s;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_theta);
    cfg.blockDim = dim3(128);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_finalize<128>, (const double*)part, nacc, tg, ep, theta, value, grad, hdr) !=
        cudaSuccess)
        return CG_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

}  // namespace cg

using namespace cg;

extern "C" {

int cg_num_params(const cg_problem* pb) {
    if (validate(pb) != CG_OK) return -1;
    return num_params(pb);
}

size_t cg_workspace_size(const cg_problem* pb, int64_t n_theta) { return grad_workspace_bytes(pb, n_theta); }

cg_status cg_objective(const cg_problem* pb, const double* theta, double* value, void* ws, size_t ws_bytes,
                       void* stream) {
    if (!value) return CG_ERR_INVALID_ARG;
    return grad_points(pb, theta, 1, value, nullptr, ws, ws_bytes, (cudaStream_t)stream, nullptr);
}

cg_status cg_gradient(const cg_problem* pb, const double* theta, double* value, double* grad, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!value || !grad) return CG_ERR_INVALID_ARG;
    return grad_points(pb, theta, 1, value, grad, ws, ws_bytes, (cudaStream_t)stream, nullptr);
}

void cg_set_profile_events(void* start, void* stop) {
    g_prof_start = (cudaEvent_t)start;
    g_prof_stop = (cudaEvent_t)stop;
}

cg_status cg_get_status(const void* ws, void* stream) {
    if (!ws) return CG_ERR_INVALID_ARG;
    int32_t st = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&st, ws, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CG_ERR_CUDA;
    if (st & DEV_TIMEOUT) return CG_ERR_TIMEOUT;
    if (st & DEV_DOMAIN) return CG_ERR_DOMAIN;
    return CG_OK;
}

const char* cg_status_string(cg_status s) {
    switch (s) {
        case CG_OK: return "ok";
        case CG_ERR_INVALID_ARG: return "invalid argument";
        case CG_ERR_DOMAIN: return "domain error (non-positive model value under a log, or non-finite term)";
        case CG_ERR_CUDA: return "CUDA error";
        case CG_ERR_TIMEOUT: return "device wait timed out";
        case CG_ERR_NOT_CONVERGED: return "not converged";
        case CG_ERR_UNSUPPORTED: return "unsupported combination";
        case CG_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown status";
    }
}

}  // extern "C"
