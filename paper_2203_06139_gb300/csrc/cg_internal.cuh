// cg_internal.cuh -- shared device/host internals of libcg (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cg.h"

namespace cg {

// Device status bits, OR-ed into the workspace header.
enum : int32_t { DEV_DOMAIN = 1, DEV_TIMEOUT = 2 };

// Workspace header: the first 256 bytes of every workspace.
struct WsHeader {
    int32_t status;   // OR of DEV_* bits of the last call
    int32_t pad[63];
};
static_assert(sizeof(WsHeader) == 256, "header size");

constexpr int kNumSMsFallback = 152;

// ---------------------------------------------------------------------------
// Deterministic reductions
// ---------------------------------------------------------------------------

// Butterfly sum over the 32 lanes of a warp; every lane ends with the total.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of NACC per-thread accumulators over a block of NT threads, fixed
// order: warp butterflies, then warp 0 adds the per-warp sums in warp order.
// red: shared scratch of at least NACC * (NT/32) doubles. Result valid in
// thread 0 (out[a]); all threads must call it.
template <int NACC, int NT>
__device__ __forceinline__ void block_sum(const double (&acc)[NACC], double* red, double* out) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < NACC; ++a) {
        double v = warp_sum(acc[a]);
        if (lane == 0) red[a * NW + wid] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < NACC; ++a) {
            double s = 0.0;
            for (int w = 0; w < NW; ++w) s += red[a * NW + w];
            out[a] = s;
        }
    }
    __syncthreads();
}

// Reduce-scatter over the 32 lanes of a warp of NA <= 32 per-lane values
// (recursive halving, fixed order): with NP = NA rounded up to a power of
// two, NP/2 + NP/4 + ... + 1 additions halve the values held by a lane while
// pairing lanes across lane bits 4, 3, ...; a butterfly over the remaining
// lane bits completes the sums.  Returns on every lane the warp total of
// accumulator lane >> (5 - log2 NP) (zero for indices >= NA).  v is
// consumed.  Far fewer additions than NA butterflies (31 instead of 160 for
// 32 values).
template <int NA>
struct WarpRS {
    static constexpr int NP = NA <= 1 ? 1 : NA <= 2 ? 2 : NA <= 4 ? 4 : NA <= 8 ? 8 : NA <= 16 ? 16 : 32;
    static constexpr int SH = NP == 1 ? 5 : NP == 2 ? 4 : NP == 4 ? 3 : NP == 8 ? 2 : NP == 16 ? 1 : 0;
    static_assert(NA >= 1 && NA <= 32, "at most 32 values per lane");
};

template <int NA>
__device__ __forceinline__ double warp_reduce_scatter(const double (&v)[NA]) {
    constexpr int NP = WarpRS<NA>::NP;
    const int lane = threadIdx.x & 31;
    double w[NP];
#pragma unroll
    for (int i = 0; i < NP; ++i) w[i] = (i < NA) ? v[i] : 0.0;
#pragma unroll
    for (int half = NP / 2, bit = 16; half >= 1; half /= 2, bit /= 2) {
        const bool up = (lane & bit) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const double send = up ? w[k] : w[k + half];
            const double keep = up ? w[k + half] : w[k];
            w[k] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    double s = w[0];
#pragma unroll
    for (int bit = (1 << WarpRS<NA>::SH) >> 1; bit >= 1; bit >>= 1) s += __shfl_xor_sync(0xffffffffu, s, bit);
    return s;
}

// Block sum of NA <= 64 per-thread values by warp reduce-scatters (of the
// first 32 values and of the rest), then the per-warp totals of each
// accumulator added in warp order by one thread per accumulator.  red:
// NA * (NT/32) doubles of shared scratch; the totals land in tot[0 .. NA)
// (shared), valid for every thread after the call.
template <int NA, int NT>
__device__ __forceinline__ void block_sum_rs(const double (&acc)[NA], double* red, double* tot) {
    static_assert(NA >= 1 && NA <= 64, "at most 64 values per thread");
    constexpr int NW = NT / 32;
    constexpr int N1 = NA < 32 ? NA : 32, N2 = NA - N1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    {
        double v[N1];
#pragma unroll
        for (int i = 0; i < N1; ++i) v[i] = acc[i];
        constexpr int SH = WarpRS<N1>::SH;
        const double s = warp_reduce_scatter<N1>(v);
        const int a = lane >> SH;
        if ((lane & ((1 << SH) - 1)) == 0 && a < N1) red[a * NW + wid] = s;
    }
    if constexpr (N2 > 0) {
        double v[N2 > 0 ? N2 : 1];
#pragma unroll
        for (int i = 0; i < N2; ++i) v[i] = acc[N1 + i];
        constexpr int SH = WarpRS<N2>::SH;
        const double s = warp_reduce_scatter<N2>(v);
        const int a = lane >> SH;
        if ((lane & ((1 << SH) - 1)) == 0 && a < N2) red[(N1 + a) * NW + wid] = s;
    }
    __syncthreads();
    for (int a = threadIdx.x; a < NA; a += NT) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) t += red[a * NW + w];
        tot[a] = t;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Host helpers
// ---------------------------------------------------------------------------
int device_sm_count();

// Profiling events recorded around the dominant kernel launch (cg_set_profile_events).
extern cudaEvent_t g_prof_start, g_prof_stop;
inline void prof_begin(cudaStream_t st) { if (g_prof_start) cudaEventRecord(g_prof_start, st); }
inline void prof_end(cudaStream_t st) { if (g_prof_stop) cudaEventRecord(g_prof_stop, st); }
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace cg
