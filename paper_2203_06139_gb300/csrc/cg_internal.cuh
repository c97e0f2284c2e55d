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
