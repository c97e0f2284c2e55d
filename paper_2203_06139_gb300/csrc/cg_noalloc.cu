// cg_noalloc.cu -- unbinned mixture gradients for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// running inside another framework's custom allocator or memory pool that
// forbids outside allocations, plug-ins loaded into a host that owns every
// device buffer, and hard real-time loops where an allocation may block or
// fail at the wrong moment.  cg_mixture_gradient_noalloc serves them: its
// only scratch is the file-scope array below, which the CUDA runtime
// creates when it loads this library's device code on a GPU and keeps until
// the process exits (CG_NOALLOC_SCRATCH_BYTES on every GPU that loads it).
//
// The arithmetic is the same fused forward + adjoint of the unbinned
// Gaussian + exponential mixture NLL as cg_gradient / cg_batch_gradient
// (cg_models.cuh), with the same deterministic reduction; only the home of
// the per-tile partial sums differs.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "cg_internal.cuh"
#include "cg_models.cuh"

namespace cg {
namespace {

// The shared scratch: per-tile partial sums of every call.  Every tile of a
// call overwrites its own slot before the finalize kernel reads it, so
// nothing needs clearing between calls; two calls running at the same time
// on the GPU would overwrite each other's partials.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CG_NOALLOC_SCRATCH_BYTES];

constexpr int kNT = 256;
constexpr int kNacc = MixAcc::N;  // 6 accumulators per parameter point
constexpr int kMaxDevices = 64;

// Accumulation: one partial vector (kNacc sums + a domain flag) per tile.
template <bool W>
__global__ void __launch_bounds__(kNT) k_mix_noalloc(MixData d, const double* __restrict__ theta, TileGrid tg,
                                                     double* __restrict__ part) {
    __shared__ MixConsts cs;
    __shared__ int cs_bad;
    __shared__ double red[kNacc * (kNT / 32)];
    __shared__ double tot[kNacc];
    for (int t = blockIdx.x; t < tg.n_tiles; t += gridDim.x) {
        const int th = t / tg.nbx, c = t - th * tg.nbx;
        if (threadIdx.x == 0) cs_bad = mix_prologue(theta + (size_t)th * 4, d.lo, d.hi, cs) ? 0 : 1;
        __syncthreads();
        double acc[kNacc];
#pragma unroll
        for (int a = 0; a < kNacc; ++a) acc[a] = 0.0;
        bool bad = false;
        const int64_t e0 = (int64_t)c * tg.chunk;
        const int64_t e1 = min(tg.n_elem, e0 + tg.chunk);
        for (int64_t i = e0 + threadIdx.x; i < e1; i += kNT)
            mix_elem_fp64<W>(d.x[i], W ? d.w[i] : 1.0, cs, acc, bad);
        const int any_bad = __syncthreads_or(bad ? 1 : 0) | cs_bad;
        block_sum<kNacc, kNT>(acc, red, tot);
        if (threadIdx.x == 0) {
            double* p = part + (size_t)th * (kNacc + 1) * tg.nbx + c;
            for (int a = 0; a < kNacc; ++a) p[(size_t)a * tg.nbx] = tot[a];
            p[(size_t)kNacc * tg.nbx] = any_bad ? 1.0 : 0.0;
        }
    }
}

// Finalize: one block per parameter point, partials summed in tile order,
// then the epilogue.  A flagged point gets a NaN value so the caller sees it.
__global__ void __launch_bounds__(128) k_mix_noalloc_finalize(const double* __restrict__ part, TileGrid tg,
                                                              EpiParams ep, const double* __restrict__ theta,
                                                              double* __restrict__ value,
                                                              double* __restrict__ grad) {
    __shared__ double tot[kNacc + 1];
    __shared__ double red[4];
    const int th = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int a = 0; a <= kNacc; ++a) {
        const double* p = part + ((size_t)th * (kNacc + 1) + a) * tg.nbx;
        double s = 0.0;
        for (int c = threadIdx.x; c < tg.nbx; c += 128) s += p[c];
        s = warp_sum(s);
        if (lane == 0) red[wid] = s;
        __syncthreads();
        if (threadIdx.x == 0) tot[a] = ((red[0] + red[1]) + red[2]) + red[3];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double g[4];
        const double v = epilogue(ep, theta + (size_t)th * 4, tot, g);
        value[th] = (tot[kNacc] != 0.0) ? __longlong_as_double(0x7ff8000000000000LL) : v;
        for (int k = 0; k < 4; ++k) grad[(size_t)th * 4 + k] = g[k];
    }
}

// Device address of the scratch array, looked up once per device with that
// device current (a host-side reference to the array is not a device address).
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

cg_status scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CG_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CG_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return CG_OK;
}

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" cg_status cg_mixture_gradient_noalloc(const cg_problem* pb, const double* theta, int64_t n_theta,
                                                 double* value, double* grad, void* stream) {
    if (!pb || pb->model != CG_MODEL_MIX_GAUSS_EXP || pb->objective != CG_OBJ_UNBINNED_NLL ||
        pb->precision != CG_PREC_FP64)
        return CG_ERR_INVALID_ARG;
    if (pb->n_events < 0 || (pb->n_events > 0 && !pb->data) || !(pb->hi[0] > pb->lo[0])) return CG_ERR_INVALID_ARG;
    if (!theta || !value || !grad || n_theta < 1) return CG_ERR_INVALID_ARG;
    if (n_theta > CG_NOALLOC_MAX_POINTS) return CG_ERR_INVALID_ARG;  // beyond what the scratch array holds

    void* scratch = nullptr;
    cg_status s = scratch_address(&scratch);
    if (s != CG_OK) return s;

    // Tile grid as for cg_batch_gradient, capped by the scratch capacity.
    const bool W = pb->weights != nullptr;
    const void* fn = W ? (const void*)k_mix_noalloc<true> : (const void*)k_mix_noalloc<false>;
    int R = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&R, fn, kNT, 0) != cudaSuccess || R < 1) R = 1;
    const int64_t G = (int64_t)device_sm_count() * R;
    const int64_t cap_doubles = CG_NOALLOC_SCRATCH_BYTES / sizeof(double);
    const int64_t nbx_cap = cap_doubles / ((kNacc + 1) * n_theta);
    const int64_t n = pb->n_events;
    int64_t nbx = (G * 4 + n_theta - 1) / n_theta;
    const int64_t most = (n + kNT * 8 - 1) / (kNT * 8);
    if (nbx > most) nbx = most;
    if (nbx > nbx_cap) nbx = nbx_cap;
    if (nbx < 1) nbx = 1;
    int64_t chunk = (n + nbx - 1) / nbx;
    chunk = (chunk + kNT - 1) / kNT * kNT;
    if (chunk < kNT) chunk = kNT;
    nbx = (n + chunk - 1) / chunk;
    if (nbx < 1) nbx = 1;

    TileGrid tg;
    tg.n_elem = n;
    tg.chunk = chunk;
    tg.nbx = (int)nbx;
    tg.n_theta = (int)n_theta;
    tg.n_tiles = (int)(n_theta * nbx);
    MixData d;
    d.x = pb->data;
    d.w = pb->weights;
    d.lo = pb->lo[0];
    d.hi = pb->hi[0];
    d.vec_ok = 0;
    EpiParams ep;
    ep.model = CG_MODEL_MIX_GAUSS_EXP;
    ep.P = 4;
    ep.K = 0;
    ep.D = 0;
    ep.lo = pb->lo[0];
    ep.hi = pb->hi[0];

    cudaStream_t st = (cudaStream_t)stream;
    double* part = (double*)scratch;
    const int grid = (int)(tg.n_tiles < G ? tg.n_tiles : G);
    if (W) k_mix_noalloc<true><<<grid, kNT, 0, st>>>(d, theta, tg, part);
    else k_mix_noalloc<false><<<grid, kNT, 0, st>>>(d, theta, tg, part);
    k_mix_noalloc_finalize<<<(unsigned)n_theta, 128, 0, st>>>(part, tg, ep, theta, value, grad);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}
