// Test helper: evaluates the FP64 functions of cg_fp64.cuh next to the CUDA
// math library's and IEEE division on device arrays (compiled by
// tests/test_gpu_fp64_math.py).  One thread per input; every index is
// checked against n.
#include <cuda_runtime.h>

#include "../../paper_2203_06139_gb300/csrc/cg_fp64.cuh"

using namespace cg;

namespace {

__global__ void k_check(const double* __restrict__ y, const double* __restrict__ p, int n, double* __restrict__ out) {
    __shared__ Fp64Tab tab;
    fp64_tab_load(tab);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double* o = out + (size_t)i * 6;
    o[0] = fexp2(y[i], tab);
    o[1] = exp2(y[i]);
    o[2] = frcp_any(p[i]);
    o[3] = 1.0 / p[i];
    o[4] = flog(p[i], tab);
    o[5] = log(p[i]);
}

// Sum of the logs of p[64 g .. 64 g + 63] through the running product.
__global__ void k_logprod(const double* __restrict__ p, int groups, double* __restrict__ out) {
    __shared__ Fp64Tab tab;
    fp64_tab_load(tab);
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= groups) return;
    LogProd s;
    logprod_init(s);
    for (int k = 0; k < 64; ++k) logprod_mul(s, p[(size_t)g * 64 + k]);
    out[g] = logprod_log(s, tab);
}

// 2^(a b) through the product folded into the reduction, and CUDA's exp2 of
// the rounded product beside it.
__global__ void k_exp2_prod(const double* __restrict__ a, const double* __restrict__ b, int n,
                            double* __restrict__ out) {
    __shared__ Fp64Tab tab;
    fp64_tab_load(tab);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[2 * (size_t)i] = fexp2_prod(a[i], b[i], tab);
    out[2 * (size_t)i + 1] = exp2(a[i] * b[i]);
}

}  // namespace

extern "C" int fp64_exp2_prod(const double* a, const double* b, int n, double* out) {
    k_exp2_prod<<<(n + 255) / 256, 256>>>(a, b, n, out);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}

extern "C" int fp64_check(const double* y, const double* p, int n, double* out) {
    k_check<<<(n + 255) / 256, 256>>>(y, p, n, out);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}

extern "C" int fp64_logprod(const double* p, int groups, double* out) {
    k_logprod<<<(groups + 127) / 128, 128>>>(p, groups, out);
    if (cudaGetLastError() != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 2;
}
