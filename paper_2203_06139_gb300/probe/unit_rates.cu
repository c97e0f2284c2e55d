// unit_rates.cu -- measures the arithmetic rates that set the ALU roofline of
// the fused kernels on the current GPU: FP64 FMA and add, the FP64 exp, log
// and reciprocal calls of the CUDA math library, and FP32 FMA.  Every kernel
// keeps its work in registers and writes one value per thread.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

template <int CH>
__global__ void k_dfma(double* out, int iters, double a, double b) {
    double c[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) c[j] = threadIdx.x * 1e-3 + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CH; ++j) c[j] = fma(c[j], a, b);
    }
    double s = 0;
#pragma unroll
    for (int j = 0; j < CH; ++j) s += c[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void k_ffma(double* out, int iters, float a, float b) {
    float c[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) c[j] = threadIdx.x * 1e-3f + j;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < CH; ++j) c[j] = fmaf(c[j], a, b);
    }
    float s = 0;
#pragma unroll
    for (int j = 0; j < CH; ++j) s += c[j];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_exp(double* out, int iters) {
    double x = -(threadIdx.x & 63) * 0.1 - 0.5, s = 0;
    for (int i = 0; i < iters; ++i) { s += exp(x); x -= 1e-7; }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_log(double* out, int iters) {
    double x = 1.5 + (threadIdx.x & 63) * 0.1, s = 0;
    for (int i = 0; i < iters; ++i) { s += log(x); x += 1e-7; }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rcp(double* out, int iters) {
    double x = 1.5 + (threadIdx.x & 63) * 0.1, s = 0;
    for (int i = 0; i < iters; ++i) { s += 1.0 / x; x += 1e-7; }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
float time_ms(F launch) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace

extern "C" {

// out[0] FP64 FMA/s, out[1] FP64 exp calls/s, out[2] FP64 log calls/s,
// out[3] FP64 reciprocal calls/s, out[4] FP32 FMA/s, out[5] SM count.
// scratch: device buffer of at least n_sm * 4 * 256 doubles.
int cgp_unit_rates(double* out, double* scratch) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = nsm * 4, th = 256;
    const double threads = (double)blocks * th;
    float ms;
    ms = time_ms([&] { k_dfma<8><<<blocks, th>>>(scratch, 2048, 1.0000001, 1e-9); });
    out[0] = 8.0 * 2048 * threads / (ms * 1e-3);
    ms = time_ms([&] { k_exp<<<blocks, th>>>(scratch, 512); });
    out[1] = 512 * threads / (ms * 1e-3);
    ms = time_ms([&] { k_log<<<blocks, th>>>(scratch, 512); });
    out[2] = 512 * threads / (ms * 1e-3);
    ms = time_ms([&] { k_rcp<<<blocks, th>>>(scratch, 512); });
    out[3] = 512 * threads / (ms * 1e-3);
    ms = time_ms([&] { k_ffma<8><<<blocks, th>>>(scratch, 8192, 1.0000001f, 1e-9f); });
    out[4] = 8.0 * 8192 * threads / (ms * 1e-3);
    out[5] = nsm;
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
