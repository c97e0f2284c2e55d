// unit_rates.cu -- measures the peak arithmetic rates that bench.py sets its
// ALU rooflines against: FP64 FMA (the FP64 pipe of the FP64 kernels) and
// FP32 FMA (the FP32 pipe of the double-float kernels).  Eight independent
// FMA chains per thread, four 256-thread blocks per SM, work in registers,
// one value written per thread.  Built by bench.py (nvcc, sm_103a).
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

// out[0] FP64 FMA instructions/s (thread-level), out[1] FP32 FMA/s, out[2]
// SM count.  scratch: device buffer of at least n_sm * 4 * 256 doubles.
int cgp_unit_rates(double* out, double* scratch) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = nsm * 4, th = 256;
    const double threads = (double)blocks * th;
    float ms = time_ms([&] { k_dfma<8><<<blocks, th>>>(scratch, 2048, 1.0000001, 1e-9); });
    out[0] = 8.0 * 2048 * threads / (ms * 1e-3);
    ms = time_ms([&] { k_ffma<8><<<blocks, th>>>(scratch, 8192, 1.0000001f, 1e-9f); });
    out[1] = 8.0 * 8192 * threads / (ms * 1e-3);
    out[2] = nsm;
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
