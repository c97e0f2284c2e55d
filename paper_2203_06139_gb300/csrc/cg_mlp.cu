// cg_mlp.cu -- BF16 tensor-core kernels of the learned-start network.
//
// GEMM: C[M, N] = sum_k A[m, k] B[n, k] with BF16 operands and FP32
// accumulation on the 5th-generation tensor cores: one elected thread issues
// tcgen05.mma (kind::f16, M = 128, N = BN) from shared-memory operands, the
// accumulator lives in tensor memory (TMEM, allocated per CTA), completion is
// signalled through an mbarrier, and the epilogue reads the accumulator with
// tcgen05.ld (warp w of the 4-warp CTA owns TMEM lanes 32w .. 32w + 31, i.e.
// rows 32w .. 32w + 31 of the tile).  Operands are staged K-major in the
// canonical no-swizzle layout of 8 x 16-byte core matrices; the loader
// transposes on the fly, so A and B may each be stored either way round.
// Every wait on the mbarrier is bounded by a clock budget; on timeout the
// kernel records an error, waits once more (bounded), frees its TMEM and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kTM = 128;          // tile rows (tcgen05 M)
constexpr int kKC = 64;           // K chunk staged per round (elements)
constexpr int kThreads = 128;     // 4 warps: one per 32 TMEM lanes
constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

enum { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_GELU = 2, EPI_GELU_GRAD = 3 };

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int M, N, K, lda, ldb, transA, transB;
    float* Cf;               // fp32 output (or nullptr)
    __nv_bfloat16* Cb;       // bf16 output (or nullptr)
    int ldc;
    const float* bias;       // [N]
    const float* aux_in;     // [M][ldc] pre-activations (EPI_GELU_GRAD)
    float* aux_out;          // [M][ldc] pre-activations written by EPI_BIAS_GELU
    int epi;
    int* err;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, descriptor
// version 1 in 46-47, layout (0 = no swizzle) in 61-63.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3fffu);
    d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// Stage rows [r0, r0 + R) x K-chunk [k0, k0 + kKC) of a K-major operand into
// the core-matrix layout: element (r, k) at (r/8)*SBO + (k/8)*128 + (r%8)*16 + (k%8)*2,
// SBO = (kKC/8)*128.  trans = 0: X[r*ld + k]; trans = 1: X[k*ld + r].
template <int R>
__device__ __forceinline__ void stage(uint8_t* dst, const __nv_bfloat16* X, int rows, int K, int ld, int trans,
                                      int r0, int k0) {
    constexpr int SBO = (kKC / 8) * 128;
    constexpr int PIECES = R * (kKC / 8);   // 16-byte pieces
    for (int p = threadIdx.x; p < PIECES; p += kThreads) {
        int r, kg;
        if (!trans) { r = p / (kKC / 8); kg = p % (kKC / 8); }
        else { r = p % R; kg = p / R; }
        const int gr = r0 + r, gk = k0 + kg * 8;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gr < rows) {
            if (!trans) {
                if (gk + 8 <= K && ((((uintptr_t)(X + (size_t)gr * ld + gk)) & 15) == 0)) {
                    v = *reinterpret_cast<const uint4*>(X + (size_t)gr * ld + gk);
                } else {
                    __nv_bfloat16 t[8];
                    for (int j = 0; j < 8; ++j) t[j] = (gk + j < K) ? X[(size_t)gr * ld + gk + j] : __float2bfloat16(0.0f);
                    v = *reinterpret_cast<uint4*>(t);
                }
            } else {
                __nv_bfloat16 t[8];
                for (int j = 0; j < 8; ++j) t[j] = (gk + j < K) ? X[(size_t)(gk + j) * ld + gr] : __float2bfloat16(0.0f);
                v = *reinterpret_cast<uint4*>(t);
            }
        }
        *reinterpret_cast<uint4*>(dst + (r / 8) * SBO + kg * 128 + (r % 8) * 16) = v;
    }
}

template <int BN>
__global__ void __launch_bounds__(kThreads) k_gemm_tc(GemmArgs g) {
    constexpr int SBO = (kKC / 8) * 128;
    constexpr int TCOLS = BN < 32 ? 32 : BN;            // TMEM columns (power of two >= 32)
    __shared__ __align__(128) uint8_t sA[kTM * kKC * 2];
    __shared__ __align__(128) uint8_t sB[BN * kKC * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * BN;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(&tmem_base)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t bar_a = smem_addr(&bar);
    constexpr uint32_t idesc = idesc_bf16(kTM, BN);
    bool ok = true;
    int nchunk = 0;

    for (int k0 = 0; k0 < g.K; k0 += kKC, ++nchunk) {
        stage<kTM>(sA, g.A, g.M, g.K, g.lda, g.transA, m0, k0);
        stage<BN>(sB, g.B, g.N, g.K, g.ldb, g.transB, n0, k0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
#pragma unroll
            for (int kk = 0; kk < kKC / 16; ++kk) {
                // each K = 16 step covers two core matrices along K (2 x 128 bytes)
                const uint64_t ad = sdesc(a0 + kk * 256, 128, SBO);
                const uint64_t bd = sdesc(b0 + kk * 256, 128, SBO);
                const uint32_t acc = (k0 > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(bar_a) : "memory");
        }
        const bool done = mbar_wait(bar_a, (uint32_t)(nchunk & 1));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ok = __syncthreads_and(done ? 1 : 0) != 0;   // one decision for the whole CTA
        if (!ok) break;
    }
    if (!ok) {
        if (g.err) atomicOr(g.err, 1);
        mbar_wait(bar_a, (uint32_t)(nchunk & 1));   // let the tensor core finish before TMEM is freed
    } else {
        // epilogue: warp w reads rows 32w..32w+31, 32 columns at a time
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            if (BN >= 32 || c0 == 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                      "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                      "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            }
            if (row < g.M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = n0 + c0 + j;
                    if (c0 + j >= BN || col >= g.N) continue;
                    float a = __uint_as_float(v[j]);
                    const size_t o = (size_t)row * g.ldc + col;
                    if (g.epi == EPI_F32) {
                        g.Cf[o] = a;
                    } else if (g.epi == EPI_BIAS_F32) {
                        g.Cf[o] = a + g.bias[col];
                    } else if (g.epi == EPI_BIAS_GELU) {
                        const float z = a + g.bias[col];
                        if (g.aux_out) g.aux_out[o] = z;
                        if (g.Cb) g.Cb[o] = __float2bfloat16(gelu(z));
                        if (g.Cf) g.Cf[o] = gelu(z);
                    } else {  // EPI_GELU_GRAD: a = upstream gradient of the activation
                        const float dz = a * gelu_grad(g.aux_in[o]);
                        if (g.Cb) g.Cb[o] = __float2bfloat16(dz);
                        if (g.Cf) g.Cf[o] = dz;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS) : "memory");
    }
}

template <int BN>
cg_status launch_gemm_bn(const GemmArgs& g, cudaStream_t st) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + kTM - 1) / kTM);
    k_gemm_tc<BN><<<grid, kThreads, 0, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

}  // namespace

cg_status gemm_bf16(const GemmArgs& g, cudaStream_t st) {
    if (!g.A || !g.B || g.M < 1 || g.N < 1 || g.K < 1) return CG_ERR_INVALID_ARG;
    if (g.epi < EPI_F32 || g.epi > EPI_GELU_GRAD) return CG_ERR_INVALID_ARG;
    if ((g.epi == EPI_F32 || g.epi == EPI_BIAS_F32) && !g.Cf) return CG_ERR_INVALID_ARG;
    if ((g.epi == EPI_BIAS_F32 || g.epi == EPI_BIAS_GELU) && !g.bias) return CG_ERR_INVALID_ARG;
    if (g.epi == EPI_GELU_GRAD && !g.aux_in) return CG_ERR_INVALID_ARG;
    if (g.N <= 16) return launch_gemm_bn<16>(g, st);
    if (g.N <= 64) return launch_gemm_bn<64>(g, st);
    return launch_gemm_bn<128>(g, st);
}

}  // namespace cg

using namespace cg;

extern "C" cg_status cg_gemm_bf16(const void* A, const void* B, int M, int N, int K, int lda, int ldb, int transA,
                                  int transB, float* Cf, void* Cb, int ldc, const float* bias, const float* aux_in,
                                  float* aux_out, int epilogue, int* err, void* stream) {
    GemmArgs g;
    g.A = (const __nv_bfloat16*)A;
    g.B = (const __nv_bfloat16*)B;
    g.M = M; g.N = N; g.K = K; g.lda = lda; g.ldb = ldb; g.transA = transA; g.transB = transB;
    g.Cf = Cf; g.Cb = (__nv_bfloat16*)Cb; g.ldc = ldc;
    g.bias = bias; g.aux_in = aux_in; g.aux_out = aux_out; g.epi = epilogue; g.err = err;
    return gemm_bf16(g, (cudaStream_t)stream);
}
