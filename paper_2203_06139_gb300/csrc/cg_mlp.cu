// cg_mlp.cu -- BF16 tensor-core kernels of the learned-start network.
//
// GEMM: C[M, N] = sum_k A[m, k] B[n, k] with BF16 operands and FP32
// accumulation on the 5th-generation tensor cores: one elected thread issues
// tcgen05.mma (kind::f16, M = 128, N = BN) from shared-memory operands, the
// accumulator lives in tensor memory (TMEM, allocated per CTA), completion is
// signalled through mbarriers, and the epilogue reads the accumulator with
// tcgen05.ld (a warp owns the 32 TMEM lanes of its quarter, i.e. 32 rows of
// the tile).  Three kernels:
//  k_gemm_persist  K-major operands, N >= 128: persistent, TMA loads into a
//                  4-stage ring, two TMEM accumulators (epilogue of one tile
//                  overlaps the MMAs of the next);
//  k_gemm_pipe     K-major operands, N < 128: the same TMA ring, one tile per
//                  CTA;
//  k_gemm_tc       anything else: operands staged through registers into the
//                  canonical no-swizzle layout (8 x 16-byte core matrices),
//                  transposed on the fly, so A and B may be stored either way.
// Every wait on an mbarrier is bounded by a clock budget; on timeout the
// kernel records an error, lets its issued copies and MMAs finish (bounded),
// frees its TMEM and returns.
#include <algorithm>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
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

// ---------------------------------------------------------------------------
// Pipelined GEMM for K-major A [M][lda] and B [N][ldb]: the tensor memory
// accelerator (TMA) loads 128 x 64 and BN x 64 tiles with 128-byte swizzle
// into a ring of kStages shared-memory stages (full / empty mbarriers per
// stage); one thread issues tcgen05.mma (M = 128, N = BN, K = 16 per
// instruction) into a 128 x BN FP32 accumulator in tensor memory; four
// epilogue warps read it back with tcgen05.ld, stage 32 x 32 blocks through
// shared memory and apply the epilogue with loads and stores coalesced along
// the columns.  Warp 0 = TMA producer, warp 1 = TMEM owner and MMA issuer,
// warps 2-5 = epilogue (warp w may read TMEM lanes 32 (w % 4) .. + 31).
// Every mbarrier wait is bounded; a wait that gives up sets a shared abort
// flag and bit 0 of *err, the other roles stop at their next wait, and the
// CTA lets its issued loads and MMAs finish (bounded) before freeing TMEM.
// ---------------------------------------------------------------------------
constexpr int kStages = 3;
constexpr int kPipeThreads = 192;
constexpr int kBK = 64;                      // 64 bf16 = one 128-byte swizzle row
constexpr int kEpiLd = 33;                   // staging row stride (floats), conflict-free

template <int BN>
struct PipeSmem {
    static constexpr int A_BYTES = kTM * kBK * 2;
    static constexpr int B_BYTES = BN * kBK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;   // a multiple of 1024: every tile 1024-aligned
    static constexpr int PIPE = kStages * STAGE;
    static constexpr int EPI = 4 * 32 * kEpiLd * 4;   // epilogue staging, reuses the stage buffers
    static constexpr int BUF = PIPE > EPI ? PIPE : EPI;
    static constexpr int BARS = (2 * kStages + 1) * 8;
    static constexpr int TOTAL = 1024 + BUF + BARS + 16;
    static_assert(STAGE % 1024 == 0 && A_BYTES % 1024 == 0, "swizzle atoms need 1024-byte aligned tiles");
};

// Shared-memory descriptor of a K-major tile in the 128-byte swizzle layout
// written by TMA: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO);
// the leading offset is not used by this layout; version 1; layout 2
// (128-byte swizzle).  A K = 16 step inside the row advances the start
// address by 32 bytes.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3fffu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool pipe_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    const long long t0 = clock64();
    for (int it = 0;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 63 && (*abort_flag || clock64() - t0 > kWaitCycles)) return false;
    }
}

__device__ __forceinline__ void pipe_fail(volatile int* abort_flag, int* err) {
    *abort_flag = 1;
    if (err) atomicOr(err, 1);
}

template <int BN>
__global__ void __launch_bounds__(kPipeThreads) k_gemm_pipe(const __grid_constant__ CUtensorMap tmA,
                                                            const __grid_constant__ CUtensorMap tmB, GemmArgs g) {
    using L = PipeSmem<BN>;
    constexpr int TCOLS = BN < 32 ? 32 : BN;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::BUF);   // full[S], empty[S], acc
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t sbase = smem_addr(smem);
    const uint32_t bar0 = smem_addr(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (uint32_t)(kStages + s); };
    const uint32_t acc_bar = bar0 + 8u * (uint32_t)(2 * kStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * BN;
    const int nk = (g.K + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(full_bar(s)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(empty_bar(s)) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(acc_bar) : "memory");
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(tmem_slot)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    int issued = 0;   // producer: loads issued

    if (warp == 0) {
        if (lane == 0) {
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % kStages;
                if (kc >= kStages && !pipe_wait(empty_bar(s), (uint32_t)((kc / kStages - 1) & 1), abort_flag)) {
                    pipe_fail(abort_flag, g.err);
                    break;
                }
                const uint32_t a_dst = sbase + (uint32_t)(s * L::STAGE), b_dst = a_dst + (uint32_t)L::A_BYTES;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             :: "r"(full_bar(s)), "r"((uint32_t)L::STAGE) : "memory");
                asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                             " [%0], [%1, {%2, %3}], [%4];"
                             :: "r"(a_dst), "l"((uint64_t)&tmA), "r"(kc * kBK), "r"(m0), "r"(full_bar(s))
                             : "memory");
                asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                             " [%0], [%1, {%2, %3}], [%4];"
                             :: "r"(b_dst), "l"((uint64_t)&tmB), "r"(kc * kBK), "r"(n0), "r"(full_bar(s))
                             : "memory");
                issued = kc + 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kTM, BN);
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % kStages;
                if (!pipe_wait(full_bar(s), (uint32_t)((kc / kStages) & 1), abort_flag)) {
                    pipe_fail(abort_flag, g.err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = sbase + (uint32_t)(s * L::STAGE), b0 = a0 + (uint32_t)L::A_BYTES;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                    const uint64_t ad = sdesc_sw128(a0 + 32u * (uint32_t)kk);
                    const uint64_t bd = sdesc_sw128(b0 + 32u * (uint32_t)kk);
                    const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                        :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(empty_bar(s)) : "memory");
            }
            // the accumulator barrier completes once every MMA issued above has
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(acc_bar) : "memory");
        }
    } else {
        const int q = warp & 3;                         // TMEM lane quarter of this warp
        float* stg = reinterpret_cast<float*>(smem) + (warp - 2) * 32 * kEpiLd;
        const bool ok = pipe_wait(acc_bar, 0u, abort_flag) && !*abort_flag;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // the staging area was last written by TMA (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!ok) {
            if (lane == 0) pipe_fail(abort_flag, g.err);
        } else {
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
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
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane * kEpiLd + j] = __uint_as_float(v[j]);
                __syncwarp();
                const int col = n0 + c0 + lane;
                const bool col_ok = (c0 + lane < BN) && col < g.N;
                float bv = 0.0f;
                if (col_ok && (g.epi == EPI_BIAS_F32 || g.epi == EPI_BIAS_GELU)) bv = g.bias[col];
                for (int r = 0; r < 32; ++r) {
                    const int row = m0 + q * 32 + r;
                    if (row >= g.M || !col_ok) continue;
                    const float a = stg[r * kEpiLd + lane];
                    const size_t o = (size_t)row * g.ldc + col;
                    if (g.epi == EPI_F32) {
                        g.Cf[o] = a;
                    } else if (g.epi == EPI_BIAS_F32) {
                        g.Cf[o] = a + bv;
                    } else if (g.epi == EPI_BIAS_GELU) {
                        const float z = a + bv;
                        const float h = gelu(z);
                        if (g.aux_out) g.aux_out[o] = z;
                        if (g.Cb) g.Cb[o] = __float2bfloat16(h);
                        if (g.Cf) g.Cf[o] = h;
                    } else {
                        const float dz = a * gelu_grad(g.aux_in[o]);
                        if (g.Cb) g.Cb[o] = __float2bfloat16(dz);
                        if (g.Cf) g.Cf[o] = dz;
                    }
                }
                __syncwarp();
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag) {
        // let issued loads and MMAs finish before the shared memory and TMEM go away
        if (warp == 0 && lane == 0) {
            for (int kc = issued - kStages < 0 ? 0 : issued - kStages; kc < issued; ++kc) {
                const long long t0 = clock64();
                while (!mbar_try(full_bar(kc % kStages), (uint32_t)((kc / kStages) & 1)) &&
                       clock64() - t0 < kWaitCycles) {
                }
            }
        }
        if (warp == 1 && lane == 0) {
            const long long t0 = clock64();
            while (!mbar_try(acc_bar, 0u) && clock64() - t0 < kWaitCycles) {
            }
        }
        __syncthreads();
    }
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Persistent TMA + tcgen05 GEMM for N >= 128 (K-major operands): one CTA per
// SM walks output tiles t = blockIdx.x, + gridDim.x, ... (N-tiles fastest).
// Warp 0 = TMA producer over a kPStages ring that runs across tiles; warp 1 =
// TMEM owner and MMA issuer into two accumulators of BN columns each (tile i
// uses accumulator i & 1); warps 2-9 = epilogue, which drains accumulator
// i & 1 while the MMAs of tile i + 1 go into the other.  A warp reads the
// TMEM lanes of its quarter (warp % 4), so two warps share each quarter and
// take half of the tile's columns each: with bias + GELU in the epilogue
// (an erf per element) four warps per SM were the bottleneck of the
// network's layers.  Barriers: full / empty per stage, acc_full (one
// tcgen05.commit per tile) and acc_empty (one arrival per epilogue warp)
// per accumulator.  Every wait is bounded;
// on a failed wait all roles stop, the producer waits (bounded) for its
// issued loads and the MMA thread for a final commit before TMEM is freed.
// ---------------------------------------------------------------------------
constexpr int kPStages = 4;
constexpr int kEpiWarps = 8;                                 // two per TMEM lane quarter
constexpr int kPersistThreads = 32 * (2 + kEpiWarps);        // producer, MMA, epilogue

template <int BN>
struct PersistSmem {
    static constexpr int A_BYTES = kTM * kBK * 2;
    static constexpr int B_BYTES = BN * kBK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int PIPE = kPStages * STAGE;
    static constexpr int XPOSE = kEpiWarps * 32 * 32 * 4;   // one 32 x 32 FP32 block per epilogue warp
    static constexpr int NBARS = 2 * kPStages + 5;   // full, empty, acc_full[2], acc_empty[2], drain
    static constexpr int TOTAL = 1024 + PIPE + XPOSE + NBARS * 8 + 16;
    static_assert(STAGE % 1024 == 0 && A_BYTES % 1024 == 0, "swizzle atoms need 1024-byte aligned tiles");
    static_assert(TOTAL <= 227 * 1024, "shared memory per CTA");
    static_assert(BN % 64 == 0, "two epilogue warps per lane quarter take BN / 2 columns each, in steps of 32");
};

// One accumulator row segment (columns col0 .. col0 + 31 of row `row`, the
// 32 values tcgen05.ld gave this lane) through the epilogue of g, straight
// from registers: 16-byte stores when the segment is inside N and every
// operand is 16-byte aligned with ldc a multiple of 8, else element by element.
__device__ __forceinline__ void epi_segment(const GemmArgs& g, const uint32_t (&v)[32], int row, int col0, bool vec) {
    if (row >= g.M) return;
    const size_t o = (size_t)row * g.ldc + col0;
    if (vec) {
#pragma unroll
        for (int j = 0; j < 32; j += 8) {
            float a[8], z[8], r[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) a[e] = __uint_as_float(v[j + e]);
            if (g.epi == EPI_F32) {
#pragma unroll
                for (int e = 0; e < 8; ++e) r[e] = a[e];
            } else if (g.epi == EPI_BIAS_F32 || g.epi == EPI_BIAS_GELU) {
                const float4 b0 = *reinterpret_cast<const float4*>(g.bias + col0 + j);
                const float4 b1 = *reinterpret_cast<const float4*>(g.bias + col0 + j + 4);
                const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    z[e] = a[e] + bb[e];
                    r[e] = g.epi == EPI_BIAS_GELU ? gelu(z[e]) : z[e];
                }
                if (g.epi == EPI_BIAS_GELU && g.aux_out) {
                    *reinterpret_cast<float4*>(g.aux_out + o + j) = make_float4(z[0], z[1], z[2], z[3]);
                    *reinterpret_cast<float4*>(g.aux_out + o + j + 4) = make_float4(z[4], z[5], z[6], z[7]);
                }
            } else {
                const float4 z0 = *reinterpret_cast<const float4*>(g.aux_in + o + j);
                const float4 z1 = *reinterpret_cast<const float4*>(g.aux_in + o + j + 4);
                const float zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
                for (int e = 0; e < 8; ++e) r[e] = a[e] * gelu_grad(zz[e]);
            }
            if (g.Cf) {
                *reinterpret_cast<float4*>(g.Cf + o + j) = make_float4(r[0], r[1], r[2], r[3]);
                *reinterpret_cast<float4*>(g.Cf + o + j + 4) = make_float4(r[4], r[5], r[6], r[7]);
            }
            if (g.Cb && g.epi != EPI_F32 && g.epi != EPI_BIAS_F32) {
                __nv_bfloat162 p[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) p[e] = __floats2bfloat162_rn(r[2 * e], r[2 * e + 1]);
                *reinterpret_cast<uint4*>(g.Cb + o + j) = *reinterpret_cast<const uint4*>(p);
            }
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int col = col0 + j;
        if (col >= g.N) continue;
        const float a = __uint_as_float(v[j]);
        const size_t oj = o + j;
        if (g.epi == EPI_F32) {
            g.Cf[oj] = a;
        } else if (g.epi == EPI_BIAS_F32) {
            g.Cf[oj] = a + g.bias[col];
        } else if (g.epi == EPI_BIAS_GELU) {
            const float z = a + g.bias[col];
            const float h = gelu(z);
            if (g.aux_out) g.aux_out[oj] = z;
            if (g.Cb) g.Cb[oj] = __float2bfloat16(h);
            if (g.Cf) g.Cf[oj] = h;
        } else {
            const float dz = a * gelu_grad(g.aux_in[oj]);
            if (g.Cb) g.Cb[oj] = __float2bfloat16(dz);
            if (g.Cf) g.Cf[oj] = dz;
        }
    }
}

// A 32 x 32 FP32 block (lane l holds row row0 + l, columns col0 .. col0 + 31,
// bias already added) stored with whole 128-byte rows per 8 lanes: the rows
// go through this warp's 4 KB buffer, float4 slot c of row r kept at
// c ^ (r & 7) so that both the writes and the reads are free of bank
// conflicts; then each store instruction writes 4 full rows.
__device__ __forceinline__ void store_block_f32(float* C, int ldc, int M, int row0, int col0, const float (&a)[32],
                                                float4* buf, int lane) {
#pragma unroll
    for (int c = 0; c < 8; ++c)
        buf[lane * 8 + (c ^ (lane & 7))] = make_float4(a[4 * c], a[4 * c + 1], a[4 * c + 2], a[4 * c + 3]);
    __syncwarp();
    const int c = lane & 7;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int r = 4 * k + (lane >> 3);
        const float4 val = buf[r * 8 + (c ^ (r & 7))];
        if (row0 + r < M) *reinterpret_cast<float4*>(C + (size_t)(row0 + r) * ldc + col0 + 4 * c) = val;
    }
    __syncwarp();
}

// The same for a BF16 output (64 bytes per row): 16-byte slot c of row r kept
// at c ^ ((r >> 1) & 3) of the row's 4 (conflict-free both ways); each store
// instruction writes 8 rows of 64 bytes.
__device__ __forceinline__ void store_block_bf16(__nv_bfloat16* C, int ldc, int M, int row0, int col0,
                                                 const float (&a)[32], float4* buf, int lane) {
    uint4* b16 = reinterpret_cast<uint4*>(buf);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        __nv_bfloat162 p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) p[e] = __floats2bfloat162_rn(a[8 * c + 2 * e], a[8 * c + 2 * e + 1]);
        b16[lane * 4 + (c ^ ((lane >> 1) & 3))] = *reinterpret_cast<const uint4*>(p);
    }
    __syncwarp();
    const int c = lane & 3;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int r = 8 * k + (lane >> 2);
        const uint4 val = b16[r * 4 + (c ^ ((r >> 1) & 3))];
        if (row0 + r < M) *reinterpret_cast<uint4*>(C + (size_t)(row0 + r) * ldc + col0 + 8 * c) = val;
    }
    __syncwarp();
}

template <int BN>
__global__ void __launch_bounds__(kPersistThreads, 1) k_gemm_persist(const __grid_constant__ CUtensorMap tmA,
                                                                  const __grid_constant__ CUtensorMap tmB,
                                                                  GemmArgs g) {
    using L = PersistSmem<BN>;
    constexpr int TCOLS = 2 * BN;   // two accumulators
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    uint8_t* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    float4* xpose_all = reinterpret_cast<float4*>(smem + L::PIPE);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::PIPE + L::XPOSE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + L::NBARS);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const uint32_t sbase = smem_addr(smem);
    const uint32_t bar0 = smem_addr(bars);
    auto full_bar = [&](int st) { return bar0 + 8u * (uint32_t)st; };
    auto empty_bar = [&](int st) { return bar0 + 8u * (uint32_t)(kPStages + st); };
    auto accf_bar = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kPStages + b); };
    auto acce_bar = [&](int b) { return bar0 + 8u * (uint32_t)(2 * kPStages + 2 + b); };
    const uint32_t drain_bar = bar0 + 8u * (uint32_t)(2 * kPStages + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = (g.K + kBK - 1) / kBK;
    const int ntn = (g.N + BN - 1) / BN;
    const int n_tiles = ntn * ((g.M + kTM - 1) / kTM);

    if (threadIdx.x == 0) {
        for (int st = 0; st < kPStages; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(full_bar(st)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(empty_bar(st)) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(accf_bar(b)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(acce_bar(b)), "r"(kEpiWarps) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(drain_bar) : "memory");
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_addr(tmem_slot)), "r"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    int issued = 0;     // producer: chunks whose loads were issued
    bool mma_any = false;

    if (warp == 0) {
        if (lane == 0) {
            int c = 0;
            for (int t = blockIdx.x; t < n_tiles && !*abort_flag; t += gridDim.x) {
                const int m0 = (t / ntn) * kTM, n0 = (t % ntn) * BN;
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int st = c % kPStages;
                    if (c >= kPStages && !pipe_wait(empty_bar(st), (uint32_t)((c / kPStages - 1) & 1), abort_flag)) {
                        pipe_fail(abort_flag, g.err);
                        ok = false;
                        break;
                    }
                    const uint32_t a_dst = sbase + (uint32_t)(st * L::STAGE), b_dst = a_dst + (uint32_t)L::A_BYTES;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 :: "r"(full_bar(st)), "r"((uint32_t)L::STAGE) : "memory");
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];"
                                 :: "r"(a_dst), "l"((uint64_t)&tmA), "r"(kc * kBK), "r"(m0), "r"(full_bar(st))
                                 : "memory");
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];"
                                 :: "r"(b_dst), "l"((uint64_t)&tmB), "r"(kc * kBK), "r"(n0), "r"(full_bar(st))
                                 : "memory");
                    issued = c + 1;
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kTM, BN);
            int c = 0, i = 0;
            for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
                const int b = i & 1;
                if (i >= 2 && !pipe_wait(acce_bar(b), (uint32_t)(((i >> 1) - 1) & 1), abort_flag)) {
                    pipe_fail(abort_flag, g.err);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dt = tmem + (uint32_t)(b * BN);
                bool ok = true;
                for (int kc = 0; kc < nk; ++kc, ++c) {
                    const int st = c % kPStages;
                    if (!pipe_wait(full_bar(st), (uint32_t)((c / kPStages) & 1), abort_flag)) {
                        pipe_fail(abort_flag, g.err);
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = sbase + (uint32_t)(st * L::STAGE), b0 = a0 + (uint32_t)L::A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t ad = sdesc_sw128(a0 + 32u * (uint32_t)kk);
                        const uint64_t bd = sdesc_sw128(b0 + 32u * (uint32_t)kk);
                        const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                            :: "r"(dt), "l"(ad), "l"(bd), "r"(idesc), "r"(acc) : "memory");
                    }
                    mma_any = true;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(empty_bar(st)) : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(accf_bar(b)) : "memory");
            }
        }
    } else {
        const int q = warp & 3;                         // TMEM lane quarter of this warp
        const int cb = ((warp - 2) >> 2) * (BN / 2), ce = cb + BN / 2;   // its half of the columns
        auto al16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
        const bool aligned = g.ldc % 8 == 0 && al16(g.Cf) && al16(g.Cb) && al16(g.aux_in) && al16(g.aux_out) &&
                             al16(g.bias);
        int i = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++i) {
            const int b = i & 1;
            const bool ok = pipe_wait(accf_bar(b), (uint32_t)((i >> 1) & 1), abort_flag) && !*abort_flag;
            if (!ok) {
                if (lane == 0) pipe_fail(abort_flag, g.err);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (t / ntn) * kTM, n0 = (t % ntn) * BN;
            for (int c0 = cb; c0 < ce; c0 += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + c0);
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
                if (c0 + 32 >= ce) {
                    // this warp's part of the accumulator is in registers or stored: hand it back
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(acce_bar(b)) : "memory");
                }
                const int col0 = n0 + c0;
                if (col0 >= g.N) continue;
                const bool vec = aligned && col0 + 32 <= g.N;
                if (vec && g.epi != EPI_GELU_GRAD) {
                    float4* xb = xpose_all + (warp - 2) * 256;
                    float a[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) a[j] = __uint_as_float(v[j]);
                    if (g.epi != EPI_F32) {   // + bias
#pragma unroll
                        for (int j = 0; j < 32; j += 4) {
                            const float4 bb = *reinterpret_cast<const float4*>(g.bias + col0 + j);
                            a[j] += bb.x;
                            a[j + 1] += bb.y;
                            a[j + 2] += bb.z;
                            a[j + 3] += bb.w;
                        }
                    }
                    const int row0 = m0 + q * 32;
                    if (g.epi == EPI_BIAS_GELU) {
                        if (g.aux_out) store_block_f32(g.aux_out, g.ldc, g.M, row0, col0, a, xb, lane);
#pragma unroll
                        for (int j = 0; j < 32; ++j) a[j] = gelu(a[j]);
                        if (g.Cb) store_block_bf16(g.Cb, g.ldc, g.M, row0, col0, a, xb, lane);
                    }
                    if (g.Cf) store_block_f32(g.Cf, g.ldc, g.M, row0, col0, a, xb, lane);
                } else {
                    epi_segment(g, v, m0 + q * 32 + lane, col0, vec);
                }
            }
        }
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag) {
        // let issued loads and MMAs finish before the shared memory and TMEM go away
        if (warp == 0 && lane == 0) {
            for (int c = issued - kPStages < 0 ? 0 : issued - kPStages; c < issued; ++c) {
                const long long t0 = clock64();
                while (!mbar_try(full_bar(c % kPStages), (uint32_t)((c / kPStages) & 1)) &&
                       clock64() - t0 < kWaitCycles) {
                }
            }
        }
        if (warp == 1 && lane == 0 && mma_any) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(drain_bar) : "memory");
            const long long t0 = clock64();
            while (!mbar_try(drain_bar, 0u) && clock64() - t0 < kWaitCycles) {
            }
        }
        __syncthreads();
    }
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS) : "memory");
    }
}

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point query.
PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }();
    return fn;
}

// 2-D tensor map of a K-major bf16 matrix [rows][ld] (K = inner), box 64 x box_rows,
// 128-byte swizzle, out-of-range elements read as zero.
bool make_tmap(CUtensorMap* m, const void* ptr, int K, int rows, int ld, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cg_status launch_gemm_pipe(const GemmArgs& g, cudaStream_t st) {
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, g.A, g.K, g.M, g.lda, kTM) || !make_tmap(&tb, g.B, g.K, g.N, g.ldb, BN))
        return CG_ERR_UNSUPPORTED;
    using L = PipeSmem<BN>;
    if (cudaFuncSetAttribute(k_gemm_pipe<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL) != cudaSuccess)
        return CG_ERR_CUDA;
    const dim3 grid((g.N + BN - 1) / BN, (g.M + kTM - 1) / kTM);
    k_gemm_pipe<BN><<<grid, kPipeThreads, L::TOTAL, st>>>(ta, tb, g);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

template <int BN>
cg_status launch_gemm_persist(const GemmArgs& g, cudaStream_t st) {
    CUtensorMap ta, tb;
    if (!make_tmap(&ta, g.A, g.K, g.M, g.lda, kTM) || !make_tmap(&tb, g.B, g.K, g.N, g.ldb, BN))
        return CG_ERR_UNSUPPORTED;
    using L = PersistSmem<BN>;
    if (cudaFuncSetAttribute(k_gemm_persist<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL) !=
        cudaSuccess)
        return CG_ERR_CUDA;
    const long long tiles = (long long)((g.N + BN - 1) / BN) * ((g.M + kTM - 1) / kTM);
    if (tiles >= INT32_MAX) return CG_ERR_UNSUPPORTED;   // the kernel counts tiles in int
    const int sms = device_sm_count();
    const int grid = (int)(tiles < sms ? tiles : sms);   // one CTA per SM (shared memory and TMEM)
    k_gemm_persist<BN><<<grid, kPersistThreads, L::TOTAL, st>>>(ta, tb, g);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
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
    // K-major operands with 16-byte aligned rows: the TMA pipeline
    const bool pipe = !g.transA && !g.transB && g.lda % 8 == 0 && g.ldb % 8 == 0 && g.lda >= g.K && g.ldb >= g.K &&
                      ((uintptr_t)g.A & 15) == 0 && ((uintptr_t)g.B & 15) == 0 && g.M < (1 << 30) &&
                      g.N < (1 << 30) && g.M <= 65535 * kTM;
    if (pipe) {
        cg_status r;
        if (g.N >= 256) r = launch_gemm_persist<256>(g, st);
        else if (g.N >= 128) r = launch_gemm_persist<128>(g, st);
        else if (g.N > 32) r = launch_gemm_pipe<64>(g, st);
        else if (g.N > 16) r = launch_gemm_pipe<32>(g, st);
        else r = launch_gemm_pipe<16>(g, st);
        if (r != CG_ERR_UNSUPPORTED) return r;
    }
    if (g.N <= 16) return launch_gemm_bn<16>(g, st);
    if (g.N <= 64) return launch_gemm_bn<64>(g, st);
    return launch_gemm_bn<128>(g, st);
}

// Failure detection: the bounded wait of the GEMM pipelines (pipe_wait,
// pipe_fail) on an mbarrier that nothing ever completes.  The wait gives up
// after kWaitCycles, sets bit 0 of err and the kernel returns: nothing is in
// flight, so the context stays usable.
__global__ void k_wait_check(int* err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    const uint32_t b = smem_addr(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b) : "memory");
    abort_flag = 0;
    // phase 0 completes on one arrival, which never comes
    if (!pipe_wait(b, 0u, &abort_flag)) pipe_fail(&abort_flag, err);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(b) : "memory");
}

}  // namespace cg

using namespace cg;

extern "C" cg_status cg_check_wait_timeout(int* err, void* stream) {
    if (!err) return CG_ERR_INVALID_ARG;
    k_wait_check<<<1, 32, 0, (cudaStream_t)stream>>>(err);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

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

// ===========================================================================
// Learned-start helpers: rebinning, heuristic start, loss, sums, optimiser
// ===========================================================================
namespace cg {
namespace {

// One warp per histogram for the rebinning and the heuristic start; shared
// memory per warp: the rebinned sums (rebin) or sums + smoothed sums
// (heuristic).
constexpr int kHistWarps = 4;

// x[h][j] = bf16(r_j / max_j r_j), r_j = sum of `factor` consecutive counts
// (added in order); scale[h] = max_j r_j (1 when the histogram is empty).
__global__ void k_rebin(const double* __restrict__ y, int64_t H, int n_bins, int factor, __nv_bfloat16* x,
                        float* scale) {
    extern __shared__ double sr_all[];
    const int nr = n_bins / factor;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* sr = sr_all + (size_t)wid * nr;
    for (int64_t h = (int64_t)blockIdx.x * nw + wid; h < H; h += (int64_t)gridDim.x * nw) {
        const double* yh = y + h * (int64_t)n_bins;
        double m = 0.0;
        for (int j = lane; j < nr; j += 32) {
            double t = 0.0;
            for (int i = 0; i < factor; ++i) t += yh[j * factor + i];
            sr[j] = t;
            m = fmax(m, t);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        const double mx = m > 0.0 ? m : 1.0;
        const double inv = 1.0 / mx;
        if (lane == 0) scale[h] = (float)mx;
        __syncwarp();
        for (int j = lane; j < nr; j += 32) x[h * nr + j] = __float2bfloat16((float)(sr[j] * inv));
        __syncwarp();
    }
}

// First index of the minimum of v[j0 .. j1) over the warp (all lanes get it).
__device__ __forceinline__ int warp_argmin_first(const double* v, int j0, int j1) {
    const int lane = threadIdx.x & 31;
    int bj = -1;
    double bv = 0.0;
    for (int j = j0 + lane; j < j1; j += 32)
        if (bj < 0 || v[j] < bv) { bv = v[j]; bj = j; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (oj >= 0 && (bj < 0 || ov < bv || (ov == bv && oj < bj))) { bv = ov; bj = oj; }
    }
    return bj;
}

// Heuristic starting point for K Gaussian peaks on a linear background, from
// the rebinned histogram (sums of `factor` counts, in order): 5-bin box
// smoothing; background = line through the minima (first index of the
// minimum) of the first and last eighth; peaks = the K highest local maxima
// of the smoothed residual (first index on ties), each closer than 3 rebinned
// bins to no earlier peak; amplitude = residual height; width from the
// half-maximum crossings.  One warp per histogram.  Output per original bin:
// theta = (A_1, mu_1, s_1, ..., A_K, mu_K, s_K, b0, b1), peaks sorted by mu.
__global__ void k_heuristic(const double* __restrict__ y, int64_t H, int n_bins, int factor, double lo, double hi,
                            int K, double* theta) {
    extern __shared__ double sm_all[];
    const int nr = n_bins / factor;
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* r = sm_all + (size_t)wid * 2 * nr;
    double* s = r + nr;
    const double wr = (hi - lo) / nr;        // rebinned bin width
    for (int64_t h = (int64_t)blockIdx.x * nw + wid; h < H; h += (int64_t)gridDim.x * nw) {
        const double* yh = y + h * (int64_t)n_bins;
        for (int j = lane; j < nr; j += 32) {
            double t = 0.0;
            for (int i = 0; i < factor; ++i) t += yh[j * factor + i];
            r[j] = t;
        }
        __syncwarp();
        for (int j = lane; j < nr; j += 32) {
            double t = 0.0;
            int c = 0;
            for (int q = j - 2; q <= j + 2; ++q)
                if (q >= 0 && q < nr) { t += r[q]; ++c; }
            s[j] = t / c;
        }
        __syncwarp();
        const int seg = nr / 8 > 1 ? nr / 8 : 1;
        const int jl = warp_argmin_first(s, 0, seg), jr = warp_argmin_first(s, nr - seg, nr);
        const double xl = (jl + 0.5), xr = (jr + 0.5);
        const double slope = (jr != jl) ? (s[jr] - s[jl]) / (xr - xl) : 0.0;   // per rebinned bin
        // products and sums rounded separately (no contraction): the definition in the header
        const double b_at0 = __dsub_rn(s[jl], __dmul_rn(slope, xl));          // at rebinned coordinate 0
        __syncwarp();
        for (int j = lane; j < nr; j += 32) r[j] = __dsub_rn(s[j], __dadd_rn(b_at0, __dmul_rn(slope, j + 0.5)));
        __syncwarp();
        int pk_j[8];
        double pk_A[8], pk_s[8];
        int found = 0;
        for (int k = 0; k < K && k < 8; ++k) {
            int bj = -1;
            double bv = 0.0;
            for (int j = 1 + lane; j < nr - 1; j += 32) {
                if (!(r[j] >= r[j - 1] && r[j] >= r[j + 1])) continue;
                bool far = true;
                for (int q = 0; q < found; ++q)
                    if (abs(j - pk_j[q]) < 3) far = false;
                if (far && (bj < 0 || r[j] > bv)) { bv = r[j]; bj = j; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
                if (oj >= 0 && (bj < 0 || ov > bv || (ov == bv && oj < bj))) { bv = ov; bj = oj; }
            }
            if (bj < 0 || !(r[bj] > 0.0)) break;
            const double half = 0.5 * r[bj];   // every lane walks the same short way
            int a = bj, b = bj;
            while (a > 0 && r[a] > half) --a;
            while (b < nr - 1 && r[b] > half) ++b;
            double fw = (double)(b - a);
            if (fw < 1.0) fw = 1.0;
            pk_j[found] = bj;
            pk_A[found] = r[bj] / factor;
            pk_s[found] = fw * wr / 2.3548200450309493;
            ++found;
        }
        if (lane == 0) {
            double pk_mu[8];
            for (int k = 0; k < found; ++k) pk_mu[k] = __dadd_rn(lo, __dmul_rn(pk_j[k] + 0.5, wr));
            for (int k = found; k < K; ++k) {    // not enough peaks: small ones spread over the range
                pk_mu[k] = lo + (hi - lo) * (k + 0.5) / K;
                pk_A[k] = 1.0;
                pk_s[k] = 2.0 * wr;
            }
            for (int i = 1; i < K; ++i)          // sort by mu (insertion)
                for (int j = i; j > 0 && pk_mu[j] < pk_mu[j - 1]; --j) {
                    double t;
                    t = pk_mu[j]; pk_mu[j] = pk_mu[j - 1]; pk_mu[j - 1] = t;
                    t = pk_A[j]; pk_A[j] = pk_A[j - 1]; pk_A[j - 1] = t;
                    t = pk_s[j]; pk_s[j] = pk_s[j - 1]; pk_s[j - 1] = t;
                }
            double* th = theta + h * (3 * K + 2);
            for (int k = 0; k < K; ++k) {
                th[3 * k] = pk_A[k];
                th[3 * k + 1] = pk_mu[k];
                th[3 * k + 2] = pk_s[k];
            }
            // background per original bin: b(x) = b0 + b1 x with x the bin centre
            const double per_bin = 1.0 / factor;
            th[3 * K] = (b_at0 - slope * lo / wr) * per_bin;
            th[3 * K + 1] = slope / wr * per_bin;
        }
        __syncwarp();
    }
}

// Refinement of starting points of K peaks + linear background on the
// full-resolution histogram, one warp per histogram (see cg.h,
// cg_refine_start).  Window bounds and bin centres are rounded operation by
// operation (no fused multiply-add), so that a plain restatement reproduces
// which bins each window holds.
__global__ void k_refine(const double* __restrict__ y, int64_t H, int n_bins, double lo, double hi, int K,
                         const double* __restrict__ th_in, double* __restrict__ th_out, int sweeps, double half) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int P = 3 * K + 2;
    const double h = __ddiv_rn(__dsub_rn(hi, lo), (double)n_bins);
    for (int64_t hh = (int64_t)blockIdx.x * nw + wid; hh < H; hh += (int64_t)gridDim.x * nw) {
        const double* yh = y + hh * (int64_t)n_bins;
        const double* ti = th_in + hh * P;
        double A[8], mu[8], s[8];
        for (int k = 0; k < K; ++k) {
            A[k] = ti[3 * k];
            mu[k] = ti[3 * k + 1];
            s[k] = fabs(ti[3 * k + 2]);
        }
        const double b0 = ti[3 * K], b1 = ti[3 * K + 1];
        auto sort_peaks = [&]() {
            for (int i = 1; i < K; ++i)
                for (int j = i; j > 0 && mu[j] < mu[j - 1]; --j) {
                    double t;
                    t = mu[j]; mu[j] = mu[j - 1]; mu[j - 1] = t;
                    t = A[j]; A[j] = A[j - 1]; A[j - 1] = t;
                    t = s[j]; s[j] = s[j - 1]; s[j - 1] = t;
                }
        };
        sort_peaks();
        for (int sw = 0; sw < sweeps; ++sw) {
            for (int k = 0; k < K; ++k) {
                const double w = __dmul_rn(half, fmax(s[k], __dmul_rn(4.0, h)));
                if (!(isfinite(mu[k]) && isfinite(w) && w > 0.0)) continue;
                const double a0 = floor(__ddiv_rn(__dsub_rn(__dsub_rn(mu[k], w), lo), h));
                const double a1 = ceil(__ddiv_rn(__dsub_rn(__dadd_rn(mu[k], w), lo), h));
                const int i0 = a0 < 0.0 ? 0 : (a0 > (double)(n_bins - 1) ? n_bins : (int)a0);
                const int i1 = a1 > (double)(n_bins - 1) ? n_bins - 1 : (a1 < 0.0 ? -1 : (int)a1);
                double S0 = 0.0, S1 = 0.0, S2 = 0.0;
                for (int i = i0 + lane; i <= i1; i += 32) {
                    const double x = __dadd_rn(lo, __dmul_rn((double)i + 0.5, h));
                    const double dx = __dsub_rn(x, mu[k]);
                    if (!(fabs(dx) <= w)) continue;
                    double r = __dsub_rn(yh[i], __dadd_rn(b0, __dmul_rn(b1, x)));
                    for (int j = 0; j < K; ++j) {
                        if (j == k) continue;
                        const double z = __ddiv_rn(__dsub_rn(x, mu[j]), s[j]);
                        r = __dsub_rn(r, __dmul_rn(A[j], exp(__dmul_rn(-0.5, __dmul_rn(z, z)))));
                    }
                    if (!(r > 0.0)) continue;
                    S0 = __dadd_rn(S0, r);
                    S1 = __dadd_rn(S1, __dmul_rn(r, dx));
                    S2 = __dadd_rn(S2, __dmul_rn(__dmul_rn(r, dx), dx));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {   // butterfly: every lane ends with the same sums
                    S0 = __dadd_rn(S0, __shfl_xor_sync(0xffffffffu, S0, o));
                    S1 = __dadd_rn(S1, __shfl_xor_sync(0xffffffffu, S1, o));
                    S2 = __dadd_rn(S2, __shfl_xor_sync(0xffffffffu, S2, o));
                }
                if (!(S0 > 0.0)) continue;
                const double m1 = __ddiv_rn(S1, S0);
                double var = __dsub_rn(__ddiv_rn(S2, S0), __dmul_rn(m1, m1));
                const double vmin = __dmul_rn(__dmul_rn(0.5, h), __dmul_rn(0.5, h));
                if (!(var > vmin)) var = vmin;
                // width of a Gaussian truncated at +-w with this variance: one step of
                // var = s^2 (1 - 2 z phi(z) / erf(z / sqrt 2)), z = w / s, from z = w / sqrt(var)
                double z = __ddiv_rn(w, sqrt(var));
                z = fmin(fmax(z, 0.5), 10.0);
                const double phi = __dmul_rn(0.3989422804014327, exp(__dmul_rn(-0.5, __dmul_rn(z, z))));
                const double frac = __dsub_rn(1.0, __ddiv_rn(__dmul_rn(__dmul_rn(2.0, z), phi),
                                                             erf(__dmul_rn(z, 0.7071067811865476))));
                const double s2 = sqrt(__ddiv_rn(var, frac));
                const double cover = erf(__dmul_rn(__ddiv_rn(w, s2), 0.7071067811865476));
                A[k] = __ddiv_rn(__dmul_rn(S0, h), __dmul_rn(__dmul_rn(s2, 2.5066282746310002), cover));
                mu[k] = __dadd_rn(mu[k], m1);
                s[k] = s2;
            }
            sort_peaks();
        }
        double* to = th_out + hh * P;
        __syncwarp();
        if (lane == 0) {
            for (int k = 0; k < K; ++k) {
                to[3 * k] = A[k];
                to[3 * k + 1] = mu[k];
                to[3 * k + 2] = s[k];
            }
            to[3 * K] = b0;
            to[3 * K + 1] = b1;
        }
        __syncwarp();
    }
}

// Mean squared error over the first n_out of ld columns, and its gradient.
// One block; fixed-order sums.
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ tgt, int64_t B, int n_out, int ld,
                      float* loss, float* dpred, __nv_bfloat16* dpred_b) {
    __shared__ double red[32];
    double acc = 0.0;
    const float sc = 2.0f / (float)(B * n_out);
    for (int64_t i = threadIdx.x; i < B * ld; i += blockDim.x) {
        const int64_t b = i / ld;
        const int c = (int)(i - b * ld);
        float d = 0.0f;
        if (c < n_out) {
            d = pred[i] - tgt[b * n_out + c];
            acc += (double)d * d;
        }
        if (dpred) dpred[i] = sc * d;
        if (dpred_b) dpred_b[i] = __float2bfloat16(sc * d);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *loss = (float)(t / (double)(B * n_out));
    }
}

// out[c] = sum_r X[r][c], rows summed in order by one thread per column.
__global__ void k_colsum(const float* __restrict__ X, int64_t rows, int cols, float* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0;
    for (int64_t r = 0; r < rows; ++r) s += X[r * cols + c];
    out[c] = (float)s;
}

// AdamW on FP32 master weights, with a BF16 copy for the GEMMs.
__global__ void k_adamw(float* w, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                        float eps, float wd, float bc1, float bc2, __nv_bfloat16* wb) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float wi = w[i] * (1.0f - lr * wd);
        wi -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_to_bf16(const float* __restrict__ a, int64_t n, __nv_bfloat16* b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace cg

extern "C" {

cg_status cg_rebin_normalize(const double* y, int64_t H, int n_bins, int factor, void* x_bf16, float* scale,
                             void* stream) {
    if (!y || !x_bf16 || !scale || H < 1 || factor < 1 || n_bins < factor || n_bins % factor) return CG_ERR_INVALID_ARG;
    const int nr = n_bins / factor;
    const size_t per_warp = (size_t)nr * sizeof(double);
    if (per_warp > 48 * 1024) return CG_ERR_INVALID_ARG;
    const int nw = (int)std::min<size_t>(cg::kHistWarps, 48 * 1024 / per_warp);
    const int64_t blocks = (H + nw - 1) / nw;
    const int g = (int)std::min<int64_t>(blocks, 16 * (int64_t)cg::device_sm_count());
    cg::k_rebin<<<g, 32 * nw, nw * per_warp, (cudaStream_t)stream>>>(y, H, n_bins, factor, (__nv_bfloat16*)x_bf16,
                                                                     scale);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_heuristic_start(const double* y, int64_t H, int n_bins, int factor, double lo, double hi, int n_peaks,
                             double* theta0, void* stream) {
    if (!y || !theta0 || H < 1 || factor < 1 || n_bins % factor || n_peaks < 1 || n_peaks > 8 || !(hi > lo))
        return CG_ERR_INVALID_ARG;
    const int nr = n_bins / factor;
    if (nr < 8) return CG_ERR_INVALID_ARG;
    const size_t per_warp = 2 * (size_t)nr * sizeof(double);
    if (per_warp > 48 * 1024) return CG_ERR_INVALID_ARG;
    const int nw = (int)std::min<size_t>(cg::kHistWarps, 48 * 1024 / per_warp);
    const int64_t blocks = (H + nw - 1) / nw;
    const int g = (int)std::min<int64_t>(blocks, 16 * (int64_t)cg::device_sm_count());
    cg::k_heuristic<<<g, 32 * nw, nw * per_warp, (cudaStream_t)stream>>>(y, H, n_bins, factor, lo, hi, n_peaks,
                                                                        theta0);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_refine_start(const double* y, int64_t H, int n_bins, double lo, double hi, int n_peaks,
                          const double* theta_in, double* theta_out, int sweeps, double half_width, void* stream) {
    if (!y || !theta_in || !theta_out || H < 1 || n_bins < 1 || n_peaks < 1 || n_peaks > 8 || !(hi > lo) ||
        sweeps < 0 || sweeps > 16 || !(half_width > 0.0) || !(half_width <= 10.0))
        return CG_ERR_INVALID_ARG;
    const int nw = 8;
    const int64_t blocks = (H + nw - 1) / nw;
    const int g = (int)std::min<int64_t>(blocks, 16 * (int64_t)cg::device_sm_count());
    cg::k_refine<<<g, 32 * nw, 0, (cudaStream_t)stream>>>(y, H, n_bins, lo, hi, n_peaks, theta_in, theta_out,
                                                         sweeps, half_width);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_mse_loss(const float* pred, const float* target, int64_t B, int n_out, int ld, float* loss,
                      float* dpred, void* dpred_bf16, void* stream) {
    if (!pred || !target || !loss || B < 1 || n_out < 1 || ld < n_out) return CG_ERR_INVALID_ARG;
    cg::k_mse<<<1, 1024, 0, (cudaStream_t)stream>>>(pred, target, B, n_out, ld, loss, dpred,
                                                   (__nv_bfloat16*)dpred_bf16);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_colsum(const float* X, int64_t rows, int cols, float* out, void* stream) {
    if (!X || !out || rows < 0 || cols < 1) return CG_ERR_INVALID_ARG;
    cg::k_colsum<<<(cols + 127) / 128, 128, 0, (cudaStream_t)stream>>>(X, rows, cols, out);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_adamw(float* w, const float* g, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                   float eps, float weight_decay, int step, void* w_bf16, void* stream) {
    if (!w || !g || !m || !v || n < 1 || step < 1) return CG_ERR_INVALID_ARG;
    const float bc1 = 1.0f - powf(beta1, (float)step), bc2 = 1.0f - powf(beta2, (float)step);
    cg::k_adamw<<<cg::grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(w, g, m, v, n, lr, beta1, beta2, eps,
                                                                       weight_decay, bc1, bc2,
                                                                       (__nv_bfloat16*)w_bf16);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

cg_status cg_to_bf16(const float* a, int64_t n, void* b, void* stream) {
    if (!a || !b || n < 0) return CG_ERR_INVALID_ARG;
    if (n == 0) return CG_OK;
    cg::k_to_bf16<<<cg::grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(a, n, (__nv_bfloat16*)b);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

}  // extern "C"

namespace cg {
namespace {

// Network output -> fit parameters.  Per histogram h with row y[h][.] (stride
// ld) the encoded targets are z-scores of (A_k f, mu_k, log s_k, b0 f, b1 f),
// f = factor / scale[h]; the inverse is clamped into the model's domain
// (A > 0, mu in [lo, hi], s between half a rebinned bin and the range,
// background >= 0 at both ends) and the peaks are sorted by mu.
__global__ void k_decode(const float* __restrict__ y, int ld, const float* __restrict__ scale,
                         const float* __restrict__ mean, const float* __restrict__ stdv, int64_t H, int K, int factor,
                         int n_bins, double lo, double hi, double* theta) {
    const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= H) return;
    const int P = 3 * K + 2;
    double t[3 * 8 + 2];
    for (int j = 0; j < P; ++j) t[j] = (double)y[h * ld + j] * stdv[j] + mean[j];
    const double f = (double)factor / (double)scale[h];
    const double wr = (hi - lo) * factor / n_bins;
    for (int k = 0; k < K; ++k) {
        t[3 * k] = fmax(t[3 * k] / f, 1e-3 / f);
        t[3 * k + 1] = fmin(fmax(t[3 * k + 1], lo), hi);
        t[3 * k + 2] = fmin(fmax(exp(t[3 * k + 2]), 0.5 * wr), hi - lo);
    }
    double b0 = t[3 * K] / f, b1 = t[3 * K + 1] / f;
    // keep the line non-negative at both ends of the range
    const double e0 = fmax(b0 + b1 * lo, 1e-3 / f), e1 = fmax(b0 + b1 * hi, 1e-3 / f);
    b1 = (e1 - e0) / (hi - lo);
    b0 = e0 - b1 * lo;
    for (int i = 1; i < K; ++i)
        for (int j = i; j > 0 && t[3 * j + 1] < t[3 * (j - 1) + 1]; --j)
            for (int q = 0; q < 3; ++q) {
                const double s = t[3 * j + q];
                t[3 * j + q] = t[3 * (j - 1) + q];
                t[3 * (j - 1) + q] = s;
            }
    double* o = theta + h * P;
    for (int j = 0; j < 3 * K; ++j) o[j] = t[j];
    o[3 * K] = b0;
    o[3 * K + 1] = b1;
}

}  // namespace
}  // namespace cg

extern "C" cg_status cg_decode_start(const float* y, int ld, const float* scale, const float* mean, const float* stdv,
                                     int64_t H, int n_peaks, int factor, int n_bins, double lo, double hi,
                                     double* theta0, void* stream) {
    if (!y || !scale || !mean || !stdv || !theta0 || H < 1 || n_peaks < 1 || n_peaks > 8 || ld < 3 * n_peaks + 2 ||
        factor < 1 || n_bins < factor || !(hi > lo))
        return CG_ERR_INVALID_ARG;
    cg::k_decode<<<(unsigned)((H + 127) / 128), 128, 0, (cudaStream_t)stream>>>(y, ld, scale, mean, stdv, H, n_peaks,
                                                                              factor, n_bins, lo, hi, theta0);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}

namespace cg {
namespace {
// Per histogram, the candidate whose objective value is lower (a non-finite
// value loses); ties keep candidate a.
__global__ void k_select(const double* fa, const double* fb, const double* ta, const double* tb, int64_t H, int P,
                         double* out, int* took_a) {
    const int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (h >= H) return;
    const double a = fa[h], b = fb[h];
    const bool pick_a = isfinite(a) && (!isfinite(b) || a <= b);
    const double* src = pick_a ? ta + h * P : tb + h * P;
    for (int k = 0; k < P; ++k) out[h * P + k] = src[k];
    if (took_a) took_a[h] = pick_a ? 1 : 0;
}
}  // namespace
}  // namespace cg

extern "C" cg_status cg_select_start(const double* fa, const double* fb, const double* theta_a, const double* theta_b,
                                     int64_t H, int P, double* theta_out, int* took_a, void* stream) {
    if (!fa || !fb || !theta_a || !theta_b || !theta_out || H < 1 || P < 1) return CG_ERR_INVALID_ARG;
    cg::k_select<<<(unsigned)((H + 255) / 256), 256, 0, (cudaStream_t)stream>>>(fa, fb, theta_a, theta_b, H, P,
                                                                              theta_out, took_a);
    return cudaGetLastError() == cudaSuccess ? CG_OK : CG_ERR_CUDA;
}
