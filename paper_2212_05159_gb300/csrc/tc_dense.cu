// Dense layer of the network on the 5th-generation tensor cores (tcgen05, TMEM):
//   Y = [X1 X2] W + b  with the epilogues of spx_dense_forward (raw, relu, residual),
// BF16 operands (activations rounded to BF16 while staged, BF16 weights), FP32
// accumulation in tensor memory.
//
// One CTA of 128 threads per 128-row tile:
//   * all threads stage the tile's activations (FP32 -> BF16) and W^T into shared memory
//     in the canonical no-swizzle K-major layout: 8-row x 16-byte core matrices, the core
//     matrices of one 8-row group contiguous along K (leading byte offset 128), groups
//     (K/8) * 128 bytes apart (stride byte offset);
//   * warp 0 allocates N columns of tensor memory; one thread issues K/16 tcgen05.mma
//     (M = 128, N, K = 16 each) and commits them to an mbarrier;
//   * after a bounded wait each warp reads its 32 accumulator lanes with tcgen05.ld and
//     applies the epilogue; warp 0 frees the tensor memory.
// A wait that does not complete within 2 s records a device error; the kernel still frees
// its tensor memory before returning.
#include <cuda_bf16.h>

#include "common.cuh"

namespace spx {
namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 128;
constexpr int TC_KMAX = 128;
constexpr int TC_NMAX = 128;

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;                    // descriptor version of the sm_100 family
    return d;                                  // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D F32, A and B BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) in the core-matrix layout of a rows x Kpad operand
__device__ __forceinline__ uint32_t core_off(int row, int k, int kpad) {
    return (uint32_t)((row >> 3) * (kpad >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__global__ void __launch_bounds__(TC_THREADS) dense_tc_kernel(int64_t n, const float* __restrict__ X1, int K1,
                                                              const float* __restrict__ X2, int K2,
                                                              const __nv_bfloat16* __restrict__ W,
                                                              const float* __restrict__ bias, int N, int mode,
                                                              const float* __restrict__ Hin, float* __restrict__ Y,
                                                              float* __restrict__ U, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int K = K1 + K2;
    const int kpad = (K + 15) & ~15;
    unsigned char* sA = smem;                                   // 128 x kpad bf16
    unsigned char* sB = smem + TC_M * TC_KMAX * 2;              // N x kpad bf16
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;
    const int ncols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);

    // ---- stage A: 8-element chunks (16 bytes) of the tile rows, FP32 -> BF16
    const int kch = kpad >> 3;
    for (int t = threadIdx.x; t < TC_M * kch; t += TC_THREADS) {
        const int r = t / kch, kc = t % kch;
        const int64_t row = row0 + r;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kc * 8 + q;
            float x = 0.f;
            if (row < n) {
                if (k < K1) x = X1[row * K1 + k];
                else if (k < K) x = X2[row * K2 + (k - K1)];
            }
            v[q] = x;
        }
        uint4 pk = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                              pack_bf16x2(v[6], v[7]));
        *reinterpret_cast<uint4*>(sA + core_off(r, kc * 8, kpad)) = pk;
    }
    // ---- stage B = W^T (N rows, K-major)
    for (int t = threadIdx.x; t < N * kch; t += TC_THREADS) {
        const int nn = t / kch, kc = t % kch;
        unsigned short h[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kc * 8 + q;
            __nv_bfloat16 w = k < K ? W[k * N + nn] : __float2bfloat16(0.f);
            h[q] = *reinterpret_cast<unsigned short*>(&w);
        }
        uint4 pk = make_uint4(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16), h[4] | ((uint32_t)h[5] << 16),
                              h[6] | ((uint32_t)h[7] << 16));
        *reinterpret_cast<uint4*>(sB + core_off(nn, kc * 8, kpad)) = pk;
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&mbar), 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();                   // generic smem writes -> visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (threadIdx.x == 0) {
        const uint32_t idesc = instr_desc(TC_M, N);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        const uint32_t sbo = (uint32_t)kch * 128u;
        for (int s = 0; s < kpad / 16; ++s) {
            const uint64_t ad = smem_desc(a0 + s * 256u, 128u, sbo);
            const uint64_t bd = smem_desc(b0 + s * 256u, 128u, sbo);
            const uint32_t acc = s > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&mbar))
                     : "memory");
    }
    const bool ok = __all_sync(FULL, mbar_wait(smem_u32(&mbar), 0, 2000000000ull));   // warp-uniform
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (threadIdx.x == 0 && err) atomicOr(err, 2);
    } else {
        // ---- epilogue: warp w owns accumulator lanes (rows) 32w .. 32w + 31
        const int r = warp * 32 + lane;
        const int64_t row = row0 + r;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < n) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c0 + q;
                    if (c >= N) break;
                    const float pre = __uint_as_float(v[q]) + (bias ? bias[c] : 0.f);
                    if (mode == 0) {
                        Y[row * N + c] = pre;
                    } else if (mode == 1) {
                        Y[row * N + c] = fmaxf(pre, 0.f);
                    } else {
                        U[row * N + c] = pre;
                        Y[row * N + c] = Hin[row * N + c] + fmaxf(pre, 0.f);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

size_t tc_smem_bytes() { return (size_t)TC_M * TC_KMAX * 2 + (size_t)TC_NMAX * TC_KMAX * 2; }

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_dense_forward_tc(int64_t n, const float* X1, int32_t K1, const float* X2, int32_t K2,
                                           const void* W_bf16, const float* bias, int32_t N, int32_t mode,
                                           const float* Hin, float* Y, float* U, void* stream) {
    if (n < 0 || K1 < 1 || K2 < 0 || K1 + K2 > TC_KMAX || N < 16 || N > TC_NMAX || N % 16 != 0 || mode < 0 ||
        mode > 2)
        return set_error(SPX_INVALID_ARG, "spx_dense_forward_tc: sizes (K <= 128, N in 16..128, N %% 16 == 0)");
    if (n > 0 && (!X1 || (K2 > 0 && !X2) || !W_bf16 || !Y || (mode == 2 && (!Hin || !U))))
        return set_error(SPX_INVALID_ARG, "spx_dense_forward_tc: NULL operand");
    if (n == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    const size_t smem = tc_smem_bytes();
    static bool attr = false;
    if (!attr) {
        SPX_CUDA(cudaFuncSetAttribute(dense_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                 "spx_dense_forward_tc attribute");
        attr = true;
    }
    const int64_t tiles = (n + TC_M - 1) / TC_M;
    dense_tc_kernel<<<(unsigned)tiles, TC_THREADS, smem, st>>>(n, X1, K1, X2, K2,
                                                              static_cast<const __nv_bfloat16*>(W_bf16), bias, N, mode,
                                                              Hin, Y, U, device_error_word());
    SPX_CHECK_LAUNCH("spx_dense_forward_tc");
    return SPX_OK;
}
