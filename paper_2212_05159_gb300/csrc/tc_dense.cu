// Dense layer of the network on the 5th-generation tensor cores (tcgen05, TMEM):
//   Y = [X1 X2] W + b  with the epilogues of spx_dense_forward (raw, relu, residual),
// BF16 operands (activations rounded to BF16 while staged, BF16 weights), FP32
// accumulation in tensor memory.
//
// One CTA of 128 threads per 128-row tile (the layer is memory-bound: K, N <= 128):
//   * the threads stage the tile's activations with coalesced float4 loads (consecutive
//     threads read consecutive 16-byte pieces of a row), convert them to BF16 and store
//     them in the canonical no-swizzle K-major layout: 8-row x 16-byte core matrices, the
//     core matrices of one 8-row group contiguous along K (leading byte offset 128), groups
//     (K/8) * 128 bytes apart (stride byte offset); W^T the same way;
//   * warp 0 allocates N columns of tensor memory; one thread issues K/16 tcgen05.mma
//     (M = 128, N, K = 16 each) and commits them to an mbarrier;
//   * after a bounded wait each warp reads its 32 accumulator lanes (rows) with tcgen05.ld,
//     adds the bias and parks the rows in shared memory (the operand tiles are free once
//     the MMAs have completed); the warp then writes its rows back with coalesced float4
//     accesses, reading Hin and writing U for the residual epilogue; warp 0 frees the
//     tensor memory.
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
constexpr int TC_TILES = TC_M * TC_KMAX * 2 + TC_NMAX * TC_KMAX * 2;  // A and B^T tiles: 64 KB
constexpr int TC_STAGE = TC_M * (TC_NMAX + 4) * 4;                    // epilogue rows: 66 KB
constexpr int TC_SMEM = TC_TILES > TC_STAGE ? TC_TILES : TC_STAGE;

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

// Stages rows [row0, row0 + 128) of X (n x K, row stride K, K % 4 == 0) into columns
// [kbase, kbase + K) of the A tile; rows past n are zero.  Loads are issued STAGE_BATCH at a
// time per thread before any is converted, so enough bytes are in flight to cover the
// memory latency (the layer is bandwidth-bound).
constexpr int STAGE_BATCH = 8;

__device__ __forceinline__ void stage_rows(unsigned char* sA, const float* __restrict__ X, int K, int kbase, int kpad,
                                           int64_t row0, int64_t n) {
    const int q4 = K >> 2;                                   // float4 pieces per row
    const int total = TC_M * q4;
    for (int t0 = threadIdx.x; t0 < total; t0 += STAGE_BATCH * TC_THREADS) {
        float4 v[STAGE_BATCH];
#pragma unroll
        for (int u = 0; u < STAGE_BATCH; ++u) {
            const int t = t0 + u * TC_THREADS;
            const int r = t / q4, kq = t - r * q4;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t < total && row0 + r < n) v[u] = __ldcs(reinterpret_cast<const float4*>(X + (row0 + r) * K) + kq);
        }
#pragma unroll
        for (int u = 0; u < STAGE_BATCH; ++u) {
            const int t = t0 + u * TC_THREADS;
            if (t < total) {
                const int r = t / q4, kq = t - r * q4;
                const uint2 pk = make_uint2(pack_bf16x2(v[u].x, v[u].y), pack_bf16x2(v[u].z, v[u].w));
                *reinterpret_cast<uint2*>(sA + core_off(r, kbase + kq * 4, kpad)) = pk;
            }
        }
    }
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
    unsigned char* sB = smem + TC_M * kpad * 2;                 // N x kpad bf16, after A
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;
    const int ncols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);

    // ---- stage A = [X1 X2] (FP32 -> BF16) and its zero padding up to kpad
    stage_rows(sA, X1, K1, 0, kpad, row0, n);
    if (K2 > 0) stage_rows(sA, X2, K2, K1, kpad, row0, n);
    if (kpad > K) {
        const int pq = (kpad - K) >> 2;                        // K % 4 == 0: padding in 4-column pieces
        for (int t = threadIdx.x; t < TC_M * pq; t += TC_THREADS) {
            const int r = t / pq, kq = t - r * pq;
            *reinterpret_cast<uint2*>(sA + core_off(r, K + kq * 4, kpad)) = make_uint2(0u, 0u);
        }
    }
    // ---- stage B = W^T (N rows, K-major); consecutive threads read consecutive columns of W
    for (int t = threadIdx.x; t < N * kpad; t += TC_THREADS) {
        const int k = t / N, nn = t - k * N;
        const __nv_bfloat16 w = k < K ? W[k * N + nn] : __float2bfloat16(0.f);
        *reinterpret_cast<__nv_bfloat16*>(sB + core_off(nn, k, kpad)) = w;
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
        const uint32_t sbo = (uint32_t)(kpad >> 3) * 128u;
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
        // ---- epilogue 1: accumulator lanes of this warp (rows 32w .. 32w + 31) -> shared
        // memory, bias added.  The MMAs have completed (mbarrier), so the operand tiles are
        // free; each warp reuses its own slice: 32 rows x (N + 4) floats.
        const int ldst = N + 4;                                      // padded row stride (floats)
        float* stage = reinterpret_cast<float*>(smem) + (size_t)warp * 32 * ldst;
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
#pragma unroll
            for (int q = 0; q < 16; q += 4) {
                float4 o;
                o.x = __uint_as_float(v[q + 0]) + (bias ? bias[c0 + q + 0] : 0.f);
                o.y = __uint_as_float(v[q + 1]) + (bias ? bias[c0 + q + 1] : 0.f);
                o.z = __uint_as_float(v[q + 2]) + (bias ? bias[c0 + q + 2] : 0.f);
                o.w = __uint_as_float(v[q + 3]) + (bias ? bias[c0 + q + 3] : 0.f);
                *reinterpret_cast<float4*>(stage + lane * ldst + c0 + q) = o;
            }
        }
        __syncwarp();
        // ---- epilogue 2: the warp's 32 rows to global memory, float4 pieces in row order
        const int n4 = N >> 2;
#pragma unroll 4
        for (int t = lane; t < 32 * n4; t += 32) {
            const int r = t / n4, cq = t - r * n4;
            const int64_t row = row0 + warp * 32 + r;
            if (row >= n) break;                                 // rows only grow with t
            const float4 pre = *reinterpret_cast<const float4*>(stage + r * ldst + cq * 4);
            const int64_t o = row * N + cq * 4;
            if (mode == 0) {
                __stcs(reinterpret_cast<float4*>(Y + o), pre);
            } else if (mode == 1) {
                __stcs(reinterpret_cast<float4*>(Y + o),
                       make_float4(fmaxf(pre.x, 0.f), fmaxf(pre.y, 0.f), fmaxf(pre.z, 0.f), fmaxf(pre.w, 0.f)));
            } else {
                const float4 h = __ldcs(reinterpret_cast<const float4*>(Hin + o));
                __stcs(reinterpret_cast<float4*>(U + o), pre);
                __stcs(reinterpret_cast<float4*>(Y + o),
                       make_float4(h.x + fmaxf(pre.x, 0.f), h.y + fmaxf(pre.y, 0.f), h.z + fmaxf(pre.z, 0.f),
                                   h.w + fmaxf(pre.w, 0.f)));
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

// Shared memory one launch needs: the A and B^T tiles for its K, or the epilogue rows for its
// N, whichever is larger (smaller layers fit more blocks per SM).
size_t tc_smem_bytes(int K, int N) {
    const size_t kpad = (size_t)((K + 15) & ~15);
    const size_t tiles = (size_t)TC_M * kpad * 2 + (size_t)N * kpad * 2;
    const size_t stage = (size_t)TC_M * (N + 4) * 4;
    return tiles > stage ? tiles : stage;
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

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
    if (K1 % 4 != 0 || K2 % 4 != 0 || !al16(X1) || (K2 > 0 && !al16(X2)) || !al16(Y) ||
        (mode == 2 && (!al16(Hin) || !al16(U))))
        return set_error(SPX_INVALID_ARG, "spx_dense_forward_tc: K1, K2 multiples of 4 and 16-byte aligned rows needed");
    if (n == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    const size_t smem = tc_smem_bytes(K1 + K2, N);
    static std::atomic<unsigned long long> attr_done{0};
    SPX_TRY(ensure_smem_attr(dense_tc_kernel, TC_SMEM, attr_done, "spx_dense_forward_tc attribute"));
    const int64_t tiles = (n + TC_M - 1) / TC_M;
    dense_tc_kernel<<<(unsigned)tiles, TC_THREADS, smem, st>>>(n, X1, K1, X2, K2,
                                                              static_cast<const __nv_bfloat16*>(W_bf16), bias, N, mode,
                                                              Hin, Y, U, device_error_word());
    SPX_CHECK_LAUNCH("spx_dense_forward_tc");
    return SPX_OK;
}
