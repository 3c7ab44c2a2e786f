// Dense layer of the network on the 5th-generation tensor cores (tcgen05, TMEM):
//   Y = [X1 X2] W + b  with the epilogues of spx_dense_forward (raw, relu, residual),
// BF16 operands (activations rounded to BF16 while staged, BF16 weights), FP32
// accumulation in tensor memory.
//
// Persistent CTAs of 128 threads, as many per SM as shared memory allows, each walking
// 128-row tiles (the layer is memory-bound: K, N <= 128); W^T, the mbarrier and the
// accumulator columns are set up once per CTA:
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
#include "tc_pipe.h"

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

// Byte offset of W^T in the forward kernel's shared memory: after the larger of the A tile
// and the epilogue rows, rounded up to 1 KB.
__host__ __device__ inline size_t tc_b_offset(int K, int N) {
    const size_t kpad = (size_t)((K + 15) & ~15);
    const size_t a = (size_t)TC_M * kpad * 2;
    const size_t stage = (size_t)TC_M * (N + 4) * 4;
    return ((a > stage ? a : stage) + 1023) & ~size_t(1023);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Stages rows [row0, row0 + 128) of X (n x K, row stride K, K % 4 == 0) into columns
// [kbase, kbase + K) of the A tile; rows past n are zero.  Loads are issued STAGE_BATCH at a
// time per thread before any is converted, so enough bytes are in flight to cover the
// memory latency (the layer is bandwidth-bound).
constexpr int STAGE_BATCH = 16;
constexpr int EPI_BATCH = 8;                                 // epilogue loads in flight per thread
constexpr int TD_EPI_COLS = 64;                              // data-gradient epilogue part width

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
    // [A tile | epilogue rows] (reused every tile), then W^T (staged once per CTA)
    unsigned char* sA = smem;                                   // 128 x kpad bf16
    unsigned char* sB = smem + tc_b_offset(K, N);               // N x kpad bf16
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
    const int64_t ntiles = (n + TC_M - 1) / TC_M;

    // ---- once per CTA: B = W^T (N rows, K-major), the mbarrier, the accumulator columns
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    uint32_t phase = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
        const int64_t row0 = tile * TC_M;
        // ---- stage A = [X1 X2] (FP32 -> BF16) and its zero padding up to kpad
        stage_rows(sA, X1, K1, 0, kpad, row0, n);
        if (K2 > 0) stage_rows(sA, X2, K2, K1, kpad, row0, n);
        if (kpad > K) {
            const int pq = (kpad - K) >> 2;                    // K % 4 == 0: padding in 4-column pieces
            for (int t = threadIdx.x; t < TC_M * pq; t += TC_THREADS) {
                const int r = t / pq, kq = t - r * pq;
                *reinterpret_cast<uint2*>(sA + core_off(r, K + kq * 4, kpad)) = make_uint2(0u, 0u);
            }
        }
        fence_proxy_async();               // generic smem writes -> visible to the tensor cores
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

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
        const bool ok = __all_sync(FULL, mbar_wait(smem_u32(&mbar), phase, 2000000000ull));   // warp-uniform
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // a wait that ran out in one warp ends the CTA's work after this tile for all warps
        __shared__ int stop;
        if (threadIdx.x == 0) stop = 0;
        __syncthreads();
        if (!ok && lane == 0) stop = 1;
        __syncthreads();
        if (stop) {
            if (threadIdx.x == 0 && err) atomicOr(err, 2);
            break;
        }
        // ---- epilogue 1: accumulator lanes of this warp (rows 32w .. 32w + 31) -> shared
        // memory, bias added.  The MMAs have completed (mbarrier), so the A tile is free;
        // each warp reuses its own slice of it: 32 rows x (N + 4) floats.
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
        // ---- epilogue 2: the warp's valid rows to global memory, float4 pieces in row order;
        // the residual's Hin pieces are loaded EPI_BATCH at a time before any is used
        const int n4 = N >> 2;
        const int64_t wrow0 = row0 + warp * 32;
        const int nv = n - wrow0 >= 32 ? 32 : (n > wrow0 ? (int)(n - wrow0) : 0);
        const int total = nv * n4;
        const bool residual = mode == 2 || mode == 3;
        for (int t0 = lane; t0 < total; t0 += EPI_BATCH * 32) {
            float4 h[EPI_BATCH];
            if (residual) {
#pragma unroll
                for (int u = 0; u < EPI_BATCH; ++u) {
                    const int t = t0 + u * 32;
                    if (t < total) {
                        const int r = t / n4, cq = t - r * n4;
                        h[u] = __ldcs(reinterpret_cast<const float4*>(Hin + (wrow0 + r) * N + cq * 4));
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < EPI_BATCH; ++u) {
                const int t = t0 + u * 32;
                if (t >= total) break;
                const int r = t / n4, cq = t - r * n4;
                const float4 pre = *reinterpret_cast<const float4*>(stage + r * ldst + cq * 4);
                const int64_t o = (wrow0 + r) * N + cq * 4;
                if (mode == 0) {
                    __stcs(reinterpret_cast<float4*>(Y + o), pre);
                } else if (mode == 1) {
                    __stcs(reinterpret_cast<float4*>(Y + o),
                           make_float4(fmaxf(pre.x, 0.f), fmaxf(pre.y, 0.f), fmaxf(pre.z, 0.f), fmaxf(pre.w, 0.f)));
                } else if (mode == 4) {
                    // two outputs of N / 2 columns each: the column halves of the product
                    const int h2 = N >> 1;
                    const int c = cq * 4;
                    float* dst = c < h2 ? Y + (wrow0 + r) * h2 + c : U + (wrow0 + r) * h2 + (c - h2);
                    __stcs(reinterpret_cast<float4*>(dst), pre);
                } else {
                    if (mode == 2) __stcs(reinterpret_cast<float4*>(U + o), pre);
                    __stcs(reinterpret_cast<float4*>(Y + o),
                           make_float4(h[u].x + fmaxf(pre.x, 0.f), h[u].y + fmaxf(pre.y, 0.f),
                                       h[u].z + fmaxf(pre.z, 0.f), h[u].w + fmaxf(pre.w, 0.f)));
                }
            }
        }
        // the A / epilogue region and the accumulator are free for the next tile
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// Data gradient of the layer on the tensor cores: [dX1 dX2] (+)= G W^T with G: n x N (FP32,
// rounded to BF16 while staged) and W: (K1 + K2) x N (BF16).  The same tile scheme as the
// forward kernel with the roles swapped: A = G's 128-row tile (K-major over N), B = W's rows
// (one per output column, K-major over N), M = 128, the MMA's N = K1 + K2 rounded up to 16;
// the epilogue writes (or adds into) dX1's and dX2's columns with coalesced float4 accesses.
__global__ void __launch_bounds__(TC_THREADS) dense_tc_bwd_data_kernel(int64_t n, const float* __restrict__ G, int N,
                                                                       const __nv_bfloat16* __restrict__ W, int K1,
                                                                       int K2, float* __restrict__ dX1,
                                                                       float* __restrict__ dX2, int accumulate,
                                                                       int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int K = K1 + K2;                                      // output columns
    const int kout = (K + 15) & ~15;                            // the MMA's N
    const int npad = (N + 15) & ~15;                            // reduction extent
    unsigned char* sA = smem;                                   // 128 x npad bf16 (rows of G)
    unsigned char* sB = smem + TC_M * npad * 2;                 // kout x npad bf16 (rows of W)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;
    const int ncols = kout <= 32 ? 32 : (kout <= 64 ? 64 : 128);

    stage_rows(sA, G, N, 0, npad, row0, n);
    if (npad > N) {
        const int pq = (npad - N) >> 2;
        for (int t = threadIdx.x; t < TC_M * pq; t += TC_THREADS) {
            const int r = t / pq, kq = t - r * pq;
            *reinterpret_cast<uint2*>(sA + core_off(r, N + kq * 4, npad)) = make_uint2(0u, 0u);
        }
    }
    // B row kk = W's row kk (consecutive threads read consecutive entries of a row)
    for (int t = threadIdx.x; t < kout * npad; t += TC_THREADS) {
        const int kk = t / npad, c = t - kk * npad;
        const __nv_bfloat16 w = (kk < K && c < N) ? W[kk * N + c] : __float2bfloat16(0.f);
        *reinterpret_cast<__nv_bfloat16*>(sB + core_off(kk, c, npad)) = w;
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
    fence_proxy_async();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (threadIdx.x == 0) {
        const uint32_t idesc = instr_desc(TC_M, kout);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        const uint32_t sbo = (uint32_t)(npad >> 3) * 128u;
        for (int s = 0; s < npad / 16; ++s) {
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
    const bool ok = __all_sync(FULL, mbar_wait(smem_u32(&mbar), 0, 2000000000ull));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (threadIdx.x == 0 && err) atomicOr(err, 2);
    } else {
        // epilogue in parts of TD_EPI_COLS accumulator columns, so the staged rows take a
        // quarter of the 128-column layer's shared memory and more blocks stay resident
        const int ldst = (kout < TD_EPI_COLS ? kout : TD_EPI_COLS) + 4;
        float* stage = reinterpret_cast<float*>(smem) + (size_t)warp * 32 * ldst;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        const int64_t wrow0 = row0 + warp * 32;
        const int nv = n - wrow0 >= 32 ? 32 : (n > wrow0 ? (int)(n - wrow0) : 0);
        for (int h = 0; h < K; h += TD_EPI_COLS) {
            const int hw = kout - h < TD_EPI_COLS ? kout - h : TD_EPI_COLS;     // multiple of 16
            for (int c0 = 0; c0 < hw; c0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(taddr + (uint32_t)(h + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4*>(stage + lane * ldst + c0 + q) =
                        make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]), __uint_as_float(v[q + 2]),
                                    __uint_as_float(v[q + 3]));
            }
            __syncwarp();
            // the warp's valid rows, float4 pieces of output columns [h, h + kh * 4) in row
            // order (K1, K2 multiples of 4: a piece never straddles dX1 and dX2); with
            // accumulate the old pieces are loaded EPI_BATCH at a time before any is added
            const int kh = (K - h < TD_EPI_COLS ? K - h : TD_EPI_COLS) >> 2;
            const int total = nv * kh;
            auto dst_of = [&](int t) -> float* {
                const int r = t / kh, c = h + (t - r * kh) * 4;
                if (c < K1) return dX1 + (wrow0 + r) * K1 + c;
                return dX2 ? dX2 + (wrow0 + r) * K2 + (c - K1) : nullptr;
            };
            for (int t0 = lane; t0 < total; t0 += EPI_BATCH * 32) {
                float4 old[EPI_BATCH];
                if (accumulate) {
#pragma unroll
                    for (int u = 0; u < EPI_BATCH; ++u) {
                        const int t = t0 + u * 32;
                        float* d = t < total ? dst_of(t) : nullptr;
                        old[u] = d ? *reinterpret_cast<const float4*>(d) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < EPI_BATCH; ++u) {
                    const int t = t0 + u * 32;
                    if (t >= total) break;
                    float* d = dst_of(t);
                    if (!d) continue;
                    const int r = t / kh;
                    float4 val = *reinterpret_cast<const float4*>(stage + r * ldst + (t - r * kh) * 4);
                    if (accumulate)
                        val = make_float4(old[u].x + val.x, old[u].y + val.y, old[u].z + val.z, old[u].w + val.w);
                    *reinterpret_cast<float4*>(d) = val;
                }
            }
            __syncwarp();                                       // stage read before the next part
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// ---------------------------------------------------------------------------------------
// Weight gradient of the layer on the tensor cores: dW = [X1 X2]^T G (K x N) and db = the
// column sums of G.  The reduction runs over the rows, so the operands are the transposes
// of the row tiles: A (M = 128 rows of dW, the K inputs zero-padded to 128) holds X^T and
// B (the MMA's N = N) holds G^T, both K-major over 128 rows of the tile.  A thread item is
// one 4-column piece of 8 consecutive rows (8 float4 loads, consecutive threads on
// consecutive pieces of the same rows); its 32 values become four 16-byte core-matrix rows
// of the transposed operand (one per column, the 8 rows' BF16 values side by side).  The
// 8-row groups of the operands lie TW_SBO = 2064 bytes apart instead of 2048, so the 32
// lanes' 16-byte stores fall evenly on the 8 slots of a 128-byte shared-memory window
// (with 2048 they met two slots: a 16-way bank conflict); the MMA descriptors carry the
// same stride.
//
// Two persistent CTAs per SM (one's loads in flight while the other converts) walk the row
// tiles with a stride of the grid, each with two staging buffers in turn: while the tensor
// cores run tile t's 8 MMAs (K = 16 rows each, the FP32 accumulator stays in tensor memory
// across all of the CTA's tiles), the threads stage tile t + 1 (for N <= 64 with its loads
// already in flight: PIPE, below).  A buffer is restaged only
// after the mbarrier of the commit that read it has completed (bounded wait).  db is summed
// in FP32 by the threads from the values they load (each thread owns one 4-column piece of
// G).  Each CTA writes its partial (K + 1) x N block (dW rows, then db) to the workspace; a
// second kernel adds the partials in block order, so the result does not depend on timing.
constexpr int TW_THREADS = 256;
constexpr int TW_CTAS_PER_SM = 2;                               // two staging pipelines per SM
constexpr int TW_SBO = (TC_M / 8) * 128 + 16;                   // 8-row group stride, padded
constexpr int TW_A = (TC_M / 8) * TW_SBO;                       // A buffer: 128 x 128 BF16 (+ pads)
__host__ __device__ constexpr int tw_buf_bytes(int N) { return TW_A + (N / 8) * TW_SBO; }

// byte offset of element (operand row m, tile row k) in the padded transposed operands
__device__ __forceinline__ uint32_t tw_off(int m, int k) {
    return (uint32_t)((m >> 3) * TW_SBO + (k >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2);
}

// Item t of a tile over the sources S1 (nq1 pieces) then S2 (nq2): rows row0 + 8 o .. + 7 of
// piece q, o = t / (nq1 + nq2); rows past n read as zero.
__device__ __forceinline__ void tw_item_load(float4 (&v)[8], int t, const float* __restrict__ S1, int nq1,
                                             const float* __restrict__ S2, int nq2, int64_t row0, int64_t n) {
    const int nq = nq1 + nq2;
    const int o = t / nq, q = t - o * nq;
    const bool first = q < nq1;
    const float* src = first ? S1 + 4 * q : S2 + 4 * (q - nq1);
    const int64_t step = first ? 4 * nq1 : 4 * nq2;
    const int64_t r0 = row0 + 8 * o;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        v[r] = r0 + r < n ? __ldcs(reinterpret_cast<const float4*>(src + (r0 + r) * step))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The item's four columns as four 16-byte operand rows (operand row 4 q + i, tile rows 8 o ..)
__device__ __forceinline__ void tw_item_store(unsigned char* buf, const float4 (&v)[8], int t, int nq) {
    const int o = t / nq, q = t - o * nq;
    const int m = 4 * q, k = 8 * o;
    *reinterpret_cast<uint4*>(buf + tw_off(m + 0, k)) =
        make_uint4(pack_bf16x2(v[0].x, v[1].x), pack_bf16x2(v[2].x, v[3].x), pack_bf16x2(v[4].x, v[5].x),
                   pack_bf16x2(v[6].x, v[7].x));
    *reinterpret_cast<uint4*>(buf + tw_off(m + 1, k)) =
        make_uint4(pack_bf16x2(v[0].y, v[1].y), pack_bf16x2(v[2].y, v[3].y), pack_bf16x2(v[4].y, v[5].y),
                   pack_bf16x2(v[6].y, v[7].y));
    *reinterpret_cast<uint4*>(buf + tw_off(m + 2, k)) =
        make_uint4(pack_bf16x2(v[0].z, v[1].z), pack_bf16x2(v[2].z, v[3].z), pack_bf16x2(v[4].z, v[5].z),
                   pack_bf16x2(v[6].z, v[7].z));
    *reinterpret_cast<uint4*>(buf + tw_off(m + 3, k)) =
        make_uint4(pack_bf16x2(v[0].w, v[1].w), pack_bf16x2(v[2].w, v[3].w), pack_bf16x2(v[4].w, v[5].w),
                   pack_bf16x2(v[6].w, v[7].w));
}

// Stages the tile's rows into A (X1, X2) and B (G): per round two A items and one B item a
// thread, all 24 loads issued before any store.  Thread x owns G's piece x mod N/4 (N / 4
// divides the block), whose values it adds into db.
__device__ __forceinline__ void tw_stage(unsigned char* sA, unsigned char* sB, const float* __restrict__ X1, int nq1,
                                         const float* __restrict__ X2, int nq2, const float* __restrict__ G, int nqb,
                                         int64_t row0, int64_t n, float4& db) {
    const int totA = (TC_M / 8) * (nq1 + nq2), totB = (TC_M / 8) * nqb;
    const int rounds_a = (totA + 2 * TW_THREADS - 1) / (2 * TW_THREADS);
    const int rounds_b = (totB + TW_THREADS - 1) / TW_THREADS;
    const int rounds = rounds_a > rounds_b ? rounds_a : rounds_b;
    for (int rd = 0; rd < rounds; ++rd) {
        float4 va[2][8], vb[8];
        const int ta0 = threadIdx.x + 2 * TW_THREADS * rd, ta1 = ta0 + TW_THREADS;
        const int tb = threadIdx.x + TW_THREADS * rd;
        if (ta0 < totA) tw_item_load(va[0], ta0, X1, nq1, X2, nq2, row0, n);
        if (ta1 < totA) tw_item_load(va[1], ta1, X1, nq1, X2, nq2, row0, n);
        if (tb < totB) tw_item_load(vb, tb, G, nqb, nullptr, 0, row0, n);
        if (ta0 < totA) tw_item_store(sA, va[0], ta0, nq1 + nq2);
        if (ta1 < totA) tw_item_store(sA, va[1], ta1, nq1 + nq2);
        if (tb < totB) {
            tw_item_store(sB, vb, tb, nqb);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                db.x += vb[r].x;
                db.y += vb[r].y;
                db.z += vb[r].z;
                db.w += vb[r].w;
            }
        }
    }
}

template <bool PIPE>
__global__ void __launch_bounds__(TW_THREADS, TW_CTAS_PER_SM) dense_tc_bwd_weight_kernel(int64_t n, const float* __restrict__ X1,
                                                                            int K1, const float* __restrict__ X2,
                                                                            int K2, const float* __restrict__ G, int N,
                                                                            float* __restrict__ part,
                                                                            int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    const int K = K1 + K2;
    const int bufb = tw_buf_bytes(N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
    const int64_t tiles = (n + TC_M - 1) / TC_M;

    // operand rows K..127 of A stay zero in both buffers (the staging never writes them)
    if (K < TC_M) {
        const int zq = (TC_M - K) * (TC_M / 8);                 // 16-byte pieces: (rows) x (128 / 8)
        for (int t = threadIdx.x; t < 2 * zq; t += TW_THREADS) {
            const int b = t / zq, z = t - b * zq;
            const int m = K + z / (TC_M / 8), k8 = (z % (TC_M / 8)) * 8;
            *reinterpret_cast<uint4*>(smem + b * bufb + tw_off(m, k8)) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = instr_desc(TC_M, N);
    const uint32_t sbo = (uint32_t)TW_SBO;

    float4 dbs = make_float4(0.f, 0.f, 0.f, 0.f);
    bool failed = false;
    int it = 0;
    // When a tile is one round of items a thread (N <= 64), the stage is software-pipelined:
    // each item's registers take the next tile's load as soon as the item is stored, so the
    // loads stay in flight through the barrier and the MMA issue (the next tile's loads need
    // registers only; its buffer is written after the wait below).
    const int nq1 = K1 >> 2, nq2 = K2 >> 2, nqb = N >> 2;
    const int totA = (TC_M / 8) * (nq1 + nq2), totB = (TC_M / 8) * nqb;
    const int ta0 = threadIdx.x, ta1 = threadIdx.x + TW_THREADS, tb = threadIdx.x;
    float4 va0[8], va1[8], vb[8];
    if (PIPE && (int64_t)blockIdx.x < tiles) {
        const int64_t r0 = (int64_t)blockIdx.x * TC_M;
        if (ta0 < totA) tw_item_load(va0, ta0, X1, nq1, X2, nq2, r0, n);
        if (ta1 < totA) tw_item_load(va1, ta1, X1, nq1, X2, nq2, r0, n);
        if (tb < totB) tw_item_load(vb, tb, G, nqb, nullptr, 0, r0, n);
    }
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
        const int b = it & 1;
        unsigned char* sA = smem + b * bufb;
        unsigned char* sB = sA + TW_A;
        if (it >= 2) {                                          // the MMAs of tile it - 2 read this buffer
            const bool ok = mbar_wait(smem_u32(&mbar[b]), (uint32_t)(((it - 2) >> 1) & 1), 2000000000ull);
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const int64_t row0 = tile * TC_M;
        if constexpr (PIPE) {
            const int64_t nrow0 = (tile + gridDim.x) * TC_M;
            const bool more = tile + gridDim.x < tiles;
            if (ta0 < totA) {
                tw_item_store(sA, va0, ta0, nq1 + nq2);
                if (more) tw_item_load(va0, ta0, X1, nq1, X2, nq2, nrow0, n);
            }
            if (ta1 < totA) {
                tw_item_store(sA, va1, ta1, nq1 + nq2);
                if (more) tw_item_load(va1, ta1, X1, nq1, X2, nq2, nrow0, n);
            }
            if (tb < totB) {
                tw_item_store(sB, vb, tb, nqb);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    dbs.x += vb[r].x;
                    dbs.y += vb[r].y;
                    dbs.z += vb[r].z;
                    dbs.w += vb[r].w;
                }
                if (more) tw_item_load(vb, tb, G, nqb, nullptr, 0, nrow0, n);
            }
        } else {
            tw_stage(sA, sB, X1, nq1, X2, nq2, G, nqb, row0, n, dbs);
        }
        fence_proxy_async();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (threadIdx.x == 0) {
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            for (int s = 0; s < TC_M / 16; ++s) {
                const uint64_t ad = smem_desc(a0 + s * 256u, 128u, sbo);
                const uint64_t bd = smem_desc(b0 + s * 256u, 128u, sbo);
                const uint32_t acc = (it > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[b]))
                         : "memory");
        }
    }
    // the last commit covers every MMA this CTA issued
    if (!failed && it > 0) {
        const int last = it - 1;
        const bool ok = mbar_wait(smem_u32(&mbar[last & 1]), (uint32_t)((last >> 1) & 1), 2000000000ull);
        failed = __syncthreads_or(!ok);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float* pblk = part + (size_t)blockIdx.x * (size_t)(K + 1) * N;
    if (failed) {
        if (threadIdx.x == 0 && err) atomicOr(err, 2);
    } else {
        // dW rows: warp w (< 4) reads accumulator lanes 32 w .. 32 w + 31 (operand rows = inputs)
        if (warp < 4) {
            const int m = warp * 32 + lane;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t v[16];
                if (it > 0) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                        "%12, %13, %14, %15}, [%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                          "=r"(v[14]), "=r"(v[15])
                        : "r"(taddr + (uint32_t)c0));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = 0u;
                }
                if (m < K) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4)
                        *reinterpret_cast<float4*>(pblk + (size_t)m * N + c0 + q) =
                            make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]), __uint_as_float(v[q + 2]),
                                        __uint_as_float(v[q + 3]));
                }
            }
        }
        // db row: the threads owning piece q (threadIdx.x = q mod N/4) added in thread order
        float4* red = reinterpret_cast<float4*>(smem);
        red[threadIdx.x] = dbs;
        __syncthreads();
        const int nq = N >> 2;
        if (threadIdx.x < N) {
            const int q = threadIdx.x >> 2, comp = threadIdx.x & 3;
            float s = 0.f;
            for (int t = q; t < TW_THREADS; t += nq) {
                const float4 v = red[t];
                s += comp == 0 ? v.x : (comp == 1 ? v.y : (comp == 2 ? v.z : v.w));
            }
            pblk[(size_t)K * N + threadIdx.x] = s;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// dW and db from the per-CTA partials: 32 outputs per block, 8 interleaved slices of the
// partials summed by 8 threads each, then the 8 slice sums added in slice order.
constexpr int TWR_SLICES = 8;
__global__ void __launch_bounds__(256) tc_wgrad_reduce_kernel(int nparts, int K, int N, const float* __restrict__ part,
                                                             float* __restrict__ dW, float* __restrict__ db) {
    __shared__ float s[TWR_SLICES][32];
    const int outs = (K + 1) * N;
    const int o = blockIdx.x * 32 + (threadIdx.x & 31);
    const int slice = threadIdx.x >> 5;
    float acc = 0.f;
    if (o < outs)
        for (int b = slice; b < nparts; b += TWR_SLICES) acc += part[(size_t)b * outs + o];
    s[slice][threadIdx.x & 31] = acc;
    __syncthreads();
    if (threadIdx.x < 32 && o < outs) {
        float t = 0.f;
#pragma unroll
        for (int j = 0; j < TWR_SLICES; ++j) t += s[j][threadIdx.x];
        if (o < K * N) dW[o] = t;
        else if (db) db[o - K * N] = t;
    }
}

// Shared memory one launch needs: the A and B^T tiles for its K, or the epilogue rows for its
// N, whichever is larger (smaller layers fit more blocks per SM).
size_t tc_smem_bytes(int K, int N) {
    const size_t kpad = (size_t)((K + 15) & ~15);
    return tc_b_offset(K, N) + (size_t)N * kpad * 2;
}

// Shared memory of the data-gradient kernel: G's and W's tiles over N, or the epilogue rows
// of one part of at most TD_EPI_COLS columns.
size_t td_smem_bytes(int N, int kout) {
    const size_t npad = (size_t)((N + 15) & ~15);
    const size_t tiles = (size_t)TC_M * npad * 2 + (size_t)kout * npad * 2;
    const size_t stage = (size_t)TC_M * ((kout < TD_EPI_COLS ? kout : TD_EPI_COLS) + 4) * 4;
    return tiles > stage ? tiles : stage;
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_dense_forward_tc(int64_t n, const float* X1, int32_t K1, const float* X2, int32_t K2,
                                           const void* W_bf16, const float* bias, int32_t N, int32_t mode,
                                           const float* Hin, float* Y, float* U, void* stream) {
    if (n < 0 || K1 < 1 || K2 < 0 || K1 + K2 > TC_KMAX || N < 16 || N > TC_NMAX || N % 16 != 0)
        return set_error(SPX_INVALID_ARG, "spx_dense_forward_tc: sizes (K <= 128, N in 16..128, N %% 16 == 0)");
    if (mode < 0 || mode > 4) return set_error(SPX_INVALID_ARG, "spx_dense_forward_tc: mode %d (0..4)", mode);
    if (n > 0 && (!X1 || (K2 > 0 && !X2) || !W_bf16 || !Y || ((mode == 2 || mode == 4) && !U) ||
                  ((mode == 2 || mode == 3) && !Hin)))
        return set_error(SPX_INVALID_ARG, "spx_dense_forward_tc: NULL operand");
    if (K1 % 4 != 0 || K2 % 4 != 0 || !al16(X1) || (K2 > 0 && !al16(X2)) || !al16(Y) ||
        ((mode == 2 || mode == 3) && !al16(Hin)) || ((mode == 2 || mode == 4) && !al16(U)))
        return set_error(SPX_INVALID_ARG, "spx_dense_forward_tc: K1, K2 multiples of 4 and 16-byte aligned rows needed");
    if (n == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    bool launched = false;
    SPX_TRY(tc_pipe_forward(n, X1, K1, X2, K2, static_cast<const __nv_bfloat16*>(W_bf16), bias, N, mode, Hin, Y, U, st,
                            &launched));
    if (launched) return SPX_OK;
    const size_t smem = tc_smem_bytes(K1 + K2, N);
    static std::atomic<unsigned long long> attr_done{0};
    SPX_TRY(ensure_smem_attr(dense_tc_kernel, (int)tc_smem_bytes(TC_KMAX, TC_NMAX), attr_done,
                             "spx_dense_forward_tc attribute"));
    // persistent CTAs: as many as fit an SM by shared memory (and by tensor-memory columns,
    // 512 per SM), each walking its 128-row tiles
    const int64_t tiles = (n + TC_M - 1) / TC_M;
    const int ncols = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
    int per_sm = (int)((227 * 1024) / (smem + 1024));
    if (per_sm > 512 / ncols) per_sm = 512 / ncols;
    if (per_sm > 8) per_sm = 8;
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = tiles < (int64_t)per_sm * num_sms() ? tiles : (int64_t)per_sm * num_sms();
    dense_tc_kernel<<<(unsigned)grid, TC_THREADS, smem, st>>>(n, X1, K1, X2, K2,
                                                              static_cast<const __nv_bfloat16*>(W_bf16), bias, N, mode,
                                                              Hin, Y, U, device_error_word());
    SPX_CHECK_LAUNCH("spx_dense_forward_tc");
    return SPX_OK;
}

extern "C" spx_status spx_dense_backward_data_tc(int64_t n, const float* G, int32_t N, const void* W_bf16,
                                                 int32_t K1, int32_t K2, float* dX1, float* dX2, int32_t accumulate,
                                                 void* stream) {
    if (n < 0 || N < 4 || N > TC_KMAX || N % 4 != 0 || K1 < 4 || K2 < 0 || K1 % 4 != 0 || K2 % 4 != 0 ||
        K1 + K2 > TC_NMAX)
        return set_error(SPX_INVALID_ARG,
                         "spx_dense_backward_data_tc: sizes (N <= 128, K1 + K2 <= 128, all multiples of 4)");
    if (n > 0 && (!G || !W_bf16 || !dX1)) return set_error(SPX_INVALID_ARG, "spx_dense_backward_data_tc: NULL operand");
    if (n > 0 && (!al16(G) || !al16(dX1) || (dX2 && !al16(dX2))))
        return set_error(SPX_INVALID_ARG, "spx_dense_backward_data_tc: 16-byte aligned rows needed");
    if (n == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    bool launched = false;
    SPX_TRY(tc_pipe_bwd_data(n, G, N, static_cast<const __nv_bfloat16*>(W_bf16), K1, K2, dX1, dX2, accumulate, st,
                             &launched));
    if (launched) return SPX_OK;
    const int kout = ((K1 + K2) + 15) & ~15;
    const size_t smem = td_smem_bytes(N, kout);
    static std::atomic<unsigned long long> attr_done{0};
    SPX_TRY(ensure_smem_attr(dense_tc_bwd_data_kernel, TC_SMEM, attr_done, "spx_dense_backward_data_tc attribute"));
    const int64_t tiles = (n + TC_M - 1) / TC_M;
    dense_tc_bwd_data_kernel<<<(unsigned)tiles, TC_THREADS, smem, st>>>(
        n, G, N, static_cast<const __nv_bfloat16*>(W_bf16), K1, K2, dX1, dX2, accumulate, device_error_word());
    SPX_CHECK_LAUNCH("spx_dense_backward_data_tc");
    return SPX_OK;
}

extern "C" spx_status spx_dense_backward_weight_tc_workspace_size(int64_t n, int32_t K, int32_t N, size_t* bytes) {
    if (!bytes || n < 0 || K < 4 || K > TC_M || K % 4 != 0 || (N != 16 && N != 32 && N != 64 && N != 128))
        return set_error(SPX_INVALID_ARG,
                         "spx_dense_backward_weight_tc_workspace_size: sizes (K <= 128, K %% 4 == 0, N in 16/32/64/128)");
    const int64_t tiles = (n + TC_M - 1) / TC_M;
    const int64_t parts = tiles < TW_CTAS_PER_SM * num_sms() ? tiles : TW_CTAS_PER_SM * num_sms();
    *bytes = (size_t)(parts > 0 ? parts : 1) * (size_t)(K + 1) * N * 4 + 256;
    return SPX_OK;
}

extern "C" spx_status spx_dense_backward_weight_tc(int64_t n, const float* X1, int32_t K1, const float* X2, int32_t K2,
                                                   const float* G, int32_t N, float* dW, float* db, void* ws,
                                                   size_t ws_bytes, void* stream) {
    if (K1 < 4 || K1 % 4 != 0 || K2 < 0 || K2 % 4 != 0)
        return set_error(SPX_INVALID_ARG, "spx_dense_backward_weight_tc: K1, K2 multiples of 4, K1 >= 4");
    const int32_t K = K1 + K2;
    size_t need = 0;
    SPX_TRY(spx_dense_backward_weight_tc_workspace_size(n, K, N, &need));
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_dense_backward_weight_tc: workspace too small");
    if (!dW || (n > 0 && (!X1 || (K2 > 0 && !X2) || !G)))
        return set_error(SPX_INVALID_ARG, "spx_dense_backward_weight_tc: NULL operand");
    if (n > 0 && (!al16(X1) || (K2 > 0 && !al16(X2)) || !al16(G) || !al16(ws)))
        return set_error(SPX_INVALID_ARG, "spx_dense_backward_weight_tc: 16-byte aligned rows needed");
    cudaStream_t st = as_stream(stream);
    if (n == 0) {
        SPX_CUDA(cudaMemsetAsync(dW, 0, sizeof(float) * (size_t)K * N, st), "spx_dense_backward_weight_tc memset");
        if (db) SPX_CUDA(cudaMemsetAsync(db, 0, sizeof(float) * (size_t)N, st), "spx_dense_backward_weight_tc memset");
        return SPX_OK;
    }
    const int64_t tiles = (n + TC_M - 1) / TC_M;
    const int parts = (int)(tiles < TW_CTAS_PER_SM * num_sms() ? tiles : TW_CTAS_PER_SM * num_sms());
    static std::atomic<unsigned long long> attr_done{0}, attr_done_pipe{0};
    SPX_TRY(ensure_smem_attr(dense_tc_bwd_weight_kernel<false>, 2 * tw_buf_bytes(TC_NMAX), attr_done,
                             "spx_dense_backward_weight_tc attribute"));
    SPX_TRY(ensure_smem_attr(dense_tc_bwd_weight_kernel<true>, 2 * tw_buf_bytes(TC_NMAX), attr_done_pipe,
                             "spx_dense_backward_weight_tc attribute"));
    float* partial = static_cast<float*>(ws);
    // a tile of one round of items a thread (K <= 128 always; N <= 64): the pipelined stage
    const bool pipe = (TC_M / 8) * (N / 4) <= TW_THREADS && (TC_M / 8) * (K / 4) <= 2 * TW_THREADS;
    if (pipe)
        dense_tc_bwd_weight_kernel<true><<<(unsigned)parts, TW_THREADS, 2 * tw_buf_bytes(N), st>>>(
            n, X1, K1, X2, K2, G, N, partial, device_error_word());
    else
        dense_tc_bwd_weight_kernel<false><<<(unsigned)parts, TW_THREADS, 2 * tw_buf_bytes(N), st>>>(
            n, X1, K1, X2, K2, G, N, partial, device_error_word());
    SPX_CHECK_LAUNCH("spx_dense_backward_weight_tc");
    const int outs = (K + 1) * N;
    tc_wgrad_reduce_kernel<<<(unsigned)((outs + 31) / 32), 256, 0, st>>>(parts, K, N, partial, dW, db);
    SPX_CHECK_LAUNCH("spx_dense_backward_weight_tc reduce");
    return SPX_OK;
}
