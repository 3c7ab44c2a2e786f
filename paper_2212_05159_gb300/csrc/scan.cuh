// Device-wide prefix sums used to turn per-row / per-column counts into CSR offsets.
//
// scan_counts(in[0..n), out[0..n]) writes out[0] = 0 and out[i+1] = in[0] + ... + in[i].
// Three phases per level (tile reduce, scan of the tile sums, tile scan with offsets),
// recursing on the tile sums; deterministic (integer sums).
#pragma once

#include "common.cuh"

namespace spx {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* smem_warp, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) smem_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (SCAN_THREADS / 32) ? smem_warp[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < (SCAN_THREADS / 32)) smem_warp[lane] = wi - w;
        if (lane == (SCAN_THREADS / 32) - 1) smem_warp[SCAN_THREADS / 32] = wi;
    }
    __syncthreads();
    T res = smem_warp[warp] + inc - v;
    if (total) *total = smem_warp[SCAN_THREADS / 32];
    return res;
}

template <typename Tin, typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_kernel(const Tin* __restrict__ in, int64_t n,
                                                                   T* __restrict__ sums) {
    __shared__ T sw[SCAN_THREADS / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int64_t i = base + (int64_t)q * SCAN_THREADS + threadIdx.x;
        if (i < n) s += (T)in[i];
    }
    T tot;
    block_exclusive_sum<T>(s, sw, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// out[i+1] = offset + inclusive sum; block 0 also writes out[0] = 0 when first_zero.
template <typename Tin, typename T>
__global__ void __launch_bounds__(SCAN_THREADS) scan_tile_kernel(const Tin* __restrict__ in, int64_t n,
                                                                 const T* __restrict__ offsets,
                                                                 T* __restrict__ out) {
    __shared__ T sw[SCAN_THREADS / 32 + 1];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    // blocked arrangement: thread t owns items [t*ITEMS, (t+1)*ITEMS) of the tile
    T v[SCAN_ITEMS];
    T s = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + q;
        v[q] = i < n ? (T)in[i] : T(0);
        s += v[q];
    }
    T ex = block_exclusive_sum<T>(s, sw, (T*)nullptr);
    T off = offsets ? offsets[blockIdx.x] : T(0);
    T run = off + ex;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + q;
        run += v[q];
        if (i < n) out[i + 1] = run;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = T(0);
}

// Workspace elements of type T needed to scan n items (all recursion levels).
inline int64_t scan_workspace_elems(int64_t n) {
    int64_t tot = 0;
    while (n > SCAN_TILE) {
        int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
        tot += 2 * tiles + 1;
        n = tiles;
    }
    return tot + 1;
}

template <typename T>
inline size_t scan_workspace_bytes(int64_t n) {
    return (size_t)scan_workspace_elems(n) * sizeof(T) + 256;
}

// Exclusive scan of n counts into out[0..n]; ws holds scan_workspace_bytes<T>(n).
template <typename Tin, typename T>
spx_status scan_counts(const Tin* in, T* out, int64_t n, T* ws, cudaStream_t st) {
    if (n <= SCAN_TILE) {
        scan_tile_kernel<Tin, T><<<1, SCAN_THREADS, 0, st>>>(in, n, (const T*)nullptr, out);
        SPX_CHECK_LAUNCH("scan_tile");
        return SPX_OK;
    }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    T* sums = ws;             // tiles entries
    T* offs = ws + tiles;     // tiles + 1 entries (scanned sums)
    T* rest = offs + tiles + 1;
    scan_reduce_kernel<Tin, T><<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, n, sums);
    SPX_CHECK_LAUNCH("scan_reduce");
    SPX_TRY((scan_counts<T, T>(sums, offs, tiles, rest, st)));
    scan_tile_kernel<Tin, T><<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, n, offs, out);
    SPX_CHECK_LAUNCH("scan_tile");
    return SPX_OK;
}

}  // namespace spx
