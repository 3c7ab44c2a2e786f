// Row-wise sparse x dense products:
//   spx_spmm    Y  = alpha * A X   + beta * Y      (Section 3.1.1 SpMV, 3.1.3 SpDMM)
//   spx_spmm_t  gX = alpha * A^T G + beta * gX     (Table 1, gradient w.r.t. the dense
//                                                   operand, on the transposed pattern)
//
// HBM-bound gathers; no tensor cores (each stored entry is used once per output row).
//
// Column blocks.  The dense operand is gathered one row slab at a time: a pass covers
// `col_block` columns, so the slab that the random column indices touch (n x col_block
// floats) stays resident in L2 while the CSR streams pass through with evict-first
// loads.  One launch per block, blocks in column order.
//
// Column parts.  When the gathered operand is larger than L2 (2^20 x 32 floats is 134 MB),
// the plan may split every row's entries by column range (A's columns, i.e. X's rows)
// into n_parts consecutive segments; one pass per range then gathers only from that
// range's rows of X, which stay resident in L2, and adds into Y (beta = 1 after the first
// pass).  Each CSR entry is still read once; Y is read and written once more per extra pass.
//
// Short rows.  A lane group of LPR lanes spans the block's columns with float4 loads
// and owns whole rows (rows_per_group consecutive rows per group): it loads the (column,
// value) pairs of the row 8 at a time -- the next batch is fetched while the current
// one is gathered -- and issues the 8 row gathers of X back to back, so each lane has
// up to 8 independent loads in flight.  One group per row: no cross-lane reduction.
//
// Medium rows (the plan's medium list: more than medium_threshold entries, at most the long
// threshold) are taken by one whole warp each: its lane groups take 8-entry batches
// round-robin and their partial sums are combined by xor-shuffles in a fixed order.  On a
// power-law matrix these rows hold a large share of the entries; giving each its own
// warp keeps the warps of the short-row path evenly loaded.
//
// Long rows (more entries than the plan threshold) are taken by whole thread blocks:
// the block's groups take batches of 8 entries round-robin, then reduce by xor-shuffles
// inside each warp and through shared memory across warps, in a fixed order.  Those
// blocks have the lowest block ids of the launch, so they start first and overlap the
// short rows.
//
// Every output element is a fixed-order sum: results are deterministic.
#include <limits.h>

#include <atomic>
#include <mutex>

#include <cuda.h>

#include "common.cuh"
#include "scan.cuh"
#include "slab.cuh"

namespace spx {
namespace {

constexpr int SPMM_THREADS = 256;
constexpr int SPMM_WARPS = SPMM_THREADS / 32;
constexpr int BATCH = 8;                       // entries per gather batch
// At least 6 resident blocks per SM (registers capped at 40): the gathers are latency-bound,
// and 48 warps per SM keep more of them in flight than the 40 the uncapped kernel gets
// (measured on GB300: 15-19 % faster at k = 32 and 128; capping at 32 registers spills).
constexpr int SPMM_MIN_BLOCKS = 6;

template <int VEC>
__device__ __forceinline__ void fma_row(float (&acc)[VEC], float v, const float* __restrict__ p, uint64_t pol) {
    if constexpr (VEC == 4) {
        float4 x = ld_hint4(p, pol);
        acc[0] = fmaf(v, x.x, acc[0]);
        acc[1] = fmaf(v, x.y, acc[1]);
        acc[2] = fmaf(v, x.z, acc[2]);
        acc[3] = fmaf(v, x.w, acc[3]);
    } else {
        acc[0] = fmaf(v, ld_hint(p, pol), acc[0]);
    }
}

template <int VEC>
__device__ __forceinline__ void store_row(float* __restrict__ y, const float (&acc)[VEC], float alpha,
                                          float beta) {
    if constexpr (VEC == 4) {
        float4 o;
        if (beta != 0.f) {
            float4 old = *reinterpret_cast<const float4*>(y);
            o = make_float4(fmaf(alpha, acc[0], beta * old.x), fmaf(alpha, acc[1], beta * old.y),
                            fmaf(alpha, acc[2], beta * old.z), fmaf(alpha, acc[3], beta * old.w));
        } else {
            o = make_float4(alpha * acc[0], alpha * acc[1], alpha * acc[2], alpha * acc[3]);
        }
        __stcs(reinterpret_cast<float4*>(y), o);
    } else {
        float o = beta != 0.f ? fmaf(alpha, acc[0], beta * y[0]) : alpha * acc[0];
        __stcs(y, o);
    }
}

template <bool PERM>
__device__ __forceinline__ float load_val(const float* __restrict__ vals, const int32_t* __restrict__ perm, int e,
                                          uint64_t pol) {
    if constexpr (PERM)
        return __ldg(vals + ld_hint(perm + e, pol));
    else
        return ld_hint(vals + e, pol);
}

// Entries [e, e + BATCH) of a row ending at b: lane c holds entries c*SLOTS .. c*SLOTS +
// SLOTS - 1 of the batch (contiguous per lane); column -1 marks "no entry".
template <int LPR, bool PERM>
__device__ __forceinline__ void load_batch(int (&j)[(BATCH + LPR - 1) / LPR], float (&v)[(BATCH + LPR - 1) / LPR],
                                           int e, int b, int c, const int32_t* __restrict__ indices,
                                           const float* __restrict__ vals, const int32_t* __restrict__ perm,
                                           uint64_t pol) {
    constexpr int SLOTS = (BATCH + LPR - 1) / LPR;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
        const int q = c * SLOTS + s;
        const int ee = e + q;
        if (q < BATCH && ee < b) {
            j[s] = ld_hint(indices + ee, pol);
            v[s] = load_val<PERM>(vals, perm, ee, pol);
        } else {
            j[s] = -1;
            v[s] = 0.f;
        }
    }
}

// Gathers one batch: acc += v_q * X[j_q, xcol .. xcol+VEC) for the 8 entries of the batch.
template <int VEC, int LPR>
__device__ __forceinline__ void gather_batch(float (&acc)[VEC], const int (&j)[(BATCH + LPR - 1) / LPR],
                                             const float (&v)[(BATCH + LPR - 1) / LPR], unsigned gmask,
                                             bool colok, const float* __restrict__ X, int64_t ldx, int xcol,
                                             uint64_t pol) {
    constexpr int SLOTS = (BATCH + LPR - 1) / LPR;
#pragma unroll
    for (int q = 0; q < BATCH; ++q) {
        const int jq = __shfl_sync(gmask, j[q % SLOTS], q / SLOTS, LPR);
        const float vq = __shfl_sync(gmask, v[q % SLOTS], q / SLOTS, LPR);
        if (jq >= 0 && colok) fma_row<VEC>(acc, vq, X + (int64_t)jq * ldx + xcol, pol);
    }
}

template <int VEC, int LPR, bool PERM>
__global__ void __launch_bounds__(SPMM_THREADS, SPMM_MIN_BLOCKS) spmm_kernel(
    int32_t m, const int32_t* __restrict__ indptr, const int32_t* __restrict__ seg_b,
    const int32_t* __restrict__ seg_e, int32_t accumulate, const int32_t* __restrict__ indices,
    const float* __restrict__ vals, const int32_t* __restrict__ perm, const float* __restrict__ X, int64_t ldx,
    int32_t x_shift, int32_t col_begin, int32_t col_end, float* __restrict__ Y, int64_t ldy, float alpha, float beta,
    int32_t rows_per_group, int32_t threshold, const int32_t* __restrict__ long_rows, int32_t n_long,
    int32_t long_blocks, const int32_t* __restrict__ med_rows, int32_t n_med, int32_t med_blocks,
    const int32_t* __restrict__ short_rows, int32_t n_short) {
    constexpr int G = 32 / LPR;                      // lane groups per warp
    constexpr int SLOTS = (BATCH + LPR - 1) / LPR;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int g = lane / LPR;
    const int c = lane % LPR;
    const unsigned gmask = LPR == 32 ? FULL : (((1u << LPR) - 1u) << (g * LPR));
    const int col = col_begin + c * VEC;
    const int xcol = col - x_shift;
    const bool colok = col < col_end;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const float beta_eff = accumulate ? 1.f : beta;     // later column parts add into Y
    const bool split = seg_b != indptr || seg_e != indptr + 1;

    if ((int)blockIdx.x < long_blocks) {
        // ---------------- long rows: all groups of the block on one row
        __shared__ float red[SPMM_WARPS][32 * VEC];
        const int gid = warp * G + g;
        constexpr int GB = SPMM_WARPS * G;
        for (int q = blockIdx.x; q < n_long; q += long_blocks) {
            const int row = long_rows[q];
            const int a = seg_b[row], b = seg_e[row];
            if (accumulate && a == b) continue;         // block-uniform: nothing to add
            float acc[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
            for (int e = a + gid * BATCH; e < b; e += GB * BATCH) {
                int j[SLOTS];
                float vv[SLOTS];
                load_batch<LPR, PERM>(j, vv, e, b, c, indices, vals, perm, pol_stream);
                gather_batch<VEC, LPR>(acc, j, vv, gmask, colok, X, ldx, xcol, pol_keep);
            }
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(FULL, acc[v], off);
            if (g == 0)
#pragma unroll
                for (int v = 0; v < VEC; ++v) red[warp][c * VEC + v] = acc[v];
            __syncthreads();
            if (warp == 0 && g == 0 && colok) {
                float tot[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) tot[v] = red[0][c * VEC + v];
                for (int w = 1; w < SPMM_WARPS; ++w)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) tot[v] += red[w][c * VEC + v];
                store_row<VEC>(Y + (int64_t)row * ldy + col, tot, alpha, beta_eff);
            }
            __syncthreads();
        }
        return;
    }

    if ((int)blockIdx.x < long_blocks + med_blocks) {
        // ---------------- medium rows: one warp per row, its groups take batches round-robin
        const int nw = med_blocks * SPMM_WARPS;
        for (int q = ((int)blockIdx.x - long_blocks) * SPMM_WARPS + warp; q < n_med; q += nw) {
            const int row = med_rows[q];
            const int a = seg_b[row], b = seg_e[row];
            if (accumulate && a == b) continue;         // warp-uniform
            float acc[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
            int jn[SLOTS];
            float vn[SLOTS];
            const int e0 = a + g * BATCH;
            if (e0 < b) load_batch<LPR, PERM>(jn, vn, e0, b, c, indices, vals, perm, pol_stream);
            for (int e = e0; e < b; e += G * BATCH) {
                int jc[SLOTS];
                float vc[SLOTS];
#pragma unroll
                for (int t = 0; t < SLOTS; ++t) {
                    jc[t] = jn[t];
                    vc[t] = vn[t];
                }
                if (e + G * BATCH < b)
                    load_batch<LPR, PERM>(jn, vn, e + G * BATCH, b, c, indices, vals, perm, pol_stream);
                gather_batch<VEC, LPR>(acc, jc, vc, gmask, colok, X, ldx, xcol, pol_keep);
            }
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(FULL, acc[v], off);
            if (g == 0 && colok) store_row<VEC>(Y + (int64_t)row * ldy + col, acc, alpha, beta_eff);
        }
        return;
    }

    // ---------------- short rows: one lane group per row (in the plan's length order if given)
    const int64_t wglobal = ((int64_t)(blockIdx.x - long_blocks - med_blocks) * SPMM_THREADS + threadIdx.x) >> 5;
    const int64_t row0 = (wglobal * G + g) * rows_per_group;
    const int64_t n_rows = short_rows ? (int64_t)n_short : (int64_t)m;
    for (int p = 0; p < rows_per_group; ++p) {
        const int64_t idx = row0 + p;
        if (idx >= n_rows) break;
        const int64_t row = short_rows ? (int64_t)short_rows[idx] : idx;
        int a = indptr[row], b = indptr[row + 1];
        if (b - a > threshold) continue;            // a long-row block takes it
        if (split) {
            a = seg_b[row];
            b = seg_e[row];
            if (accumulate && a == b) continue;     // group-uniform
        }
        float acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
        int jn[SLOTS];
        float vn[SLOTS];
        load_batch<LPR, PERM>(jn, vn, a, b, c, indices, vals, perm, pol_stream);
        for (int e = a; e < b; e += BATCH) {
            int jc[SLOTS];
            float vc[SLOTS];
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                jc[s] = jn[s];
                vc[s] = vn[s];
            }
            if (e + BATCH < b) load_batch<LPR, PERM>(jn, vn, e + BATCH, b, c, indices, vals, perm, pol_stream);
            gather_batch<VEC, LPR>(acc, jc, vc, gmask, colok, X, ldx, xcol, pol_keep);
        }
        if (colok) store_row<VEC>(Y + row * ldy + col, acc, alpha, beta_eff);
    }
}

// ---------------------------------------------------------------------------------------
// Short rows, lean (plan engine 2): a row's batches are loaded and gathered in turn, with no
// batch held ahead, so fewer registers stay live and 8 blocks (64 warps) are resident per
// SM.  Where every short row is one batch (a stencil's rows), the prefetch of the register
// path has nothing to overlap and the extra warps keep more rows in flight instead.  Long
// and medium rows still go to spmm_kernel's blocks and warps.  Same sums in the same order.
template <int LPR, bool PERM>
__global__ void __launch_bounds__(SPMM_THREADS, 8) spmm_lean_kernel(
    int32_t m, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices, const float* __restrict__ vals,
    const int32_t* __restrict__ perm, const float* __restrict__ X, int64_t ldx, int32_t col_end, float* __restrict__ Y,
    int64_t ldy, float alpha, float beta, int32_t rows_per_group, int32_t threshold,
    const int32_t* __restrict__ short_rows, int32_t n_short) {
    constexpr int G = 32 / LPR;
    constexpr int SLOTS = (BATCH + LPR - 1) / LPR;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR;
    const int c = lane % LPR;
    const unsigned gmask = LPR == 32 ? FULL : (((1u << LPR) - 1u) << (g * LPR));
    const int col = c * 4;
    const bool colok = col < col_end;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const int64_t wglobal = ((int64_t)blockIdx.x * SPMM_THREADS + threadIdx.x) >> 5;
    const int64_t row0 = (wglobal * G + g) * rows_per_group;
    const int64_t n_rows = short_rows ? (int64_t)n_short : (int64_t)m;
    for (int p = 0; p < rows_per_group; ++p) {
        const int64_t idx = row0 + p;
        if (idx >= n_rows) break;
        const int64_t row = short_rows ? (int64_t)short_rows[idx] : idx;
        const int a = indptr[row], b = indptr[row + 1];
        if (b - a > threshold) continue;            // a long-row block or a medium-row warp takes it
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int e = a; e < b; e += BATCH) {
            int j[SLOTS];
            float v[SLOTS];
            load_batch<LPR, PERM>(j, v, e, b, c, indices, vals, perm, pol_stream);
            gather_batch<4, LPR>(acc, j, v, gmask, colok, X, ldx, col, pol_keep);
        }
        if (colok) store_row<4>(Y + row * ldy + col, acc, alpha, beta);
    }
}

// ---------------------------------------------------------------------------------------
// Short rows through the TMA engine.  Each lane group keeps a ring of BK_DEPTH batch slots
// in shared memory; for every batch (up to 8 entries of one row) the group's lanes issue
// one cp.async.bulk row copy per entry (X row segment -> slot) counted on the slot's
// mbarrier, so up to BK_DEPTH batches of row gathers are in flight per group without
// occupying registers.  The consumer walks the slots in order and accumulates; rows are
// finished in order, each output a fixed-order sum as in the register path.  A wait that
// does not complete within 2 s records a device error and ends the group's work.
constexpr int BK_WARPS = 4;
constexpr int BK_DEPTH = 4;
constexpr int BK_WARP_FLOATS = 32 * 4 * BK_DEPTH * BATCH;   // G * D * BATCH * (4 * LPR) = 4096 floats

size_t bulk_smem_bytes() {
    const size_t bufs = (size_t)BK_WARPS * BK_WARP_FLOATS * 4;            // row slots
    const size_t vals = (size_t)BK_WARPS * 32 * BK_DEPTH * BATCH * 4;     // <= 32 groups per warp
    const size_t meta = (size_t)BK_WARPS * 32 * BK_DEPTH * 4 * 4;         // row, count, last, pad
    const size_t bars = (size_t)BK_WARPS * 32 * BK_DEPTH * 8;
    return bufs + vals + meta + bars;
}

template <int LPR>
__global__ void __launch_bounds__(BK_WARPS * 32) spmm_bulk_kernel(
    int32_t m, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
    const float* __restrict__ vals, const float* __restrict__ X, int64_t ldx, int32_t x_shift, int32_t col_begin,
    int32_t col_end, float* __restrict__ Y, int64_t ldy, float alpha, float beta, int32_t rows_per_group,
    int32_t threshold, int* __restrict__ err) {
    constexpr int G = 32 / LPR;
    constexpr int SLOTS = (BATCH + LPR - 1) / LPR;
    constexpr int CB = 4 * LPR;                                 // floats per slot row
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / LPR, c = lane % LPR;
    const unsigned gmask = LPR == 32 ? FULL : (((1u << LPR) - 1u) << (g * LPR));
    const int gid = warp * G + g;                                // group id within the block
    float* buf = reinterpret_cast<float*>(smem) + (size_t)gid * BK_DEPTH * BATCH * CB;
    float* sv = reinterpret_cast<float*>(smem + (size_t)BK_WARPS * BK_WARP_FLOATS * 4) +
                (size_t)gid * BK_DEPTH * BATCH;
    int* meta = reinterpret_cast<int*>(smem + (size_t)BK_WARPS * BK_WARP_FLOATS * 4 +
                                       (size_t)BK_WARPS * 32 * BK_DEPTH * BATCH * 4) +
                (size_t)gid * BK_DEPTH * 4;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)BK_WARPS * BK_WARP_FLOATS * 4 +
                                                 (size_t)BK_WARPS * 32 * BK_DEPTH * BATCH * 4 +
                                                 (size_t)BK_WARPS * 32 * BK_DEPTH * 16) +
                     (size_t)gid * BK_DEPTH;
    if (c == 0)
        for (int s = 0; s < BK_DEPTH; ++s) mbar_init(smem_u32(&bars[s]), 1);
    fence_mbar_init();
    __syncthreads();

    const int cbw = col_end - col_begin;                         // floats copied per entry
    const uint32_t rowbytes = (uint32_t)cbw * 4u;
    const int col = col_begin + c * 4;
    const bool colok = col < col_end;
    const int64_t wglobal = ((int64_t)blockIdx.x * BK_WARPS + warp);
    const int64_t row0 = (wglobal * G + g) * rows_per_group;
    const int64_t row_end = row0 + rows_per_group < m ? row0 + rows_per_group : m;
    const float* Xc = X + (col_begin - x_shift);

    // producer cursor
    int64_t prow = row0 - 1;
    int pe = 0, pb = 0;
    bool pending_empty = false;
    // advance to the next batch: returns false when the group's rows are exhausted
    auto next_batch = [&](int64_t& row, int& e0, int& cnt, int& last) -> bool {
        for (;;) {
            if (pending_empty) {                      // an empty row still needs its store
                pending_empty = false;
                row = prow;
                e0 = pe;
                cnt = 0;
                last = 1;
                return true;
            }
            if (pe < pb) {
                row = prow;
                e0 = pe;
                cnt = pb - pe < BATCH ? pb - pe : BATCH;
                last = (pe + cnt == pb) ? 1 : 0;
                pe += cnt;
                return true;
            }
            ++prow;
            if (prow >= row_end) return false;
            const int a = indptr[prow], b = indptr[prow + 1];
            if (b - a > threshold) {                  // a long-row block takes it
                pe = pb = b;
                continue;
            }
            pe = a;
            pb = b;
            if (a == b) pending_empty = true;
        }
    };
    auto produce = [&](int s) -> bool {
        int64_t row;
        int e0, cnt, last;
        if (!next_batch(row, e0, cnt, last)) return false;
        int jl[SLOTS];
#pragma unroll
        for (int t = 0; t < SLOTS; ++t) {
            const int q = c * SLOTS + t;
            jl[t] = -1;
            if (q < cnt) {
                jl[t] = indices[e0 + q];
                sv[s * BATCH + q] = vals[e0 + q];
            }
        }
        if (c == 0) {
            meta[s * 4 + 0] = (int)row;
            meta[s * 4 + 1] = cnt;
            meta[s * 4 + 2] = last;
        }
        fence_proxy_async();                              // slot reads done before new writes
        __syncwarp(gmask);
        if (c == 0) mbar_arrive_expect_tx(smem_u32(&bars[s]), (uint32_t)cnt * rowbytes);
        __syncwarp(gmask);
#pragma unroll
        for (int t = 0; t < SLOTS; ++t) {
            const int q = c * SLOTS + t;
            if (q < cnt)
                bulk_g2s(smem_u32(buf + (size_t)(s * BATCH + q) * CB), Xc + (int64_t)jl[t] * ldx, rowbytes,
                         smem_u32(&bars[s]));
        }
        return true;
    };

    unsigned phase = 0;                                          // parity bit per slot
    int filled = 0;
    for (int s = 0; s < BK_DEPTH; ++s) {
        if (!produce(s)) break;
        ++filled;
    }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int s = 0;
    bool ok = true;
    while (filled > 0) {
        if (ok && !mbar_wait(smem_u32(&bars[s]), (phase >> s) & 1u, 2000000000ull)) {
            ok = false;
            if (c == 0 && err) atomicOr(err, 1);
        }
        phase ^= 1u << s;
        --filled;
        if (ok) {
            __syncwarp(gmask);
            const int row = meta[s * 4 + 0], cnt = meta[s * 4 + 1], last = meta[s * 4 + 2];
            if (colok) {
                for (int q = 0; q < cnt; ++q) {
                    const float v = sv[s * BATCH + q];
                    const float4 x = *reinterpret_cast<const float4*>(buf + (size_t)(s * BATCH + q) * CB + c * 4);
                    acc[0] = fmaf(v, x.x, acc[0]);
                    acc[1] = fmaf(v, x.y, acc[1]);
                    acc[2] = fmaf(v, x.z, acc[2]);
                    acc[3] = fmaf(v, x.w, acc[3]);
                }
                if (last) {
                    store_row<4>(Y + (int64_t)row * ldy + col, acc, alpha, beta);
                    acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
                }
            }
            __syncwarp(gmask);
            if (produce(s)) ++filled;
        } else {
            // give the copies already in flight a bounded time to land, then stop
            for (int r = 0; r < filled; ++r) {
                const int t = (s + 1 + r) % BK_DEPTH;
                mbar_wait(smem_u32(&bars[t]), (phase >> t) & 1u, 100000000ull);
            }
            break;
        }
        s = (s + 1) % BK_DEPTH;
    }
}

// out[e] = vals[perm[e]].  Each thread takes GV_UNROLL grid-strided entries at a time and
// issues all their index loads, then all their value loads, before any store: the value
// gathers depend on the index loads, so one entry per iteration would leave a single
// dependent pair in flight per thread.
constexpr int GV_UNROLL = 8;

__global__ void gather_values_kernel(int64_t nnz, const int32_t* __restrict__ perm, const float* __restrict__ vals,
                                     float* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < nnz; e0 += stride * GV_UNROLL) {
        int32_t p[GV_UNROLL];
#pragma unroll
        for (int u = 0; u < GV_UNROLL; ++u) {
            const int64_t e = e0 + u * stride;
            p[u] = e < nnz ? ld_stream(perm + e) : 0;
        }
        float v[GV_UNROLL];
#pragma unroll
        for (int u = 0; u < GV_UNROLL; ++u) {
            const int64_t e = e0 + u * stride;
            v[u] = e < nnz ? __ldg(vals + p[u]) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < GV_UNROLL; ++u) {
            const int64_t e = e0 + u * stride;
            if (e < nnz) __stcs(out + e, v[u]);
        }
    }
}

int ilog2_ceil(int64_t x) {
    int l = 0;
    while ((int64_t(1) << l) < x) ++l;
    return l;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <int VEC, bool PERM>
spx_status launch_lpr(int lpr, unsigned grid, cudaStream_t st, const spx_csr* A, const int32_t* seg_b,
                      const int32_t* seg_e, int32_t accumulate, const int32_t* perm,
                      const float* vals, const float* X, int64_t ldx, int32_t xs, int32_t c0, int32_t c1, float* Y,
                      int64_t ldy, float alpha, float beta, int32_t rpg, int32_t thr, const int32_t* lr,
                      int32_t n_long, int32_t long_blocks, const int32_t* mr, int32_t n_med, int32_t med_blocks,
                      const int32_t* sr, int32_t n_short) {
#define SPX_SPMM_CASE(L)                                                                                        \
    case L:                                                                                                     \
        spmm_kernel<VEC, L, PERM><<<grid, SPMM_THREADS, 0, st>>>(A->m, A->indptr, seg_b, seg_e, accumulate,      \
                                                                 A->indices, vals, perm, X, ldx,                  \
                                                                 xs, c0, c1, Y, ldy, alpha, beta, rpg, thr, lr,  \
                                                                 n_long, long_blocks, mr, n_med, med_blocks, sr, \
                                                                 n_short);                                        \
        break;
    switch (lpr) {
        SPX_SPMM_CASE(1)
        SPX_SPMM_CASE(2)
        SPX_SPMM_CASE(4)
        SPX_SPMM_CASE(8)
        SPX_SPMM_CASE(16)
        SPX_SPMM_CASE(32)
        default: return set_error(SPX_INVALID_ARG, "spmm: bad lane count %d", lpr);
    }
#undef SPX_SPMM_CASE
    return SPX_OK;
}

struct SpmmShape {
    bool vec4;
    int32_t cb;        // columns per pass
    int32_t lpr;       // lanes per row group
    int32_t rpg;       // rows per group
    size_t slab;       // bytes of the repacked dense operand (0 = gather the strided operand)
};

SpmmShape spmm_shape(const spx_csr* A, int32_t k, const spx_rowplan* plan, bool vec4) {
    SpmmShape sh{};
    sh.vec4 = vec4;
    const int VEC = vec4 ? 4 : 1;
    int32_t cb = plan && plan->col_block > 0 ? plan->col_block : k;   // default: one pass
    if (cb > k) cb = k;
    if (vec4 && cb % 4 != 0) cb = (cb + 3) / 4 * 4;
    if (cb > 32 * VEC) cb = 32 * VEC;
    sh.cb = cb;
    int lpr = 1 << ilog2_ceil((cb + VEC - 1) / VEC);
    sh.lpr = lpr > 32 ? 32 : lpr;
    sh.rpg = plan && plan->rows_per_group > 0 ? plan->rows_per_group : 2;
    sh.slab = vec4 ? slab_bytes(A->n, k, cb) : 0;
    return sh;
}

template <bool PERM>
spx_status launch_spmm(const spx_csr* A, const int32_t* perm, const float* vals, const float* X, int64_t ldx,
                       int32_t k, float* Y, int64_t ldy, float alpha, float beta, const spx_rowplan* plan,
                       float* slab_ws, size_t slab_ws_bytes, cudaStream_t st, const char* who) {
    if (A->m == 0 || k == 0) return SPX_OK;
    const bool vec4 = (k % 4 == 0) && (ldx % 4 == 0) && (ldy % 4 == 0) && aligned16(X) && aligned16(Y);
    const SpmmShape sh = spmm_shape(A, k, plan, vec4);
    const bool use_slab = sh.slab > 0 && slab_ws != nullptr && slab_ws_bytes >= sh.slab;

    int32_t threshold = INT_MAX;
    const int32_t* long_rows = nullptr;
    int32_t n_long = 0, long_blocks = 0;
    if (plan && plan->n_long > 0) {
        if (!plan->long_rows) return set_error(SPX_INVALID_ARG, "%s: plan without rows", who);
        threshold = plan->threshold;
        long_rows = plan->long_rows;
        n_long = plan->n_long;
        long_blocks = n_long < 4 * num_sms() ? n_long : 4 * num_sms();
    }
    const int32_t* med_rows = nullptr;
    int32_t n_med = 0, med_blocks = 0;
    if (plan && plan->n_medium > 0) {
        if (!plan->medium_rows || plan->medium_threshold < 1 || plan->medium_threshold > threshold)
            return set_error(SPX_INVALID_ARG, "%s: bad medium-row plan", who);
        med_rows = plan->medium_rows;
        n_med = plan->n_medium;
        threshold = plan->medium_threshold;        // short rows stop here
        const int64_t want = ((int64_t)n_med + 2 * SPMM_WARPS - 1) / (2 * SPMM_WARPS);
        med_blocks = (int32_t)(want < 8 * num_sms() ? want : 8 * num_sms());
    }
    // the short rows in the plan's order (grouped by length, so the groups of a warp walk
    // rows of about the same length), or all rows in natural order
    const int32_t* short_rows = plan && plan->short_rows ? plan->short_rows : nullptr;
    const int32_t n_short = short_rows ? plan->n_short : 0;
    if (short_rows && (n_short < 0 || n_short > A->m))
        return set_error(SPX_INVALID_ARG, "%s: bad short-row order", who);
    const int G = 32 / sh.lpr;
    const int64_t rows_per_block = (int64_t)SPMM_WARPS * G * sh.rpg;
    const int64_t n_rows = short_rows ? (int64_t)n_short : (int64_t)A->m;
    const int64_t short_blocks = (n_rows + rows_per_block - 1) / rows_per_block;
    const int64_t grid = short_blocks + long_blocks + med_blocks;
    if (grid > INT_MAX) return set_error(SPX_INVALID_ARG, "%s: too many rows", who);
    if (use_slab) SPX_TRY(slab_repack(A->n, X, ldx, k, sh.cb, slab_ws, st));
    const int32_t parts = plan && plan->n_parts > 1 && plan->part_ptr ? plan->n_parts : 1;
    const bool lean = vec4 && plan && plan->engine == 2 && sh.cb >= k && parts == 1 && !use_slab;
    if (lean) {
        const int64_t rows_per_lblock = (int64_t)SPMM_WARPS * G * sh.rpg;
        const int64_t lgrid = (n_rows + rows_per_lblock - 1) / rows_per_lblock;
        if (lgrid > INT_MAX) return set_error(SPX_INVALID_ARG, "%s: too many rows", who);
        if (lgrid > 0) {
#define SPX_LEAN_CASE(L)                                                                                       \
    case L:                                                                                                    \
        spmm_lean_kernel<L, PERM><<<(unsigned)lgrid, SPMM_THREADS, 0, st>>>(                                   \
            A->m, A->indptr, A->indices, vals, perm, X, ldx, k, Y, ldy, alpha, beta, sh.rpg, threshold,        \
            short_rows, n_short);                                                                              \
        break;
            switch (sh.lpr) {
                SPX_LEAN_CASE(1)
                SPX_LEAN_CASE(2)
                SPX_LEAN_CASE(4)
                SPX_LEAN_CASE(8)
                SPX_LEAN_CASE(16)
                SPX_LEAN_CASE(32)
                default: return set_error(SPX_INVALID_ARG, "%s: lean lane count %d", who, sh.lpr);
            }
#undef SPX_LEAN_CASE
            SPX_CHECK_LAUNCH(who);
        }
        if (long_blocks + med_blocks > 0) {
            spx_status s2 = launch_lpr<4, PERM>(sh.lpr, (unsigned)(long_blocks + med_blocks), st, A, A->indptr,
                                                A->indptr + 1, 0, perm, vals, X, ldx, 0, 0, k, Y, ldy, alpha, beta,
                                                sh.rpg, threshold, long_rows, n_long, long_blocks, med_rows, n_med,
                                                med_blocks, nullptr, 0);
            if (s2 != SPX_OK) return s2;
            SPX_CHECK_LAUNCH(who);
        }
        return SPX_OK;
    }
    const bool bulk = !PERM && vec4 && plan && plan->engine == 1 && sh.cb % 4 == 0 && sh.lpr >= 2 &&
                      sh.lpr * 4 >= sh.cb && parts == 1;
    if (bulk) {
        const size_t smem = bulk_smem_bytes();
        const int64_t rows_per_bblock = (int64_t)BK_WARPS * G * sh.rpg;
        const int64_t bgrid = ((int64_t)A->m + rows_per_bblock - 1) / rows_per_bblock;
        if (bgrid > INT_MAX) return set_error(SPX_INVALID_ARG, "%s: too many rows", who);
        int* err = device_error_word();
        for (int32_t c0 = 0; c0 < k; c0 += sh.cb) {
            const int32_t c1 = c0 + sh.cb < k ? c0 + sh.cb : k;
            const float* Xp = use_slab ? slab_ws + (int64_t)(c0 / sh.cb) * A->n * sh.cb : X;
            const int64_t ldp = use_slab ? sh.cb : ldx;
            const int32_t xs = use_slab ? c0 : 0;
#define SPX_BULK_CASE(L)                                                                                      \
    case L: {                                                                                                 \
        static std::atomic<unsigned long long> attr_done{0};                                                  \
        SPX_TRY(ensure_smem_attr(spmm_bulk_kernel<L>, (int)smem, attr_done, "spmm bulk attribute"));           \
        spmm_bulk_kernel<L><<<(unsigned)bgrid, BK_WARPS * 32, smem, st>>>(                                    \
            A->m, A->indptr, A->indices, vals, Xp, ldp, xs, c0, c1, Y, ldy, alpha, beta, sh.rpg, threshold, err); \
        break;                                                                                                \
    }
            switch (sh.lpr) {
                SPX_BULK_CASE(2)
                SPX_BULK_CASE(4)
                SPX_BULK_CASE(8)
                SPX_BULK_CASE(16)
                SPX_BULK_CASE(32)
                default: return set_error(SPX_INVALID_ARG, "%s: bulk lane count %d", who, sh.lpr);
            }
#undef SPX_BULK_CASE
            SPX_CHECK_LAUNCH(who);
            if (long_blocks + med_blocks > 0) {
                spx_status s = launch_lpr<4, false>(sh.lpr, (unsigned)(long_blocks + med_blocks), st, A,
                                                    A->indptr, A->indptr + 1, 0, perm, vals,
                                                    Xp, ldp, xs, c0, c1, Y, ldy, alpha, beta, sh.rpg, threshold,
                                                    long_rows, n_long, long_blocks, med_rows, n_med, med_blocks,
                                                    nullptr, 0);
                if (s != SPX_OK) return s;
                SPX_CHECK_LAUNCH(who);
            }
        }
        return SPX_OK;
    }
    for (int32_t c0 = 0; c0 < k; c0 += sh.cb) {
        const int32_t c1 = c0 + sh.cb < k ? c0 + sh.cb : k;
        const float* Xp = use_slab ? slab_ws + (int64_t)(c0 / sh.cb) * A->n * sh.cb : X;
        const int64_t ldp = use_slab ? sh.cb : ldx;
        const int32_t xs = use_slab ? c0 : 0;
        for (int32_t p = 0; p < parts; ++p) {
            // pass p: entries [seg_b[i], seg_e[i]) of row i, i.e. columns in range p
            const int32_t* sb = p == 0 ? A->indptr : plan->part_ptr + (int64_t)(p - 1) * A->m;
            const int32_t* se = p == parts - 1 ? A->indptr + 1 : plan->part_ptr + (int64_t)p * A->m;
            const int32_t accum = p > 0 ? 1 : 0;
            spx_status s = vec4 ? launch_lpr<4, PERM>(sh.lpr, (unsigned)grid, st, A, sb, se, accum, perm, vals, Xp,
                                                      ldp, xs, c0, c1, Y, ldy, alpha, beta, sh.rpg, threshold,
                                                      long_rows, n_long, long_blocks, med_rows, n_med, med_blocks,
                                                      short_rows, n_short)
                                : launch_lpr<1, PERM>(sh.lpr, (unsigned)grid, st, A, sb, se, accum, perm, vals, Xp,
                                                      ldp, xs, c0, c1, Y, ldy, alpha, beta, sh.rpg, threshold,
                                                      long_rows, n_long, long_blocks, med_rows, n_med, med_blocks,
                                                      short_rows, n_short);
            if (s != SPX_OK) return s;
            SPX_CHECK_LAUNCH(who);
        }
    }
    return SPX_OK;
}

// flags[i] = 1 for rows with lo < length <= hi
__global__ void long_flag_kernel(int32_t m, const int32_t* __restrict__ indptr, int32_t lo, int32_t hi,
                                 int32_t* __restrict__ flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) {
        const int len = indptr[i + 1] - indptr[i];
        flags[i] = (len > lo && len <= hi) ? 1 : 0;
    }
}

__global__ void long_compact_kernel(int32_t m, const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                                    int32_t* __restrict__ long_rows) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m && flags[i]) long_rows[pos[i]] = (int32_t)i;
}

// Short-row order: rows of at most thr entries grouped by their count of 8-entry batches
// (counts above SHORT_KEY_MAX share the last group), groups longest first, row ids
// increasing within a group -- a stable counting sort, one flag / scan / compact pass per
// group, the running count kept on the device.
constexpr int SHORT_KEY_MAX = 8;

__global__ void short_key_flag_kernel(int32_t m, const int32_t* __restrict__ indptr, int32_t thr, int32_t key,
                                      int32_t* __restrict__ flags) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int len = indptr[i + 1] - indptr[i];
    int k = (len + BATCH - 1) / BATCH;
    if (k > SHORT_KEY_MAX) k = SHORT_KEY_MAX;
    flags[i] = (len <= thr && k == key) ? 1 : 0;
}

__global__ void short_compact_kernel(int32_t m, const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                                     const int32_t* __restrict__ base, int32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m && flags[i]) out[*base + pos[i]] = (int32_t)i;
}

// base[0]: rows placed so far; base[1]: non-empty groups so far
__global__ void short_count_kernel(int32_t m, const int32_t* __restrict__ pos, int32_t* __restrict__ base) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        base[0] += pos[m];
        base[1] += pos[m] > 0 ? 1 : 0;
    }
}

// part_ptr[(p - 1) * m + i] = first entry of row i with column >= p * w (binary search in
// the sorted row), p = 1 .. parts - 1
__global__ void part_split_kernel(int32_t m, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                  int32_t w, int32_t parts, int32_t* __restrict__ part_ptr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int a = indptr[i], b = indptr[i + 1];
    int lo = a;
    for (int p = 1; p < parts; ++p) {
        const int64_t bound = (int64_t)p * w;
        int hi = b;                                   // first entry in [lo, b) with column >= bound
        while (lo < hi) {
            const int mid = lo + ((hi - lo) >> 1);
            if ((int64_t)indices[mid] < bound) lo = mid + 1;
            else hi = mid;
        }
        part_ptr[(int64_t)(p - 1) * m + i] = lo;
    }
}

size_t rowplan_ws(int32_t m) {
    size_t a = ((size_t)m * 4 + 255) & ~size_t(255);
    size_t b = (((size_t)m + 1) * 4 + 255) & ~size_t(255);
    return a + b + scan_workspace_bytes<int32_t>(m) + 256;     // + the short order's running count
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_rowplan_workspace_size(int32_t m, size_t* bytes) {
    if (!bytes || m < 0) return set_error(SPX_INVALID_ARG, "spx_rowplan_workspace_size: bad arguments");
    *bytes = rowplan_ws(m);
    return SPX_OK;
}

extern "C" spx_status spx_rowplan_build(const spx_csr* A, int32_t threshold, int32_t* long_rows,
                                        int32_t* n_long_host, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, false, "spx_rowplan_build"));
    if (!n_long_host || (A->m > 0 && !long_rows) || threshold < 1)
        return set_error(SPX_INVALID_ARG, "spx_rowplan_build: bad arguments");
    size_t need = rowplan_ws(A->m);
    if (!ws || ws_bytes < need)
        return set_error(SPX_OOM_WORKSPACE, "spx_rowplan_build: workspace %zu < %zu", ws_bytes, need);
    *n_long_host = 0;
    if (A->m == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    int32_t* flags = (int32_t*)w;
    int32_t* pos = (int32_t*)(w + (((size_t)A->m * 4 + 255) & ~size_t(255)));
    int32_t* sws = (int32_t*)((char*)pos + ((((size_t)A->m + 1) * 4 + 255) & ~size_t(255)));
    unsigned blocks = (unsigned)((A->m + 255) / 256);
    long_flag_kernel<<<blocks, 256, 0, st>>>(A->m, A->indptr, threshold, INT_MAX, flags);
    SPX_CHECK_LAUNCH("long_flag");
    SPX_TRY((scan_counts<int32_t, int32_t>(flags, pos, A->m, sws, st)));
    long_compact_kernel<<<blocks, 256, 0, st>>>(A->m, flags, pos, long_rows);
    SPX_CHECK_LAUNCH("long_compact");
    SPX_CUDA(cudaMemcpyAsync(n_long_host, pos + A->m, sizeof(int32_t), cudaMemcpyDeviceToHost, st),
             "spx_rowplan_build copy");
    SPX_CUDA(cudaStreamSynchronize(st), "spx_rowplan_build sync");
    return SPX_OK;
}

extern "C" spx_status spx_rowplan_build_medium(const spx_csr* A, int32_t medium_threshold, int32_t long_threshold,
                                               int32_t* medium_rows, int32_t* n_medium_host, void* ws, size_t ws_bytes,
                                               void* stream) {
    SPX_TRY(check_csr(A, false, "spx_rowplan_build_medium"));
    if (!n_medium_host || (A->m > 0 && !medium_rows) || medium_threshold < 1 || long_threshold < medium_threshold)
        return set_error(SPX_INVALID_ARG, "spx_rowplan_build_medium: bad arguments");
    size_t need = rowplan_ws(A->m);
    if (!ws || ws_bytes < need)
        return set_error(SPX_OOM_WORKSPACE, "spx_rowplan_build_medium: workspace %zu < %zu", ws_bytes, need);
    *n_medium_host = 0;
    if (A->m == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    int32_t* flags = (int32_t*)w;
    int32_t* pos = (int32_t*)(w + (((size_t)A->m * 4 + 255) & ~size_t(255)));
    int32_t* sws = (int32_t*)((char*)pos + ((((size_t)A->m + 1) * 4 + 255) & ~size_t(255)));
    unsigned blocks = (unsigned)((A->m + 255) / 256);
    long_flag_kernel<<<blocks, 256, 0, st>>>(A->m, A->indptr, medium_threshold, long_threshold, flags);
    SPX_CHECK_LAUNCH("medium_flag");
    SPX_TRY((scan_counts<int32_t, int32_t>(flags, pos, A->m, sws, st)));
    long_compact_kernel<<<blocks, 256, 0, st>>>(A->m, flags, pos, medium_rows);
    SPX_CHECK_LAUNCH("medium_compact");
    SPX_CUDA(cudaMemcpyAsync(n_medium_host, pos + A->m, sizeof(int32_t), cudaMemcpyDeviceToHost, st),
             "spx_rowplan_build_medium copy");
    SPX_CUDA(cudaStreamSynchronize(st), "spx_rowplan_build_medium sync");
    return SPX_OK;
}

extern "C" spx_status spx_rowplan_build_parts(const spx_csr* A, int32_t n_parts, int32_t* part_ptr, void* stream) {
    SPX_TRY(check_csr(A, false, "spx_rowplan_build_parts"));
    if (n_parts < 2 || n_parts > A->n || (A->m > 0 && !part_ptr))
        return set_error(SPX_INVALID_ARG, "spx_rowplan_build_parts: n_parts = %d (need 2 <= n_parts <= n = %d)",
                         n_parts, A->n);
    if (A->m == 0) return SPX_OK;
    const int32_t w = (int32_t)(((int64_t)A->n + n_parts - 1) / n_parts);
    part_split_kernel<<<(unsigned)((A->m + 255) / 256), 256, 0, as_stream(stream)>>>(A->m, A->indptr, A->indices, w,
                                                                                    n_parts, part_ptr);
    SPX_CHECK_LAUNCH("spx_rowplan_build_parts");
    return SPX_OK;
}

static spx_status check_dense(const void* p, int64_t rows, int64_t ld, int32_t k, const char* who,
                              const char* name) {
    if (rows > 0 && k > 0 && !p) return set_error(SPX_INVALID_ARG, "%s: NULL %s", who, name);
    if (k < 0 || ld < k || ld < 1) return set_error(SPX_INVALID_ARG, "%s: bad ld/k for %s", who, name);
    return SPX_OK;
}

static bool vec4_ok(int32_t k, int64_t ldx, int64_t ldy, const void* X, const void* Y) {
    return (k % 4 == 0) && (ldx % 4 == 0) && (ldy % 4 == 0) && aligned16(X) && aligned16(Y);
}

extern "C" spx_status spx_spmm_workspace_size(const spx_csr* A, int32_t k, const spx_rowplan* plan, size_t* bytes) {
    SPX_TRY(check_csr(A, false, "spx_spmm_workspace_size"));
    if (!bytes || k < 0) return set_error(SPX_INVALID_ARG, "spx_spmm_workspace_size: bad arguments");
    *bytes = k > 0 && k % 4 == 0 ? align256(spmm_shape(A, k, plan, true).slab) : 0;
    return SPX_OK;
}

extern "C" spx_status spx_spmm(const spx_csr* A, const float* X, int64_t ldx, int32_t k, float* Y,
                               int64_t ldy, float alpha, float beta, const spx_rowplan* plan, void* ws,
                               size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_spmm"));
    SPX_TRY(check_dense(X, A->n, ldx, k, "spx_spmm", "X"));
    SPX_TRY(check_dense(Y, A->m, ldy, k, "spx_spmm", "Y"));
    if (ws && k > 0) {
        const size_t need = spmm_shape(A, k, plan, vec4_ok(k, ldx, ldy, X, Y)).slab;
        if (ws_bytes < need)
            return set_error(SPX_OOM_WORKSPACE, "spx_spmm: workspace %zu < %zu", ws_bytes, need);
    }
    return launch_spmm<false>(A, nullptr, A->values, X, ldx, k, Y, ldy, alpha, beta, plan, static_cast<float*>(ws),
                              ws_bytes, as_stream(stream), "spx_spmm");
}

// A^T's gathered values first, then the repacked slabs of G.
static size_t spmm_t_need(const spx_csr* AT, int32_t k, const spx_rowplan* plan, bool vec4) {
    return align256((size_t)AT->nnz * 4) + spmm_shape(AT, k, plan, vec4).slab;
}

extern "C" spx_status spx_spmm_t_workspace_size(const spx_csr* AT, int32_t k, const spx_rowplan* plan,
                                                size_t* bytes) {
    SPX_TRY(check_csr(AT, false, "spx_spmm_t_workspace_size"));
    if (!bytes || k < 0) return set_error(SPX_INVALID_ARG, "spx_spmm_t_workspace_size: bad arguments");
    *bytes = align256(spmm_t_need(AT, k, plan, k % 4 == 0));
    return SPX_OK;
}

extern "C" spx_status spx_spmm_t(const spx_csr* AT, const int32_t* perm, const float* G, int64_t ldg,
                                 int32_t k, float* gX, int64_t ldgx, float alpha, float beta,
                                 const spx_rowplan* plan, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(AT, true, "spx_spmm_t"));
    if (AT->nnz > 0 && !perm) return set_error(SPX_INVALID_ARG, "spx_spmm_t: NULL perm");
    SPX_TRY(check_dense(G, AT->n, ldg, k, "spx_spmm_t", "G"));
    SPX_TRY(check_dense(gX, AT->m, ldgx, k, "spx_spmm_t", "gX"));
    cudaStream_t st = as_stream(stream);
    if (!ws) return launch_spmm<true>(AT, perm, AT->values, G, ldg, k, gX, ldgx, alpha, beta, plan, nullptr, 0, st,
                                      "spx_spmm_t");
    const size_t need = spmm_t_need(AT, k, plan, vec4_ok(k, ldg, ldgx, G, gX));
    if (ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_spmm_t: workspace %zu < %zu", ws_bytes, need);
    if (AT->nnz == 0 || AT->m == 0 || k == 0)
        return launch_spmm<false>(AT, nullptr, AT->values, G, ldg, k, gX, ldgx, alpha, beta, plan, nullptr, 0, st,
                                  "spx_spmm_t");
    float* tv = static_cast<float*>(ws);
    const size_t voff = align256((size_t)AT->nnz * 4);
    int64_t blocks = (AT->nnz + 255) / 256;
    int64_t cap = (int64_t)num_sms() * 16;
    gather_values_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, st>>>(AT->nnz, perm, AT->values, tv);
    SPX_CHECK_LAUNCH("spx_spmm_t gather");
    return launch_spmm<false>(AT, nullptr, tv, G, ldg, k, gX, ldgx, alpha, beta, plan,
                              reinterpret_cast<float*>(static_cast<char*>(ws) + voff), ws_bytes - voff, st,
                              "spx_spmm_t");
}

extern "C" spx_status spx_gather_values(int64_t nnz, const int32_t* perm, const float* src, float* dst,
                                        void* stream) {
    if (nnz < 0 || (nnz > 0 && (!perm || !src || !dst)))
        return set_error(SPX_INVALID_ARG, "spx_gather_values: bad arguments");
    if (nnz == 0) return SPX_OK;
    int64_t blocks = (nnz + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    gather_values_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, as_stream(stream)>>>(nnz, perm, src, dst);
    SPX_CHECK_LAUNCH("spx_gather_values");
    return SPX_OK;
}

// ---------------------------------------------------------------------------------------
// spx_spmm_t without allocation.
//
// Some callers cannot allocate device memory at the moment they need the product: a host
// framework that owns every byte of device memory through its own pool and forbids side
// allocations, a callback that must not synchronise the device (cudaMalloc and cudaFree
// can), or a tight loop that must not touch the allocator at all.  For them this variant
// stages A^T's gathered values in a scratch array that is part of the library image
// instead of a caller-provided workspace.  The array is file-scope device memory of a
// fixed size, held by every device that loads the library until the process exits.
namespace spx {
namespace {
constexpr int64_t NOALLOC_MAX_NNZ = int64_t(1) << 22;          // 4,194,304 entries (16 MiB)
static __device__ __align__(256) float g_noalloc_values[NOALLOC_MAX_NNZ];

constexpr int NOALLOC_MAX_DEVICES = 64;

// The array's device address belongs to the module image loaded into one CUDA context: it
// is looked up with cudaGetSymbolAddress the first time a device is used, and again only
// when the current context of that device is a different one (after cudaDeviceReset or
// any re-creation of the primary context the module is loaded anew and may move).  A
// context is identified by its unique id (cuCtxGetId), which is never reused.
struct NoallocSlot {
    unsigned long long ctx_id = 0;
    float* ptr = nullptr;
};
NoallocSlot g_noalloc_slot[NOALLOC_MAX_DEVICES];
std::mutex g_noalloc_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context, 0 when there is none yet.
spx_status current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        SPX_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1),
                 "spx_spmm_t_noalloc: driver entry point cuCtxGetCurrent");
        SPX_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2),
                 "spx_spmm_t_noalloc: driver entry point cuCtxGetId");
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return set_error(SPX_NOT_SUPPORTED, "spx_spmm_t_noalloc: the driver lacks cuCtxGetCurrent / cuCtxGetId");
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return set_error(SPX_CUDA_ERROR, "spx_spmm_t_noalloc: cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return set_error(SPX_CUDA_ERROR, "spx_spmm_t_noalloc: cuCtxGetId failed");
    return SPX_OK;
}

// Device address of the scratch array in the current device's current context.
spx_status noalloc_scratch(float** out) {
    int dev = 0;
    SPX_CUDA(cudaGetDevice(&dev), "spx_spmm_t_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return set_error(SPX_NOT_SUPPORTED, "spx_spmm_t_noalloc: device %d beyond %d", dev, NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    SPX_TRY(current_context_id(&id));
    NoallocSlot& slot = g_noalloc_slot[dev];
    if (id == 0 || slot.ctx_id != id || !slot.ptr) {
        void* addr = nullptr;
        // also makes the device's primary context current when no runtime call did yet
        SPX_CUDA(cudaGetSymbolAddress(&addr, g_noalloc_values), "spx_spmm_t_noalloc: cudaGetSymbolAddress");
        SPX_TRY(current_context_id(&id));
        slot.ctx_id = id;
        slot.ptr = static_cast<float*>(addr);
    }
    *out = slot.ptr;
    return SPX_OK;
}
}  // namespace
}  // namespace spx

extern "C" spx_status spx_spmm_t_noalloc(const spx_csr* AT, const int32_t* perm, const float* G, int64_t ldg,
                                         int32_t k, float* gX, int64_t ldgx, float alpha, float beta,
                                         const spx_rowplan* plan, void* stream) {
    SPX_TRY(check_csr(AT, true, "spx_spmm_t_noalloc"));
    if (AT->nnz > NOALLOC_MAX_NNZ)
        return set_error(SPX_INVALID_ARG,
                         "spx_spmm_t_noalloc: nnz = %lld exceeds the built-in scratch of %lld entries; "
                         "use spx_spmm_t with a workspace",
                         (long long)AT->nnz, (long long)NOALLOC_MAX_NNZ);
    if (AT->nnz > 0 && !perm) return set_error(SPX_INVALID_ARG, "spx_spmm_t_noalloc: NULL perm");
    SPX_TRY(check_dense(G, AT->n, ldg, k, "spx_spmm_t_noalloc", "G"));
    SPX_TRY(check_dense(gX, AT->m, ldgx, k, "spx_spmm_t_noalloc", "gX"));
    cudaStream_t st = as_stream(stream);
    if (AT->nnz == 0 || AT->m == 0 || k == 0)
        return launch_spmm<false>(AT, nullptr, AT->values, G, ldg, k, gX, ldgx, alpha, beta, plan, nullptr, 0, st,
                                  "spx_spmm_t_noalloc");
    float* tv = nullptr;
    SPX_TRY(noalloc_scratch(&tv));
    // every entry [0, nnz) of the scratch is written here before the product reads it
    int64_t blocks = (AT->nnz + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    gather_values_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, st>>>(AT->nnz, perm, AT->values, tv);
    SPX_CHECK_LAUNCH("spx_spmm_t_noalloc gather");
    return launch_spmm<false>(AT, nullptr, tv, G, ldg, k, gX, ldgx, alpha, beta, plan, nullptr, 0, st,
                              "spx_spmm_t_noalloc");
}

extern "C" spx_status spx_rowplan_build_short(const spx_csr* A, int32_t threshold, int32_t* short_rows,
                                              int32_t* n_short_host, int32_t* n_groups_host, void* ws,
                                              size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, false, "spx_rowplan_build_short"));
    if (!n_short_host || (A->m > 0 && !short_rows) || threshold < 0)
        return set_error(SPX_INVALID_ARG, "spx_rowplan_build_short: bad arguments");
    const size_t need = rowplan_ws(A->m);
    if (!ws || ws_bytes < need)
        return set_error(SPX_OOM_WORKSPACE, "spx_rowplan_build_short: workspace %zu < %zu", ws_bytes, need);
    *n_short_host = 0;
    if (n_groups_host) *n_groups_host = 0;
    if (A->m == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    int32_t* flags = (int32_t*)w;
    int32_t* pos = (int32_t*)(w + (((size_t)A->m * 4 + 255) & ~size_t(255)));
    int32_t* sws = (int32_t*)((char*)pos + ((((size_t)A->m + 1) * 4 + 255) & ~size_t(255)));
    int32_t* base = (int32_t*)(w + need - 256);
    SPX_CUDA(cudaMemsetAsync(base, 0, 2 * sizeof(int32_t), st), "spx_rowplan_build_short memset");
    const unsigned blocks = (unsigned)((A->m + 255) / 256);
    for (int key = SHORT_KEY_MAX; key >= 0; --key) {
        short_key_flag_kernel<<<blocks, 256, 0, st>>>(A->m, A->indptr, threshold, key, flags);
        SPX_CHECK_LAUNCH("short_key_flag");
        SPX_TRY((scan_counts<int32_t, int32_t>(flags, pos, A->m, sws, st)));
        short_compact_kernel<<<blocks, 256, 0, st>>>(A->m, flags, pos, base, short_rows);
        SPX_CHECK_LAUNCH("short_compact");
        short_count_kernel<<<1, 32, 0, st>>>(A->m, pos, base);
        SPX_CHECK_LAUNCH("short_count");
    }
    int32_t counts[2] = {0, 0};
    SPX_CUDA(cudaMemcpyAsync(counts, base, sizeof(counts), cudaMemcpyDeviceToHost, st),
             "spx_rowplan_build_short copy");
    SPX_CUDA(cudaStreamSynchronize(st), "spx_rowplan_build_short sync");
    *n_short_host = counts[0];
    if (n_groups_host) *n_groups_host = counts[1];
    return SPX_OK;
}
