// Both reverse-mode products of Y = A X in one pass (Table 1, SpDMM rows):
//   gX = alpha * A^T G + beta * gX        (gradient w.r.t. the dense operand)
//   gA = scale * (G X^T) masked to A       (gradient w.r.t. A's values, on A's pattern)
// Each stored entry a_ij of A couples row i of G with row j of X.  Walking A^T row by row
// (row j of A^T = column j of A), both products need the same gathered rows G_i: gX_j
// accumulates a_ij G_i, and gA_ij is the dot product of that G_i with X_j, which is
// contiguous and read once per row.  So the pass gathers one random stream (the rows of G)
// where the separate SDDMM and A^T G gather two (X's rows for the SDDMM, G's for A^T G), and
// it reads A's values through the transpose permutation, which also says where each gA_ij
// goes in A's order.
//
// Lane groups of LPR lanes span the k columns with float4 loads (k / 4 <= LPR <= 32, LPR >= 8)
// and take a row's entries LPR at a time: lane c holds entry e + c (its row i of A, its
// position p in A, and A's value there), the next batch is loaded while the current one's
// rows of G are in flight; every lane gathers the LPR rows of the batch for its columns,
// accumulates a_ij G_i and forms the LPR partial dot products with its slice of X_j; a
// butterfly transpose across the group (LPR - 1 shuffles per batch) leaves entry e + c's
// total in lane c, which writes gA[p].  Rows are binned by the row plan of A^T like the
// row-wise products: short rows one group each (in the plan's length order), medium rows one
// warp each, long rows one block each; partial sums of gX are combined in a fixed order, and
// every gA entry is a fixed-order sum: deterministic.
#include <limits.h>

#include "common.cuh"

namespace spx {
namespace {

constexpr int FB_THREADS = 256;
constexpr int FB_WARPS = FB_THREADS / 32;

struct FbEntry {
    int i;      // row of A (row of G gathered), -1 = no entry
    int p;      // position of the entry in A's order
    float v;    // A's value there
};

__device__ __forceinline__ FbEntry fb_load(const int32_t* __restrict__ t_ix, const int32_t* __restrict__ perm,
                                           const float* __restrict__ vals, int e, int b, uint64_t pol) {
    FbEntry r{-1, 0, 0.f};
    if (e < b) {
        r.i = ld_hint(t_ix + e, pol);
        r.p = ld_hint(perm + e, pol);
        r.v = __ldg(vals + r.p);
    }
    return r;
}

// One batch of LPR entries (lane c holds entry c of the batch in `cur`): acc += a_ij G_i on
// this lane's columns, and gA[p] = scale * <G_i, X_j> for the lane's own entry.
template <int LPR, bool TWO>
__device__ __forceinline__ void fb_batch(const FbEntry& cur, unsigned gmask, bool colok, const float4& xv,
                                         const float* __restrict__ G, int64_t ldg, int col, float4& acc, float scale,
                                         float* __restrict__ gA, uint64_t pol_keep) {
    float P[LPR];
    if constexpr (TWO) {
        // every row of the batch requested before A's values are needed (they come one
        // dependent load later than the row ids)
        float4 gq[LPR];
#pragma unroll
        for (int q = 0; q < LPR; ++q) {
            const int iq = __shfl_sync(gmask, cur.i, q, LPR);
            gq[q] = (iq >= 0 && colok) ? ld_hint4(G + (int64_t)iq * ldg + col, pol_keep)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < LPR; ++q) {
            const float vq = __shfl_sync(gmask, cur.v, q, LPR);
            const float4 g = gq[q];
            acc.x = fmaf(vq, g.x, acc.x);
            acc.y = fmaf(vq, g.y, acc.y);
            acc.z = fmaf(vq, g.z, acc.z);
            acc.w = fmaf(vq, g.w, acc.w);
            P[q] = fmaf(g.x, xv.x, fmaf(g.y, xv.y, fmaf(g.z, xv.z, g.w * xv.w)));
        }
    } else {
#pragma unroll
        for (int q = 0; q < LPR; ++q) {
            const int iq = __shfl_sync(gmask, cur.i, q, LPR);
            const float vq = __shfl_sync(gmask, cur.v, q, LPR);
            float d = 0.f;
            if (iq >= 0 && colok) {
                const float4 g = ld_hint4(G + (int64_t)iq * ldg + col, pol_keep);
                acc.x = fmaf(vq, g.x, acc.x);
                acc.y = fmaf(vq, g.y, acc.y);
                acc.z = fmaf(vq, g.z, acc.z);
                acc.w = fmaf(vq, g.w, acc.w);
                d = fmaf(g.x, xv.x, fmaf(g.y, xv.y, fmaf(g.z, xv.z, g.w * xv.w)));
            }
            P[q] = d;
        }
    }
    // butterfly transpose-reduction across the group: lane c ends with entry c's total
    const int c = threadIdx.x % LPR;
#pragma unroll
    for (int h = LPR / 2, cnt = LPR / 2; h >= 1; h >>= 1, cnt >>= 1) {
        const bool upper = (c & h) != 0;
#pragma unroll
        for (int q = 0; q < cnt; ++q) {
            const float send = upper ? P[q] : P[q + cnt];
            const float keep = upper ? P[q + cnt] : P[q];
            P[q] = keep + __shfl_xor_sync(gmask, send, h, LPR);
        }
    }
    if (cur.i >= 0) gA[cur.p] = scale * P[0];
}

__device__ __forceinline__ void fb_store(float* __restrict__ y, const float4& acc, float alpha, float beta) {
    float4 o;
    if (beta != 0.f) {
        const float4 old = *reinterpret_cast<const float4*>(y);
        o = make_float4(fmaf(alpha, acc.x, beta * old.x), fmaf(alpha, acc.y, beta * old.y),
                        fmaf(alpha, acc.z, beta * old.z), fmaf(alpha, acc.w, beta * old.w));
    } else {
        o = make_float4(alpha * acc.x, alpha * acc.y, alpha * acc.z, alpha * acc.w);
    }
    __stcs(reinterpret_cast<float4*>(y), o);
}

__device__ __forceinline__ float4 fb_xrow(const float* __restrict__ X, int64_t ldx, int64_t j, int col, bool colok) {
    return colok ? __ldcs(reinterpret_cast<const float4*>(X + j * ldx + col)) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// TWO: the batch's rows of G all requested before A's values are shuffled (more registers);
// MINB: resident blocks per SM the register allocation must allow; LEAN: short rows without
// the next batch held ahead.
template <int LPR, bool TWO, int MINB, bool LEAN = false>
__global__ void __launch_bounds__(FB_THREADS, MINB) spmm_t_sddmm_kernel(
    int32_t n, const int32_t* __restrict__ t_ptr, const int32_t* __restrict__ t_ix, const int32_t* __restrict__ perm,
    const float* __restrict__ vals, const float* __restrict__ G, int64_t ldg, const float* __restrict__ X,
    int64_t ldx, int32_t k, float* __restrict__ gX, int64_t ldgx, float alpha, float beta, float* __restrict__ gA,
    float scale, int32_t rows_per_group, int32_t threshold, const int32_t* __restrict__ long_rows, int32_t n_long,
    int32_t long_blocks, const int32_t* __restrict__ med_rows, int32_t n_med, int32_t med_blocks,
    const int32_t* __restrict__ short_rows, int32_t n_short) {
    constexpr int NG = 32 / LPR;                     // lane groups per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / LPR, c = lane % LPR;
    const unsigned gmask = LPR == 32 ? FULL : (((1u << LPR) - 1u) << (g * LPR));
    const int col = c * 4;
    const bool colok = col < k;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();

    if ((int)blockIdx.x < long_blocks) {
        // ---------------- long rows: all groups of the block on one row
        __shared__ float4 red[FB_WARPS][32];
        const int gid = warp * NG + g;
        constexpr int GB = FB_WARPS * NG;
        for (int q = blockIdx.x; q < n_long; q += long_blocks) {
            const int row = long_rows[q];
            const int a = t_ptr[row], b = t_ptr[row + 1];
            const float4 xv = fb_xrow(X, ldx, row, col, colok);
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int e = a + gid * LPR; e < b; e += GB * LPR) {
                const FbEntry cur = fb_load(t_ix, perm, vals, e + c, b, pol_stream);
                fb_batch<LPR, TWO>(cur, gmask, colok, xv, G, ldg, col, acc, scale, gA, pol_keep);
            }
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1) {
                acc.x += __shfl_xor_sync(FULL, acc.x, off);
                acc.y += __shfl_xor_sync(FULL, acc.y, off);
                acc.z += __shfl_xor_sync(FULL, acc.z, off);
                acc.w += __shfl_xor_sync(FULL, acc.w, off);
            }
            if (g == 0) red[warp][c] = acc;
            __syncthreads();
            if (warp == 0 && g == 0 && colok) {
                float4 tot = red[0][c];
                for (int w = 1; w < FB_WARPS; ++w) {
                    const float4 t = red[w][c];
                    tot.x += t.x;
                    tot.y += t.y;
                    tot.z += t.z;
                    tot.w += t.w;
                }
                fb_store(gX + (int64_t)row * ldgx + col, tot, alpha, beta);
            }
            __syncthreads();
        }
        return;
    }

    if ((int)blockIdx.x < long_blocks + med_blocks) {
        // ---------------- medium rows: one warp per row, its groups take batches round-robin
        const int nw = med_blocks * FB_WARPS;
        for (int q = ((int)blockIdx.x - long_blocks) * FB_WARPS + warp; q < n_med; q += nw) {
            const int row = med_rows[q];
            const int a = t_ptr[row], b = t_ptr[row + 1];
            const float4 xv = fb_xrow(X, ldx, row, col, colok);
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            const int e0 = a + g * LPR;
            FbEntry nxt = fb_load(t_ix, perm, vals, e0 + c, b, pol_stream);
            for (int e = e0; e < b; e += NG * LPR) {
                const FbEntry cur = nxt;
                nxt = fb_load(t_ix, perm, vals, e + NG * LPR + c, b, pol_stream);
                fb_batch<LPR, TWO>(cur, gmask, colok, xv, G, ldg, col, acc, scale, gA, pol_keep);
            }
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1) {
                acc.x += __shfl_xor_sync(FULL, acc.x, off);
                acc.y += __shfl_xor_sync(FULL, acc.y, off);
                acc.z += __shfl_xor_sync(FULL, acc.z, off);
                acc.w += __shfl_xor_sync(FULL, acc.w, off);
            }
            if (g == 0 && colok) fb_store(gX + (int64_t)row * ldgx + col, acc, alpha, beta);
        }
        return;
    }

    // ---------------- short rows: one lane group per row (in the plan's length order if given)
    const int64_t wglobal = ((int64_t)(blockIdx.x - long_blocks - med_blocks) * FB_THREADS + threadIdx.x) >> 5;
    const int64_t row0 = (wglobal * NG + g) * rows_per_group;
    const int64_t n_rows = short_rows ? (int64_t)n_short : (int64_t)n;
    for (int p = 0; p < rows_per_group; ++p) {
        const int64_t idx = row0 + p;
        if (idx >= n_rows) break;
        const int64_t row = short_rows ? (int64_t)short_rows[idx] : idx;
        const int a = t_ptr[row], b = t_ptr[row + 1];
        if (b - a > threshold) continue;            // a long-row block or a medium-row warp takes it
        const float4 xv = fb_xrow(X, ldx, row, col, colok);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (LEAN) {
            // no batch held ahead: fewer live registers, more resident warps
            for (int e = a; e < b; e += LPR)
                fb_batch<LPR, TWO>(fb_load(t_ix, perm, vals, e + c, b, pol_stream), gmask, colok, xv, G, ldg, col,
                                   acc, scale, gA, pol_keep);
        } else {
            FbEntry nxt = fb_load(t_ix, perm, vals, a + c, b, pol_stream);
            for (int e = a; e < b; e += LPR) {
                const FbEntry cur = nxt;
                if (e + LPR < b) nxt = fb_load(t_ix, perm, vals, e + LPR + c, b, pol_stream);
                fb_batch<LPR, TWO>(cur, gmask, colok, xv, G, ldg, col, acc, scale, gA, pol_keep);
            }
        }
        if (colok) fb_store(gX + row * ldgx + col, acc, alpha, beta);
    }
}

template <int LPR, bool TWO, int MINB, bool LEAN = false>
void fb_launch(unsigned grid, cudaStream_t st, const spx_csr* AT, const int32_t* perm, const float* vals,
               const float* G, int64_t ldg, const float* X, int64_t ldx, int32_t k, float* gX, int64_t ldgx,
               float alpha, float beta, float* gA, float scale, int32_t rpg, int32_t threshold,
               const int32_t* long_rows, int32_t n_long, int32_t long_blocks, const int32_t* med_rows, int32_t n_med,
               int32_t med_blocks, const int32_t* short_rows, int32_t n_short) {
    spmm_t_sddmm_kernel<LPR, TWO, MINB, LEAN><<<grid, FB_THREADS, 0, st>>>(AT->m, AT->indptr, AT->indices, perm, vals, G, ldg, X, ldx,
                                                                    k, gX, ldgx, alpha, beta, gA, scale, rpg,
                                                                    threshold, long_rows, n_long, long_blocks,
                                                                    med_rows, n_med, med_blocks, short_rows, n_short);
}

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_spmm_t_sddmm(const spx_csr* AT, const int32_t* perm, const float* a_values, const float* G,
                                       int64_t ldg, const float* X, int64_t ldx, int32_t k, float* gX, int64_t ldgx,
                                       float alpha, float beta, float* gA, float scale, const spx_rowplan* plan,
                                       int32_t variant, void* stream) {
    const char* who = "spx_spmm_t_sddmm";
    if (variant < 0 || variant > 5) return set_error(SPX_INVALID_ARG, "%s: variant %d (0..5)", who, variant);
    SPX_TRY(check_csr(AT, false, who));
    if (k < 4 || k > 128 || k % 4 != 0)
        return set_error(SPX_NOT_SUPPORTED, "%s: k = %d (a multiple of 4 in 4..128)", who, k);
    if (AT->nnz > 0 && (!perm || !a_values || !gA)) return set_error(SPX_INVALID_ARG, "%s: NULL operand", who);
    if (AT->m > 0 && (!X || !gX)) return set_error(SPX_INVALID_ARG, "%s: NULL operand", who);
    if (AT->n > 0 && !G) return set_error(SPX_INVALID_ARG, "%s: NULL operand", who);
    if (ldg < k || ldx < k || ldgx < k || ldg % 4 || ldx % 4 || ldgx % 4 || (G && !al16(G)) || (X && !al16(X)) ||
        (gX && !al16(gX)))
        return set_error(SPX_INVALID_ARG, "%s: dense operands need 16-byte aligned rows, ld >= k, ld %% 4 == 0", who);
    if (AT->m == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
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
        threshold = plan->medium_threshold;
        const int64_t want = ((int64_t)n_med + 2 * FB_WARPS - 1) / (2 * FB_WARPS);
        med_blocks = (int32_t)(want < 8 * num_sms() ? want : 8 * num_sms());
    }
    const int32_t* short_rows = plan && plan->short_rows ? plan->short_rows : nullptr;
    const int32_t n_short = short_rows ? plan->n_short : 0;
    if (short_rows && (n_short < 0 || n_short > AT->m)) return set_error(SPX_INVALID_ARG, "%s: bad short-row order", who);
    int lpr = 8;
    while (lpr * 4 < k) lpr <<= 1;
    const int32_t rpg = plan && plan->rows_per_group > 0 ? plan->rows_per_group : 2;
    const int64_t rows_per_block = (int64_t)FB_WARPS * (32 / lpr) * rpg;
    const int64_t n_rows = short_rows ? (int64_t)n_short : (int64_t)AT->m;
    const int64_t grid = (n_rows + rows_per_block - 1) / rows_per_block + long_blocks + med_blocks;
    if (grid > INT_MAX) return set_error(SPX_INVALID_ARG, "%s: too many rows", who);
    if (grid == 0) return SPX_OK;
#define SPX_FB_ARGS                                                                                                \
    (unsigned)grid, st, AT, perm, a_values, G, ldg, X, ldx, k, gX, ldgx, alpha, beta, gA, scale, rpg, threshold, \
        long_rows, n_long, long_blocks, med_rows, n_med, med_blocks, short_rows, n_short
    // 8-lane groups: variant 0 loads, shuffles and uses one row at a time (4 resident blocks),
    // 1 requests the batch's rows first (3 resident blocks), 2 and 3 as 0 with 5 and 6 resident
    // blocks (fewer registers), 4 and 5 without a batch held ahead at 6 and 8; 16-lane groups:
    // 3 or 4 resident blocks (2..5: as 1); 32-lane groups: one shape
    if (lpr == 8) {
        if (variant == 0) fb_launch<8, false, 4>(SPX_FB_ARGS);
        else if (variant == 1) fb_launch<8, true, 3>(SPX_FB_ARGS);
        else if (variant == 2) fb_launch<8, false, 5>(SPX_FB_ARGS);
        else if (variant == 3) fb_launch<8, false, 6>(SPX_FB_ARGS);
        else if (variant == 4) fb_launch<8, false, 6, true>(SPX_FB_ARGS);
        else fb_launch<8, false, 8, true>(SPX_FB_ARGS);
    } else if (lpr == 16) {
        if (variant == 0) fb_launch<16, false, 3>(SPX_FB_ARGS);
        else fb_launch<16, false, 4>(SPX_FB_ARGS);          // variants 1..5
    } else {
        fb_launch<32, false, 3>(SPX_FB_ARGS);
    }
#undef SPX_FB_ARGS
    SPX_CHECK_LAUNCH(who);
    return SPX_OK;
}
