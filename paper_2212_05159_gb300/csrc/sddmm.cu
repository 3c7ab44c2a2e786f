// Masked dense-dense product on a CSR pattern (SDDMM):
//   out[e] = scale * sum_c G[i,c] X[j,c]  for every stored e = (i, j)
// -- the gradient w.r.t. the sparse matrix of SpMV / SpDMM (Table 1, rows "A": V x^T or
// V B^T masked to mask(A)) and, with k = 1 and scale = -1, the SpSolve gradient.
//
// Mapping (HBM-bound; every entry gathers one row of X):
//   * each warp owns a contiguous chunk of entries, so long and short rows cost the
//     same (no row-length imbalance); the row of each entry is found by a binary
//     search for the chunk start and a forward walk of indptr;
//   * LPN lanes cover the k columns of one entry with float4 loads; 32 / LPN entries are
//     loaded per instruction, LPN instructions cover a batch of 32 entries;
//   * the LPN partial dot products per lane are summed with a butterfly transpose
//     (LPN - 1 shuffles per lane per 32 entries instead of log2(LPN) per entry), which
//     leaves the total of entry s * 32/LPN + g in lane (g, s).
// Deterministic: every output is a fixed-order sum.
#include <limits.h>

#include "common.cuh"
#include "slab.cuh"

namespace spx {
namespace {

constexpr int SDDMM_THREADS = 256;
constexpr int SDDMM_BATCHES = 8;               // 32-entry batches per warp chunk

__device__ __forceinline__ int row_of(const int32_t* __restrict__ indptr, int32_t m, int64_t e) {
    // largest r with indptr[r] <= e (indptr[m] = nnz > e)
    int lo = 0, hi = m;                            // answer in [lo, hi)
    while (hi - lo > 1) {
        int mid = lo + ((hi - lo) >> 1);
        if ((int64_t)indptr[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int VEC>
__device__ __forceinline__ float dot_slice(const float* __restrict__ g, const float* __restrict__ x, uint64_t pol) {
    if constexpr (VEC == 4) {
        float4 a = __ldg(reinterpret_cast<const float4*>(g));
        float4 b = ld_hint4(x, pol);
        return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
    } else {
        return __ldg(g) * ld_hint(x, pol);
    }
}

template <int VEC, int LPN>
__global__ void __launch_bounds__(SDDMM_THREADS) sddmm_kernel(
    int32_t m, int64_t nnz, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
    const float* __restrict__ G, int64_t ldg, const float* __restrict__ X, int64_t ldx, int32_t x_shift,
    int32_t col_begin, int32_t col_end, float scale, bool accumulate, float* __restrict__ out) {
    constexpr int NPI = 32 / LPN;                  // entries per load instruction
    constexpr int CHUNK = 32 * SDDMM_BATCHES;
    const int lane = threadIdx.x & 31;
    const int s = lane % LPN;                      // column slice
    const int gq = lane / LPN;                     // entry slot inside an instruction
    const int64_t warp = (blockIdx.x * (int64_t)SDDMM_THREADS + threadIdx.x) >> 5;
    const int64_t e_begin = warp * CHUNK;
    if (e_begin >= nnz) return;
    const int64_t e_end = e_begin + CHUNK < nnz ? e_begin + CHUNK : nnz;
    int row = row_of(indptr, m, e_begin);
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    for (int64_t base = e_begin; base < e_end; base += 32) {
        const int64_t e = base + lane;
        const bool valid = e < e_end;
        int r = row, j = 0;
        if (valid) {
            while ((int64_t)indptr[r + 1] <= e) ++r;
            j = ld_hint(indices + e, pol_stream);
        }
        float P[LPN];
#pragma unroll
        for (int u = 0; u < LPN; ++u) {
            const int t = u * NPI + gq;
            const int it = __shfl_sync(FULL, r, t);
            const int jt = __shfl_sync(FULL, j, t);
            float acc = 0.f;
            if (base + t < e_end) {
                for (int col = col_begin + s * VEC; col < col_end; col += LPN * VEC)
                    acc += dot_slice<VEC>(G + (int64_t)it * ldg + col, X + (int64_t)jt * ldx + (col - x_shift),
                                          pol_keep);
            }
            P[u] = acc;
        }
        // butterfly transpose-reduction across the LPN lanes of an entry slot
#pragma unroll
        for (int h = LPN / 2, cnt = LPN / 2; h >= 1; h >>= 1, cnt >>= 1) {
            const bool upper = (s & h) != 0;
#pragma unroll
            for (int q = 0; q < cnt; ++q) {
                float send = upper ? P[q] : P[q + cnt];
                float keep = upper ? P[q + cnt] : P[q];
                P[q] = keep + __shfl_xor_sync(FULL, send, h);
            }
        }
        const int t_out = s * NPI + gq;
        if (base + t_out < e_end) {
            float* o = out + base + t_out;
            __stcs(o, accumulate ? fmaf(scale, P[0], *o) : scale * P[0]);
        }
        row = __shfl_sync(FULL, r, 31);
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// ---------------------------------------------------------------------------------------
// Row-plan SDDMM (float4 columns).  A lane group of LPR lanes spans the columns of a block;
// it holds G's row i in registers for the whole row and takes the row's entries LPR at a
// time: lane c computes the LPR partial dot products of its column slice with the batch's
// X rows, and a butterfly transpose across the group leaves entry c's total in lane c,
// which stores it (coalesced).  Rows are binned like the row-wise products: short rows
// one group each, medium rows one warp each (groups take batches round-robin), long rows
// one block each.  Outputs are independent, so no cross-group reduction is needed.  With
// a plan split into column parts, one pass per part takes the entries of each row whose
// columns lie in that part, so the rows of X gathered in a pass stay resident in L2 (G's
// row is then read once per part that the row has entries in).
constexpr int SR_THREADS = 256;
constexpr int SR_WARPS = SR_THREADS / 32;
// Resident blocks per SM forced by register capping (latency-bound gathers want warps in
// flight); measured on GB300: 6 best with 8-lane groups (k = 32), 8 with 32-lane groups.
constexpr int sr_min_blocks(int lpr) { return lpr >= 32 ? 8 : 6; }

template <int LPR>
__device__ __forceinline__ void sddmm_batch(const int32_t* __restrict__ indices, int e, int b, int c, unsigned gmask,
                                            const float4& gv, bool colok, const float* __restrict__ X, int64_t ldx,
                                            int xcol, float scale, bool accumulate, float* __restrict__ out,
                                            uint64_t pol_stream, uint64_t pol_keep) {
    const int ee = e + c;
    const int jmine = ee < b ? ld_hint(indices + ee, pol_stream) : -1;
    float P[LPR];
#pragma unroll
    for (int q = 0; q < LPR; ++q) {
        const int jq = __shfl_sync(gmask, jmine, q, LPR);
        float acc = 0.f;
        if (jq >= 0 && colok) {
            const float4 x = ld_hint4(X + (int64_t)jq * ldx + xcol, pol_keep);
            acc = fmaf(gv.x, x.x, fmaf(gv.y, x.y, fmaf(gv.z, x.z, gv.w * x.w)));
        }
        P[q] = acc;
    }
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
    if (ee < b) {
        float* o = out + ee;
        __stcs(o, accumulate ? fmaf(scale, P[0], *o) : scale * P[0]);
    }
}

template <int LPR>
__global__ void __launch_bounds__(SR_THREADS, sr_min_blocks(LPR)) sddmm_rows_kernel(
    int32_t m, const int32_t* __restrict__ indptr, const int32_t* __restrict__ seg_b, const int32_t* __restrict__ seg_e,
    const int32_t* __restrict__ indices, const float* __restrict__ G,
    int64_t ldg, const float* __restrict__ X, int64_t ldx, int32_t x_shift, int32_t col_begin, int32_t col_end,
    float scale, bool accumulate, float* __restrict__ out, int32_t rows_per_group, int32_t threshold,
    const int32_t* __restrict__ long_rows, int32_t n_long, int32_t long_blocks, const int32_t* __restrict__ med_rows,
    int32_t n_med, int32_t med_blocks, const int32_t* __restrict__ short_rows, int32_t n_short) {
    constexpr int G_ = 32 / LPR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / LPR, c = lane % LPR;
    const unsigned gmask = LPR == 32 ? FULL : (((1u << LPR) - 1u) << (g * LPR));
    const int col = col_begin + c * 4;
    const int xcol = col - x_shift;
    const bool colok = col < col_end;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const bool split = seg_b != indptr || seg_e != indptr + 1;
    auto grow = [&](int row) {
        return colok ? __ldg(reinterpret_cast<const float4*>(G + (int64_t)row * ldg + col)) : make_float4(0, 0, 0, 0);
    };
    if ((int)blockIdx.x < long_blocks) {
        const int gid = warp * G_ + g;
        constexpr int GB = SR_WARPS * G_;
        for (int q = blockIdx.x; q < n_long; q += long_blocks) {
            const int row = long_rows[q];
            const int a = seg_b[row], b = seg_e[row];
            if (a == b) continue;
            const float4 gv = grow(row);
            for (int e = a + gid * LPR; e < b; e += GB * LPR)
                sddmm_batch<LPR>(indices, e, b, c, gmask, gv, colok, X, ldx, xcol, scale, accumulate, out, pol_stream,
                                 pol_keep);
        }
        return;
    }
    if ((int)blockIdx.x < long_blocks + med_blocks) {
        const int nw = med_blocks * SR_WARPS;
        for (int q = ((int)blockIdx.x - long_blocks) * SR_WARPS + warp; q < n_med; q += nw) {
            const int row = med_rows[q];
            const int a = seg_b[row], b = seg_e[row];
            if (a == b) continue;
            const float4 gv = grow(row);
            for (int e = a + g * LPR; e < b; e += G_ * LPR)
                sddmm_batch<LPR>(indices, e, b, c, gmask, gv, colok, X, ldx, xcol, scale, accumulate, out, pol_stream,
                                 pol_keep);
        }
        return;
    }
    const int64_t wglobal = ((int64_t)(blockIdx.x - long_blocks - med_blocks) * SR_THREADS + threadIdx.x) >> 5;
    const int64_t row0 = (wglobal * G_ + g) * rows_per_group;
    const int64_t n_rows = short_rows ? (int64_t)n_short : (int64_t)m;      // the plan's length order, if any
    for (int p = 0; p < rows_per_group; ++p) {
        const int64_t idx = row0 + p;
        if (idx >= n_rows) break;
        const int64_t row = short_rows ? (int64_t)short_rows[idx] : idx;
        int a = indptr[row], b = indptr[row + 1];
        if (b - a > threshold) continue;
        if (split) {
            a = seg_b[row];
            b = seg_e[row];
        }
        if (a == b) continue;
        const float4 gv = grow((int)row);
        for (int e = a; e < b; e += LPR)
            sddmm_batch<LPR>(indices, e, b, c, gmask, gv, colok, X, ldx, xcol, scale, accumulate, out, pol_stream,
                             pol_keep);
    }
}



template <int VEC>
spx_status launch_lpn(int lpn, dim3 grid, cudaStream_t st, int32_t m, int64_t nnz, const int32_t* ip,
                      const int32_t* ix, const float* G, int64_t ldg, const float* X, int64_t ldx, int32_t xs,
                      int32_t c0, int32_t c1, float scale, bool acc, float* out) {
#define SPX_SDDMM_CASE(L)                                                                                     \
    case L:                                                                                                   \
        sddmm_kernel<VEC, L><<<grid, SDDMM_THREADS, 0, st>>>(m, nnz, ip, ix, G, ldg, X, ldx, xs, c0, c1, scale, \
                                                             acc, out);                                       \
        break;
    switch (lpn) {
        SPX_SDDMM_CASE(1)
        SPX_SDDMM_CASE(2)
        SPX_SDDMM_CASE(4)
        SPX_SDDMM_CASE(8)
        SPX_SDDMM_CASE(16)
        SPX_SDDMM_CASE(32)
        default: return set_error(SPX_INVALID_ARG, "sddmm: bad lane count");
    }
#undef SPX_SDDMM_CASE
    SPX_CHECK_LAUNCH("sddmm");
    return SPX_OK;
}

int32_t sddmm_cb(const spx_csr* A, int32_t k, int32_t col_block, bool vec4) {
    int32_t cb = col_block > 0 ? col_block : k;       // default: one pass over all columns
    if (cb > k) cb = k;
    if (vec4 && cb % 4 != 0) cb = (cb + 3) / 4 * 4;
    return cb;
}

spx_status launch_sddmm_rows(const spx_csr* A, const float* G, int64_t ldg, const float* X, int64_t ldx,
                             int32_t k, float scale, float* out, int32_t cb, const spx_rowplan* plan, float* ws,
                             bool use_slab, cudaStream_t st) {
    int lpr = 1;
    while (lpr * 4 < cb && lpr < 32) lpr <<= 1;
    int32_t threshold = INT_MAX, n_long = 0, long_blocks = 0, n_med = 0, med_blocks = 0;
    const int32_t* long_rows = nullptr;
    const int32_t* med_rows = nullptr;
    if (plan->n_long > 0) {
        threshold = plan->threshold;
        long_rows = plan->long_rows;
        n_long = plan->n_long;
        long_blocks = n_long < 4 * num_sms() ? n_long : 4 * num_sms();
    }
    if (plan->n_medium > 0) {
        med_rows = plan->medium_rows;
        n_med = plan->n_medium;
        threshold = plan->medium_threshold;
        const int64_t want = ((int64_t)n_med + 2 * SR_WARPS - 1) / (2 * SR_WARPS);
        med_blocks = (int32_t)(want < 8 * num_sms() ? want : 8 * num_sms());
    }
    // the plan's short-row order groups rows by 8-entry batches; with 32-entry batches (k = 128)
    // every short row is one batch and the order only adds a load (measured 4-5 % slower)
    const int32_t* short_rows = lpr < 32 ? plan->short_rows : nullptr;
    const int32_t n_short = short_rows ? plan->n_short : 0;
    if (short_rows && (n_short < 0 || n_short > A->m)) return set_error(SPX_INVALID_ARG, "sddmm: bad short-row order");
    const int64_t n_rows = short_rows ? (int64_t)n_short : (int64_t)A->m;
    const int rpg = plan->rows_per_group > 0 ? plan->rows_per_group : 2;
    const int64_t rows_per_block = (int64_t)SR_WARPS * (32 / lpr) * rpg;
    const int64_t grid = (n_rows + rows_per_block - 1) / rows_per_block + long_blocks + med_blocks;
    if (grid > INT_MAX) return set_error(SPX_INVALID_ARG, "sddmm: too many rows");
    if (use_slab) SPX_TRY(slab_repack(A->n, X, ldx, k, cb, ws, st));
    const int32_t parts = plan->n_parts > 1 && plan->part_ptr ? plan->n_parts : 1;
    for (int32_t c0 = 0; c0 < k; c0 += cb) {
        const int32_t c1 = c0 + cb < k ? c0 + cb : k;
        const float* Xp = use_slab ? ws + (int64_t)(c0 / cb) * A->n * cb : X;
        const int64_t ldp = use_slab ? cb : ldx;
        const int32_t xs = use_slab ? c0 : 0;
        for (int32_t p = 0; p < parts; ++p) {
            // pass p: the entries of each row whose columns lie in range p (disjoint outputs)
            const int32_t* sb = p == 0 ? A->indptr : plan->part_ptr + (int64_t)(p - 1) * A->m;
            const int32_t* se = p == parts - 1 ? A->indptr + 1 : plan->part_ptr + (int64_t)p * A->m;
#define SPX_SR_CASE(L)                                                                                           \
    case L:                                                                                                      \
        sddmm_rows_kernel<L><<<(unsigned)grid, SR_THREADS, 0, st>>>(A->m, A->indptr, sb, se, A->indices, G, ldg, Xp, \
                                                                     ldp, xs, c0, c1, scale, c0 > 0, out, rpg,       \
                                                                     threshold, long_rows, n_long, long_blocks,      \
                                                                     med_rows, n_med, med_blocks, short_rows,        \
                                                                     n_short);                                       \
        break;
            switch (lpr) {
                SPX_SR_CASE(2)
                SPX_SR_CASE(4)
                SPX_SR_CASE(8)
                SPX_SR_CASE(16)
                SPX_SR_CASE(32)
                default: return set_error(SPX_INVALID_ARG, "sddmm: bad lane count %d", lpr);
            }
#undef SPX_SR_CASE
            SPX_CHECK_LAUNCH("sddmm rows");
        }
    }
    return SPX_OK;
}

spx_status launch_sddmm(const spx_csr* A, const float* G, int64_t ldg, const float* X, int64_t ldx, int32_t k,
                        float scale, float* out, int32_t col_block, float* ws, size_t ws_bytes, cudaStream_t st,
                        const spx_rowplan* plan = nullptr) {
    if (A->nnz == 0) return SPX_OK;
    const bool vec4 = (k % 4 == 0) && (ldg % 4 == 0) && (ldx % 4 == 0) && aligned16(G) && aligned16(X);
    const int VEC = vec4 ? 4 : 1;
    const int32_t cb = sddmm_cb(A, k, col_block, vec4);
    const size_t slab = vec4 ? slab_bytes(A->n, k, cb) : 0;
    const bool use_slab = slab > 0 && ws != nullptr && ws_bytes >= slab;
    if (plan && vec4 && cb >= 8 && cb <= 128)
        return launch_sddmm_rows(A, G, ldg, X, ldx, k, scale, out, cb, plan, ws, use_slab, st);
    int64_t lanes = (cb + VEC - 1) / VEC;
    int lpn = 1;
    while (lpn < lanes && lpn < 32) lpn <<= 1;
    const int64_t chunk = 32 * SDDMM_BATCHES;
    const int64_t warps = (A->nnz + chunk - 1) / chunk;
    const int64_t blocks = (warps * 32 + SDDMM_THREADS - 1) / SDDMM_THREADS;
    if (blocks > INT_MAX) return set_error(SPX_INVALID_ARG, "sddmm: too many entries");
    dim3 grid((unsigned)blocks);
    if (use_slab) SPX_TRY(slab_repack(A->n, X, ldx, k, cb, ws, st));
    for (int32_t c0 = 0; c0 < k; c0 += cb) {
        const int32_t c1 = c0 + cb < k ? c0 + cb : k;
        const float* Xp = use_slab ? ws + (int64_t)(c0 / cb) * A->n * cb : X;
        const int64_t ldp = use_slab ? cb : ldx;
        const int32_t xs = use_slab ? c0 : 0;
        spx_status s = vec4 ? launch_lpn<4>(lpn, grid, st, A->m, A->nnz, A->indptr, A->indices, G, ldg, Xp, ldp, xs,
                                            c0, c1, scale, c0 > 0, out)
                            : launch_lpn<1>(lpn, grid, st, A->m, A->nnz, A->indptr, A->indices, G, ldg, Xp, ldp, xs,
                                            c0, c1, scale, c0 > 0, out);
        if (s != SPX_OK) return s;
    }
    return SPX_OK;
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_sddmm_workspace_size(const spx_csr* A, int32_t k, int32_t col_block, size_t* bytes) {
    SPX_TRY(check_csr(A, false, "spx_sddmm_workspace_size"));
    if (!bytes || k < 0) return set_error(SPX_INVALID_ARG, "spx_sddmm_workspace_size: bad arguments");
    *bytes = k > 0 && k % 4 == 0 ? slab_bytes(A->n, k, sddmm_cb(A, k, col_block, true)) : 0;
    return SPX_OK;
}

extern "C" spx_status spx_sddmm(const spx_csr* A, const float* G, int64_t ldg, const float* X, int64_t ldx,
                                int32_t k, float scale, float* out, int32_t col_block, const spx_rowplan* plan,
                                void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, false, "spx_sddmm"));
    if (k < 1 || ldg < k || ldx < k) return set_error(SPX_INVALID_ARG, "spx_sddmm: bad k / leading dims");
    if (A->nnz > 0 && (!G || !X || !out)) return set_error(SPX_INVALID_ARG, "spx_sddmm: NULL operand");
    if (ws) {
        const bool vec4 = (k % 4 == 0) && (ldg % 4 == 0) && (ldx % 4 == 0) && aligned16(G) && aligned16(X);
        const size_t need = vec4 ? slab_bytes(A->n, k, sddmm_cb(A, k, col_block, true)) : 0;
        if (ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_sddmm: workspace %zu < %zu", ws_bytes, need);
    }
    if (plan && ((plan->n_long > 0 && !plan->long_rows) || (plan->n_medium > 0 && !plan->medium_rows)))
        return set_error(SPX_INVALID_ARG, "spx_sddmm: plan without rows");
    return launch_sddmm(A, G, ldg, X, ldx, k, scale, out, col_block, static_cast<float*>(ws), ws_bytes,
                        as_stream(stream), plan);
}

extern "C" spx_status spx_masked_outer(const spx_csr* A, const float* u, const float* v, float scale, float* out,
                                       void* stream) {
    SPX_TRY(check_csr(A, false, "spx_masked_outer"));
    if (A->nnz > 0 && (!u || !v || !out)) return set_error(SPX_INVALID_ARG, "spx_masked_outer: NULL operand");
    return launch_sddmm(A, u, 1, v, 1, 1, scale, out, 1, nullptr, 0, as_stream(stream));
}
