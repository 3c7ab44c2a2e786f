// Merge-path load balancing for the row-wise products (Section 3.1.1 SpMV, 3.1.3 SpDMM and
// the SDDMM of Table 1's SpDMM gradient w.r.t. A):
//
//   spx_spmm_merge   Y  = alpha * A X + beta * Y
//   spx_sddmm_merge  out[e] = scale * G[i, :] . X[j, :]   for every stored e = (i, j)
//
// The m row ends (indptr[1..m]) and the nnz entries are merged into one sequence -- entry e
// of row i comes before the end of row i -- and cut into segments of `items` consecutive
// items.  Each lane group (LPR = k / 4 lanes, one float4 column slice each) takes one
// segment, so every group has the same amount of work however the row lengths are
// distributed (power-law rows of 5 to 4096 entries, empty rows, hub rows).  The segment
// starts are found once per pattern by a binary search along each cut (the plan).
//
// Inside a segment the group walks the entries in order in full batches of B: the B column
// indices and values are loaded first (lane c holds entries c*SLOTS ..), then all B row
// gathers of X are issued back to back, then they are consumed in entry order; when an
// entry lies past the current row's end, that row is finished and written.  The next row's
// end (and, for SDDMM, the next row of G) is prefetched while the current row is summed.
//
// SpMM: a row cut by a segment boundary leaves a partial sum.  The segment that finishes
// the row writes alpha * (its part) + beta * Y; every earlier segment holding part of the
// row writes its partial sum to a carry slot, and a second kernel adds the carries of each
// row in segment order.  SDDMM outputs are per entry, so it needs no carries.  Every output
// is a fixed-order sum: results are deterministic (a different order from the row-plan
// kernels, within the same tolerance).
#include <limits.h>

#include "common.cuh"

namespace spx {
namespace {

constexpr int MG_THREADS = 256;

// Number of row ends among the first d merged items (the row the merge path is in after
// d items): the largest i in [max(0, d - nnz), min(d, m)] with indptr[i] + i <= d, found
// as the first i whose row end indptr[i + 1] lies past the entries consumed by then.
__device__ __forceinline__ int32_t merge_search(int32_t m, int64_t nnz, const int32_t* __restrict__ indptr,
                                                int64_t d) {
    int64_t lo = d - nnz > 0 ? d - nnz : 0;
    int64_t hi = d < (int64_t)m ? d : (int64_t)m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)indptr[mid + 1] <= d - mid - 1)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (int32_t)lo;
}

__global__ void merge_partition_kernel(int32_t m, int64_t nnz, const int32_t* __restrict__ indptr, int64_t items,
                                       int32_t nseg, int32_t* __restrict__ seg_row) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nseg) return;
    const int64_t tot = (int64_t)m + nnz;
    const int64_t d = s * items < tot ? s * items : tot;
    seg_row[s] = merge_search(m, nnz, indptr, d);
}

__device__ __forceinline__ float4 f4_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

__device__ __forceinline__ void f4_fma(float4& acc, float v, const float4& x) {
    acc.x = fmaf(v, x.x, acc.x);
    acc.y = fmaf(v, x.y, acc.y);
    acc.z = fmaf(v, x.z, acc.z);
    acc.w = fmaf(v, x.w, acc.w);
}

template <int LPR, int B, int MINB, bool PERM>
__global__ void __launch_bounds__(MG_THREADS, MINB) spmm_merge_kernel(
    int32_t m, int32_t nnz, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
    const float* __restrict__ vals, const int32_t* __restrict__ perm, const float* __restrict__ X, int64_t ldx,
    float* __restrict__ Y, int64_t ldy, float alpha, float beta, int32_t items, int32_t nseg,
    const int32_t* __restrict__ seg_row, int32_t* __restrict__ carry_row, float* __restrict__ carry_val) {
    constexpr int SLOTS = (B + LPR - 1) / LPR;   // entries of a batch loaded per lane
    constexpr int K = 4 * LPR;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR;
    const int c = lane % LPR;
    const unsigned gmask = LPR == 32 ? FULL : (((1u << LPR) - 1u) << (g * LPR));
    const int sg = (int)(((int64_t)blockIdx.x * MG_THREADS + threadIdx.x) / LPR);
    if (sg >= nseg) return;                      // the whole group: no shuffle partner left behind
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const int tot = m + nnz;                     // < 2^31 (checked by the host)
    const int d0 = sg * items;
    const int d1 = items < tot - d0 ? d0 + items : tot;
    int row = seg_row[sg];
    const int row_last = seg_row[sg + 1];
    int e = d0 - row;
    const int e_end = d1 - row_last;
    const float* xc = X + 4 * c;
    float4 acc = f4_zero();
    bool has = false;
    int row_end = row < m ? indptr[row + 1] : INT_MAX;
    int next_end = row + 1 < m ? indptr[row + 2] : INT_MAX;
    // the current row ends inside this segment: write it and move to the next row
    auto finish_row = [&]() {
        float4* y = reinterpret_cast<float4*>(Y + (int64_t)row * ldy + 4 * c);
        float4 o;
        if (beta != 0.f) {
            const float4 old = *y;
            o = make_float4(fmaf(alpha, acc.x, beta * old.x), fmaf(alpha, acc.y, beta * old.y),
                            fmaf(alpha, acc.z, beta * old.z), fmaf(alpha, acc.w, beta * old.w));
        } else {
            o = make_float4(alpha * acc.x, alpha * acc.y, alpha * acc.z, alpha * acc.w);
        }
        __stcs(y, o);
        acc = f4_zero();
        has = false;
        ++row;
        row_end = next_end;
        next_end = row + 1 < m ? indptr[row + 2] : INT_MAX;
    };
    // batch loads: lane c holds entries c*SLOTS .. of the batch starting at e0 (column -1: none)
    auto load_batch = [&](int e0, int (&jl)[SLOTS], float (&vl)[SLOTS]) {
        const int nb = e_end - e0 < B ? e_end - e0 : B;
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            const int q = c * SLOTS + s;
            if (q < nb) {
                jl[s] = ld_hint(indices + e0 + q, pol_stream);
                vl[s] = PERM ? __ldg(vals + ld_hint(perm + e0 + q, pol_stream)) : ld_hint(vals + e0 + q, pol_stream);
            } else {
                jl[s] = 0;
                vl[s] = 0.f;
            }
        }
    };
    int jn[SLOTS];
    float vn[SLOTS];
    if (e < e_end) load_batch(e, jn, vn);
    while (e < e_end) {
        const int nb = e_end - e < B ? e_end - e : B;
        int jl[SLOTS];
        float vl[SLOTS];
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            jl[s] = jn[s];
            vl[s] = vn[s];
        }
        float4 xv[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const int jq = __shfl_sync(gmask, jl[q % SLOTS], q / SLOTS, LPR);
            xv[q] = q < nb ? ld_hint4(xc + (int64_t)jq * ldx, pol_keep) : f4_zero();
        }
        // the next batch's indices and values travel while this batch's rows are gathered
        if (e + nb < e_end) load_batch(e + nb, jn, vn);
        // the batch as runs of entries of one row: [q, cut) belongs to the current row
        int q = 0;
        for (;;) {
            const int left = row_end - e;
            const int cut = left < nb ? left : nb;
#pragma unroll
            for (int u = 0; u < B; ++u) {
                if (u >= q && u < cut) {         // uniform across the group
                    const float v = __shfl_sync(gmask, vl[u % SLOTS], u / SLOTS, LPR);
                    f4_fma(acc, v, xv[u]);
                }
            }
            if (cut > q) has = true;
            if (cut == nb) break;
            finish_row();                        // the row ends before entry cut (an empty row: cut == q)
            q = cut;
        }
        e += nb;
    }
    while (row < row_last) finish_row();         // rows ending here after the last entry (and empty rows)
    // what is left belongs to row_last, which a later segment finishes
    if (has) *reinterpret_cast<float4*>(carry_val + (int64_t)sg * K + 4 * c) = acc;
    if (c == 0) carry_row[sg] = has ? row : -1;
}

// Adds the carries of every row, in segment order, to the value its finishing segment wrote.
// Thread (s, c) works only when segment s holds the first carry of its row.
__global__ void merge_fixup_kernel(int32_t nseg, int32_t k4, const int32_t* __restrict__ carry_row,
                                   const float* __restrict__ carry_val, float* __restrict__ Y, int64_t ldy,
                                   float alpha) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = t / k4;
    const int c = (int)(t % k4);
    if (s >= nseg) return;
    const int32_t r = carry_row[s];
    if (r < 0 || (s > 0 && carry_row[s - 1] == r)) return;
    const float4* cv = reinterpret_cast<const float4*>(carry_val);
    float4 sum = cv[s * k4 + c];
    for (int64_t u = s + 1; u < nseg && carry_row[u] == r; ++u) {
        const float4 v = cv[u * k4 + c];
        sum.x += v.x;
        sum.y += v.y;
        sum.z += v.z;
        sum.w += v.w;
    }
    float4* y = reinterpret_cast<float4*>(Y + (int64_t)r * ldy) + c;
    float4 o = *y;
    o.x = fmaf(alpha, sum.x, o.x);
    o.y = fmaf(alpha, sum.y, o.y);
    o.z = fmaf(alpha, sum.z, o.z);
    o.w = fmaf(alpha, sum.w, o.w);
    *y = o;
}

// SDDMM over the same segments.  Batches of LPR entries: lane c loads entry c's column,
// the group gathers the batch's X rows (SB at a time in flight), each lane forms the LPR
// partial dot products of its column slice with the G row of each entry's row, and a
// butterfly transpose across the group leaves entry c's total in lane c (LPR - 1 shuffles
// per lane per batch), which stores it.
template <int LPR, int SBMAX, int MINB>
__global__ void __launch_bounds__(MG_THREADS, MINB) sddmm_merge_kernel(
    int32_t m, int32_t nnz, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
    const float* __restrict__ G, int64_t ldg, const float* __restrict__ X, int64_t ldx, float scale,
    float* __restrict__ out, int32_t items, int32_t nseg, const int32_t* __restrict__ seg_row) {
    constexpr int SB = LPR < SBMAX ? LPR : SBMAX;   // gathers in flight per lane
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR;
    const int c = lane % LPR;
    const unsigned gmask = LPR == 32 ? FULL : (((1u << LPR) - 1u) << (g * LPR));
    const int sg = (int)(((int64_t)blockIdx.x * MG_THREADS + threadIdx.x) / LPR);
    if (sg >= nseg) return;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const int tot = m + nnz;                     // < 2^31 (checked by the host)
    const int d0 = sg * items;
    const int d1 = items < tot - d0 ? d0 + items : tot;
    int row = seg_row[sg];
    const int row_last = seg_row[sg + 1];
    int e = d0 - row;
    const int e_end = d1 - row_last;
    if (e >= e_end) return;
    const float* xc = X + 4 * c;
    auto grow = [&](int32_t r) {
        return r < m ? __ldg(reinterpret_cast<const float4*>(G + (int64_t)r * ldg + 4 * c)) : f4_zero();
    };
    int row_end = row < m ? indptr[row + 1] : INT_MAX;
    int next_end = row + 1 < m ? indptr[row + 2] : INT_MAX;
    float4 gcur = grow(row);
    int32_t gnext_row = row + 1;
    float4 gnext = grow(gnext_row);
    int jnext = c < e_end - e ? ld_hint(indices + e + c, pol_stream) : -1;
    while (e < e_end) {
        const int nb = e_end - e < LPR ? e_end - e : LPR;
        const int jmine = jnext;
        float P[LPR];
#pragma unroll
        for (int q0 = 0; q0 < LPR; q0 += SB) {
            float4 xv[SB];
#pragma unroll
            for (int u = 0; u < SB; ++u) {
                const int jq = __shfl_sync(gmask, jmine, q0 + u, LPR);
                xv[u] = jq >= 0 ? ld_hint4(xc + (int64_t)jq * ldx, pol_keep) : f4_zero();
            }
            if (q0 == 0) {                       // the next batch's columns travel with these gathers
                const int en = e + nb;
                jnext = c < e_end - en ? ld_hint(indices + en + c, pol_stream) : -1;
            }
            // runs of entries of one row: [q, cut) of this part of the batch use G's row `row`
            const int hi = nb < q0 + SB ? nb : q0 + SB;
            int q = q0;
            for (;;) {
                const int left = row_end - e;
                const int cut = left < hi ? (left > q ? left : q) : hi;
#pragma unroll
                for (int u = 0; u < SB; ++u)
                    if (q0 + u >= q && q0 + u < cut)
                        P[q0 + u] = fmaf(gcur.x, xv[u].x, fmaf(gcur.y, xv[u].y, fmaf(gcur.z, xv[u].z, gcur.w * xv[u].w)));
                if (cut >= hi) break;
                // entry cut lies past this row's end: move to its row, G's row from the prefetch
                do {
                    ++row;
                    row_end = next_end;
                    next_end = row + 1 < m ? indptr[row + 2] : INT_MAX;
                } while (e + cut >= row_end);
                gcur = gnext_row == row ? gnext : grow(row);
                gnext_row = row + 1;
                gnext = grow(gnext_row);
                q = cut;
            }
#pragma unroll
            for (int u = 0; u < SB; ++u)
                if (q0 + u >= hi) P[q0 + u] = 0.f;
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
        if (c < nb) __stcs(out + e + c, scale * P[0]);
        e += nb;
    }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int lanes_for(int32_t k) {
    switch (k) {
        case 4: return 1;
        case 8: return 2;
        case 16: return 4;
        case 32: return 8;
        case 64: return 16;
        case 128: return 32;
        default: return 0;
    }
}

spx_status check_plan(const spx_csr* A, const spx_mergeplan* plan, const char* who) {
    if (!plan || !plan->seg_row || plan->items < 1 || plan->n_segments < 1)
        return set_error(SPX_INVALID_ARG, "%s: bad merge plan", who);
    const int64_t tot = (int64_t)A->m + A->nnz;
    if (tot >= INT_MAX) return set_error(SPX_NOT_SUPPORTED, "%s: m + nnz >= 2^31", who);
    const int64_t want = tot == 0 ? 1 : (tot + plan->items - 1) / plan->items;
    if (want != plan->n_segments)
        return set_error(SPX_INVALID_ARG, "%s: merge plan of %d segments of %lld items, the matrix needs %lld", who,
                         plan->n_segments, (long long)plan->items, (long long)want);
    return SPX_OK;
}

template <int LPR, int B, int MINB>
spx_status launch_spmm_merge_b(bool permuted, unsigned grid, cudaStream_t st, const spx_csr* A, const int32_t* perm,
                               const float* vals, const float* X, int64_t ldx, float* Y, int64_t ldy, float alpha,
                               float beta, const spx_mergeplan* plan, int32_t* crow, float* cval) {
    if (permuted)
        spmm_merge_kernel<LPR, B, MINB, true><<<grid, MG_THREADS, 0, st>>>(
            A->m, (int32_t)A->nnz, A->indptr, A->indices, vals, perm, X, ldx, Y, ldy, alpha, beta,
            (int32_t)plan->items, plan->n_segments, plan->seg_row, crow, cval);
    else
        spmm_merge_kernel<LPR, B, MINB, false><<<grid, MG_THREADS, 0, st>>>(
            A->m, (int32_t)A->nnz, A->indptr, A->indices, vals, perm, X, ldx, Y, ldy, alpha, beta,
            (int32_t)plan->items, plan->n_segments, plan->seg_row, crow, cval);
    SPX_CHECK_LAUNCH("spx_spmm_merge");
    return SPX_OK;
}

template <int LPR>
spx_status launch_spmm_merge(int variant, bool permuted, unsigned grid, cudaStream_t st, const spx_csr* A,
                             const int32_t* perm, const float* vals, const float* X, int64_t ldx, float* Y,
                             int64_t ldy, float alpha, float beta, const spx_mergeplan* plan, int32_t* crow,
                             float* cval) {
    // variants: 0 = 8-entry batches, 4 resident blocks per SM; 1 = 8-entry, 5 blocks; 2 = 4-entry, 6 blocks
    switch (variant) {
        case 1:
            return launch_spmm_merge_b<LPR, 8, 5>(permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan,
                                                  crow, cval);
        case 2:
            return launch_spmm_merge_b<LPR, 4, 6>(permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan,
                                                  crow, cval);
        default:
            return launch_spmm_merge_b<LPR, 8, 4>(permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan,
                                                  crow, cval);
    }
}

template <int LPR, int SB, int MINB>
void sddmm_merge_go(unsigned grid, cudaStream_t st, const spx_csr* A, const float* G, int64_t ldg, const float* X,
                    int64_t ldx, float scale, float* out, const spx_mergeplan* plan) {
    sddmm_merge_kernel<LPR, SB, MINB><<<grid, MG_THREADS, 0, st>>>(A->m, (int32_t)A->nnz, A->indptr, A->indices, G,
                                                                    ldg, X, ldx, scale, out, (int32_t)plan->items,
                                                                    plan->n_segments, plan->seg_row);
}

template <int LPR>
spx_status launch_sddmm_merge(int variant, unsigned grid, cudaStream_t st, const spx_csr* A, const float* G,
                              int64_t ldg, const float* X, int64_t ldx, float scale, float* out,
                              const spx_mergeplan* plan) {
    // variants: 0 = 8 gathers in flight per lane, 4 resident blocks per SM; 1 = 4, 5 blocks; 2 = 8, 3 blocks
    switch (variant) {
        case 1: sddmm_merge_go<LPR, 4, 5>(grid, st, A, G, ldg, X, ldx, scale, out, plan); break;
        case 2: sddmm_merge_go<LPR, 8, 3>(grid, st, A, G, ldg, X, ldx, scale, out, plan); break;
        default: sddmm_merge_go<LPR, 8, 4>(grid, st, A, G, ldg, X, ldx, scale, out, plan); break;
    }
    SPX_CHECK_LAUNCH("spx_sddmm_merge");
    return SPX_OK;
}

size_t carry_bytes(int32_t nseg, int32_t k) {
    const size_t rows = ((size_t)nseg * 4 + 255) & ~size_t(255);
    return rows + (size_t)nseg * k * 4 + 256;
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_merge_plan_segments(const spx_csr* A, int64_t items, int32_t* n_segments) {
    if (!A || !n_segments || items < 1 || A->m < 0 || A->nnz < 0)
        return set_error(SPX_INVALID_ARG, "spx_merge_plan_segments: bad arguments");
    const int64_t tot = (int64_t)A->m + A->nnz;
    const int64_t ns = tot == 0 ? 1 : (tot + items - 1) / items;
    if (ns > INT_MAX - 1) return set_error(SPX_INVALID_ARG, "spx_merge_plan_segments: too many segments");
    *n_segments = (int32_t)ns;
    return SPX_OK;
}

extern "C" spx_status spx_merge_plan_build(const spx_csr* A, int64_t items, int32_t* seg_row, int32_t n_segments,
                                           void* stream) {
    SPX_TRY(check_csr(A, false, "spx_merge_plan_build"));
    int32_t ns = 0;
    SPX_TRY(spx_merge_plan_segments(A, items, &ns));
    if (!seg_row || n_segments != ns)
        return set_error(SPX_INVALID_ARG, "spx_merge_plan_build: n_segments %d, expected %d", n_segments, ns);
    const unsigned grid = (unsigned)(((int64_t)ns + 1 + 255) / 256);
    merge_partition_kernel<<<grid, 256, 0, as_stream(stream)>>>(A->m, A->nnz, A->indptr, items, ns, seg_row);
    SPX_CHECK_LAUNCH("spx_merge_plan_build");
    return SPX_OK;
}

extern "C" spx_status spx_spmm_merge_workspace_size(const spx_csr* A, int32_t k, const spx_mergeplan* plan,
                                                    size_t* bytes) {
    if (!A || !plan || !bytes || k < 1) return set_error(SPX_INVALID_ARG, "spx_spmm_merge_workspace_size: bad arguments");
    *bytes = carry_bytes(plan->n_segments, k);
    return SPX_OK;
}

extern "C" spx_status spx_spmm_merge(const spx_csr* A, const int32_t* perm, const float* X, int64_t ldx, int32_t k,
                                     float* Y, int64_t ldy, float alpha, float beta, const spx_mergeplan* plan,
                                     int32_t variant, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_spmm_merge"));
    const int lpr = lanes_for(k);
    if (lpr == 0) return set_error(SPX_NOT_SUPPORTED, "spx_spmm_merge: k = %d (4, 8, 16, 32, 64 or 128)", k);
    if (A->m > 0 && (!Y || ldy < k || ldy % 4 != 0 || !aligned16(Y)))
        return set_error(SPX_INVALID_ARG, "spx_spmm_merge: Y must be 16-byte aligned with ldy >= k, ldy %% 4 == 0");
    if (A->nnz > 0 && (!X || ldx < k || ldx % 4 != 0 || !aligned16(X)))
        return set_error(SPX_INVALID_ARG, "spx_spmm_merge: X must be 16-byte aligned with ldx >= k, ldx %% 4 == 0");
    if (variant < 0 || variant > 2) return set_error(SPX_INVALID_ARG, "spx_spmm_merge: variant %d (0..2)", variant);
    if (A->m == 0) return SPX_OK;
    SPX_TRY(check_plan(A, plan, "spx_spmm_merge"));
    const size_t need = carry_bytes(plan->n_segments, k);
    if (!ws || ws_bytes < need || !aligned16(ws))
        return set_error(SPX_OOM_WORKSPACE, "spx_spmm_merge: workspace %zu < %zu (16-byte aligned)", ws_bytes, need);
    int32_t* crow = static_cast<int32_t*>(ws);
    float* cval = reinterpret_cast<float*>(static_cast<char*>(ws) + (((size_t)plan->n_segments * 4 + 255) & ~size_t(255)));
    const float* vals = A->values;
    cudaStream_t st = as_stream(stream);
    const int64_t threads = (int64_t)plan->n_segments * lpr;
    const unsigned grid = (unsigned)((threads + MG_THREADS - 1) / MG_THREADS);
    const bool permuted = perm != nullptr;
    spx_status s;
    switch (lpr) {
        case 1: s = launch_spmm_merge<1>(variant, permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan, crow, cval); break;
        case 2: s = launch_spmm_merge<2>(variant, permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan, crow, cval); break;
        case 4: s = launch_spmm_merge<4>(variant, permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan, crow, cval); break;
        case 8: s = launch_spmm_merge<8>(variant, permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan, crow, cval); break;
        case 16: s = launch_spmm_merge<16>(variant, permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan, crow, cval); break;
        default: s = launch_spmm_merge<32>(variant, permuted, grid, st, A, perm, vals, X, ldx, Y, ldy, alpha, beta, plan, crow, cval); break;
    }
    if (s != SPX_OK) return s;
    const int32_t k4 = k / 4;
    const int64_t fix_threads = (int64_t)plan->n_segments * k4;
    merge_fixup_kernel<<<(unsigned)((fix_threads + 255) / 256), 256, 0, st>>>(plan->n_segments, k4, crow, cval, Y, ldy,
                                                                               alpha);
    SPX_CHECK_LAUNCH("spx_spmm_merge fix-up");
    return SPX_OK;
}

extern "C" spx_status spx_sddmm_merge(const spx_csr* A, const float* G, int64_t ldg, const float* X, int64_t ldx,
                                      int32_t k, float scale, float* out, const spx_mergeplan* plan, int32_t variant,
                                      void* stream) {
    SPX_TRY(check_csr(A, false, "spx_sddmm_merge"));
    const int lpr = lanes_for(k);
    if (lpr == 0) return set_error(SPX_NOT_SUPPORTED, "spx_sddmm_merge: k = %d (4, 8, 16, 32, 64 or 128)", k);
    if (A->nnz == 0) return SPX_OK;
    if (!out || !G || !X || ldg < k || ldx < k || ldg % 4 != 0 || ldx % 4 != 0 || !aligned16(G) || !aligned16(X))
        return set_error(SPX_INVALID_ARG, "spx_sddmm_merge: G, X 16-byte aligned with leading dimensions >= k, %% 4 == 0");
    if (variant < 0 || variant > 2) return set_error(SPX_INVALID_ARG, "spx_sddmm_merge: variant %d (0..2)", variant);
    SPX_TRY(check_plan(A, plan, "spx_sddmm_merge"));
    cudaStream_t st = as_stream(stream);
    const int64_t threads = (int64_t)plan->n_segments * lpr;
    const unsigned grid = (unsigned)((threads + MG_THREADS - 1) / MG_THREADS);
    switch (lpr) {
        case 1: return launch_sddmm_merge<1>(variant, grid, st, A, G, ldg, X, ldx, scale, out, plan);
        case 2: return launch_sddmm_merge<2>(variant, grid, st, A, G, ldg, X, ldx, scale, out, plan);
        case 4: return launch_sddmm_merge<4>(variant, grid, st, A, G, ldg, X, ldx, scale, out, plan);
        case 8: return launch_sddmm_merge<8>(variant, grid, st, A, G, ldg, X, ldx, scale, out, plan);
        case 16: return launch_sddmm_merge<16>(variant, grid, st, A, G, ldg, X, ldx, scale, out, plan);
        default: return launch_sddmm_merge<32>(variant, grid, st, A, G, ldg, X, ldx, scale, out, plan);
    }
}
