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
    int32_t cb = col_block > 0 ? col_block : slab_col_block(A->n, k);
    if (cb > k) cb = k;
    if (vec4 && cb % 4 != 0) cb = (cb + 3) / 4 * 4;
    return cb;
}

spx_status launch_sddmm(const spx_csr* A, const float* G, int64_t ldg, const float* X, int64_t ldx, int32_t k,
                        float scale, float* out, int32_t col_block, float* ws, size_t ws_bytes, cudaStream_t st) {
    if (A->nnz == 0) return SPX_OK;
    const bool vec4 = (k % 4 == 0) && (ldg % 4 == 0) && (ldx % 4 == 0) && aligned16(G) && aligned16(X);
    const int VEC = vec4 ? 4 : 1;
    const int32_t cb = sddmm_cb(A, k, col_block, vec4);
    const size_t slab = vec4 ? slab_bytes(A->n, k, cb) : 0;
    const bool use_slab = slab > 0 && ws != nullptr && ws_bytes >= slab;
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
                                int32_t k, float scale, float* out, int32_t col_block, void* ws, size_t ws_bytes,
                                void* stream) {
    SPX_TRY(check_csr(A, false, "spx_sddmm"));
    if (k < 1 || ldg < k || ldx < k) return set_error(SPX_INVALID_ARG, "spx_sddmm: bad k / leading dims");
    if (A->nnz > 0 && (!G || !X || !out)) return set_error(SPX_INVALID_ARG, "spx_sddmm: NULL operand");
    if (ws) {
        const bool vec4 = (k % 4 == 0) && (ldg % 4 == 0) && (ldx % 4 == 0) && aligned16(G) && aligned16(X);
        const size_t need = vec4 ? slab_bytes(A->n, k, sddmm_cb(A, k, col_block, true)) : 0;
        if (ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_sddmm: workspace %zu < %zu", ws_bytes, need);
    }
    return launch_sddmm(A, G, ldg, X, ldx, k, scale, out, col_block, static_cast<float*>(ws), ws_bytes,
                        as_stream(stream));
}

extern "C" spx_status spx_masked_outer(const spx_csr* A, const float* u, const float* v, float scale, float* out,
                                       void* stream) {
    SPX_TRY(check_csr(A, false, "spx_masked_outer"));
    if (A->nnz > 0 && (!u || !v || !out)) return set_error(SPX_INVALID_ARG, "spx_masked_outer: NULL operand");
    return launch_sddmm(A, u, 1, v, 1, 1, scale, out, 1, nullptr, 0, as_stream(stream));
}
