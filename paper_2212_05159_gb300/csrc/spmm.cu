// Row-wise sparse x dense products:
//   spx_spmm    Y  = alpha * A X   + beta * Y      (Section 3.1.1 SpMV, 3.1.3 SpDMM)
//   spx_spmm_t  gX = alpha * A^T G + beta * gX     (Table 1, gradient w.r.t. the dense
//                                                   operand, on the transposed pattern)
//
// Mapping (HBM-bound gather; no tensor cores: each A entry is used once per output row):
//   * a "row slot" of S lanes (S | 32) owns one row; inside it LPR lanes span the k
//     columns with float4 loads (VEC = 4) and G = S / LPR lane groups walk the row's
//     entries with stride G, so one warp issues G coalesced row-gathers of X at a time;
//   * partial sums of the G groups are combined with xor-shuffles in a fixed order;
//   * rows longer than the plan threshold are taken by whole thread blocks (8 warps,
//     8*G entries in flight) that reduce through shared memory in warp order; those
//     blocks are the lowest block ids of the same launch, so they start first and
//     overlap the short rows.
// Every output is reduced in a fixed order: results are deterministic.
// CSR streams are read with evict-first loads so that L2 keeps the gathered X rows.
#include <limits.h>

#include "common.cuh"
#include "scan.cuh"

namespace spx {
namespace {

constexpr int SPMM_THREADS = 256;
constexpr int SPMM_WARPS = SPMM_THREADS / 32;

template <int VEC>
struct Vec;
template <>
struct Vec<4> {
    using T = float4;
};
template <>
struct Vec<1> {
    using T = float;
};

template <int VEC>
__device__ __forceinline__ void fma_row(float (&acc)[VEC], float v, const float* __restrict__ p) {
    if constexpr (VEC == 4) {
        float4 x = __ldg(reinterpret_cast<const float4*>(p));
        acc[0] = fmaf(v, x.x, acc[0]);
        acc[1] = fmaf(v, x.y, acc[1]);
        acc[2] = fmaf(v, x.z, acc[2]);
        acc[3] = fmaf(v, x.w, acc[3]);
    } else {
        acc[0] = fmaf(v, __ldg(p), acc[0]);
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
__device__ __forceinline__ float load_val(const float* __restrict__ vals, const int32_t* __restrict__ perm,
                                          int e) {
    if constexpr (PERM)
        return __ldg(vals + ld_stream(perm + e));
    else
        return ld_stream(vals + e);
}

// blocks [0, long_blocks) process plan rows; the others process short rows.
template <int VEC, bool PERM>
__global__ void __launch_bounds__(SPMM_THREADS) spmm_kernel(
    int32_t m, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
    const float* __restrict__ vals, const int32_t* __restrict__ perm, const float* __restrict__ X, int64_t ldx,
    int32_t k, float* __restrict__ Y, int64_t ldy, float alpha, float beta, int lpr_log2, int s_log2,
    int32_t threshold, const int32_t* __restrict__ long_rows, int32_t n_long, int32_t long_blocks) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int LPR = 1 << lpr_log2;
    const int c = lane & (LPR - 1);           // column lane inside the slot
    const int colstep = LPR * VEC;

    if ((int)blockIdx.x < long_blocks) {
        // ---------------- long rows: the whole block on one row, groups of LPR lanes
        __shared__ float red[SPMM_WARPS][128];
        const int Gw = 32 >> lpr_log2;         // groups per warp
        const int g = lane >> lpr_log2;
        const int gid = warp * Gw + g;
        const int Gb = SPMM_WARPS * Gw;        // groups per block
        for (int q = blockIdx.x; q < n_long; q += long_blocks) {
            const int row = long_rows[q];
            const int a = indptr[row], b = indptr[row + 1];
            for (int col0 = 0; col0 < k; col0 += colstep) {
                const int col = col0 + c * VEC;
                const bool colok = col < k;
                float acc[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
                if (colok) {
#pragma unroll 4
                    for (int e = a + gid; e < b; e += Gb) {
                        const int j = ld_stream(indices + e);
                        const float av = load_val<PERM>(vals, perm, e);
                        fma_row<VEC>(acc, av, X + (int64_t)j * ldx + col);
                    }
                }
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
                    store_row<VEC>(Y + (int64_t)row * ldy + col, tot, alpha, beta);
                }
                __syncthreads();
            }
        }
        return;
    }

    // ---------------- short rows: S lanes per row
    const int S = 1 << s_log2;
    const int sl = lane & (S - 1);
    const int g = sl >> lpr_log2;
    const int G = S >> lpr_log2;
    const int64_t gw = ((int64_t)(blockIdx.x - long_blocks) * SPMM_THREADS + threadIdx.x) >> 5;
    const int64_t row = (gw << (5 - s_log2)) + (lane >> s_log2);
    int a = 0, b = 0;
    bool active = row < m;
    if (active) {
        a = indptr[row];
        b = indptr[row + 1];
        if (b - a > threshold) active = false;     // taken by the long-row blocks
    }
    if (!active) b = a;
    for (int col0 = 0; col0 < k; col0 += colstep) {
        const int col = col0 + c * VEC;
        const bool colok = col < k;
        float acc[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[v] = 0.f;
        if (colok) {
#pragma unroll 4
            for (int e = a + g; e < b; e += G) {
                const int j = ld_stream(indices + e);
                const float av = load_val<PERM>(vals, perm, e);
                fma_row<VEC>(acc, av, X + (int64_t)j * ldx + col);
            }
        }
        for (int off = LPR; off < S; off <<= 1)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] += __shfl_xor_sync(FULL, acc[v], off);
        if (active && g == 0 && colok) store_row<VEC>(Y + row * ldy + col, acc, alpha, beta);
    }
}

int ilog2_ceil(int64_t x) {
    int l = 0;
    while ((int64_t(1) << l) < x) ++l;
    return l;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <bool PERM>
spx_status launch_spmm(const spx_csr* A, const int32_t* perm, const float* X, int64_t ldx, int32_t k,
                       float* Y, int64_t ldy, float alpha, float beta, const spx_rowplan* plan,
                       cudaStream_t st, const char* who) {
    if (A->m == 0 || k == 0) return SPX_OK;
    const bool vec4 = (k % 4 == 0) && (ldx % 4 == 0) && (ldy % 4 == 0) && aligned16(X) && aligned16(Y);
    const int VEC = vec4 ? 4 : 1;
    const int64_t lanes_needed = (k + VEC - 1) / VEC;
    int lpr_log2 = ilog2_ceil(lanes_needed);
    if (lpr_log2 > 5) lpr_log2 = 5;
    // groups per row ~ half the mean row length (at least one), slot width <= 32 lanes
    const double mean = A->m > 0 ? (double)A->nnz / (double)A->m : 0.0;
    int glog = ilog2_ceil((int64_t)(mean / 2.0 + 0.999));
    int s_log2 = lpr_log2 + glog;
    if (s_log2 > 5) s_log2 = 5;
    if (s_log2 < lpr_log2) s_log2 = lpr_log2;

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
    const int64_t rows_per_block = (int64_t)SPMM_WARPS << (5 - s_log2);
    const int64_t short_blocks = ((int64_t)A->m + rows_per_block - 1) / rows_per_block;
    const int64_t grid = short_blocks + long_blocks;
    if (grid > INT_MAX) return set_error(SPX_INVALID_ARG, "%s: too many rows", who);
    if (vec4)
        spmm_kernel<4, PERM><<<(unsigned)grid, SPMM_THREADS, 0, st>>>(
            A->m, A->indptr, A->indices, A->values, perm, X, ldx, k, Y, ldy, alpha, beta, lpr_log2, s_log2,
            threshold, long_rows, n_long, long_blocks);
    else
        spmm_kernel<1, PERM><<<(unsigned)grid, SPMM_THREADS, 0, st>>>(
            A->m, A->indptr, A->indices, A->values, perm, X, ldx, k, Y, ldy, alpha, beta, lpr_log2, s_log2,
            threshold, long_rows, n_long, long_blocks);
    SPX_CHECK_LAUNCH(who);
    return SPX_OK;
}

__global__ void long_flag_kernel(int32_t m, const int32_t* __restrict__ indptr, int32_t threshold,
                                 int32_t* __restrict__ flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m) flags[i] = (indptr[i + 1] - indptr[i]) > threshold ? 1 : 0;
}

__global__ void long_compact_kernel(int32_t m, const int32_t* __restrict__ flags, const int32_t* __restrict__ pos,
                                    int32_t* __restrict__ long_rows) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < m && flags[i]) long_rows[pos[i]] = (int32_t)i;
}

size_t rowplan_ws(int32_t m) {
    size_t a = ((size_t)m * 4 + 255) & ~size_t(255);
    size_t b = (((size_t)m + 1) * 4 + 255) & ~size_t(255);
    return a + b + scan_workspace_bytes<int32_t>(m);
}

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
    long_flag_kernel<<<blocks, 256, 0, st>>>(A->m, A->indptr, threshold, flags);
    SPX_CHECK_LAUNCH("long_flag");
    SPX_TRY((scan_counts<int32_t, int32_t>(flags, pos, A->m, sws, st)));
    long_compact_kernel<<<blocks, 256, 0, st>>>(A->m, flags, pos, long_rows);
    SPX_CHECK_LAUNCH("long_compact");
    SPX_CUDA(cudaMemcpyAsync(n_long_host, pos + A->m, sizeof(int32_t), cudaMemcpyDeviceToHost, st),
             "spx_rowplan_build copy");
    SPX_CUDA(cudaStreamSynchronize(st), "spx_rowplan_build sync");
    return SPX_OK;
}

static spx_status check_dense(const void* p, int64_t rows, int64_t ld, int32_t k, const char* who,
                              const char* name) {
    if (rows > 0 && k > 0 && !p) return set_error(SPX_INVALID_ARG, "%s: NULL %s", who, name);
    if (k < 0 || ld < k || ld < 1) return set_error(SPX_INVALID_ARG, "%s: bad ld/k for %s", who, name);
    return SPX_OK;
}

extern "C" spx_status spx_spmm(const spx_csr* A, const float* X, int64_t ldx, int32_t k, float* Y,
                               int64_t ldy, float alpha, float beta, const spx_rowplan* plan, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_spmm"));
    SPX_TRY(check_dense(X, A->n, ldx, k, "spx_spmm", "X"));
    SPX_TRY(check_dense(Y, A->m, ldy, k, "spx_spmm", "Y"));
    return launch_spmm<false>(A, nullptr, X, ldx, k, Y, ldy, alpha, beta, plan, as_stream(stream), "spx_spmm");
}

extern "C" spx_status spx_spmm_t(const spx_csr* AT, const int32_t* perm, const float* G, int64_t ldg,
                                 int32_t k, float* gX, int64_t ldgx, float alpha, float beta,
                                 const spx_rowplan* plan, void* stream) {
    SPX_TRY(check_csr(AT, true, "spx_spmm_t"));
    if (AT->nnz > 0 && !perm) return set_error(SPX_INVALID_ARG, "spx_spmm_t: NULL perm");
    SPX_TRY(check_dense(G, AT->n, ldg, k, "spx_spmm_t", "G"));
    SPX_TRY(check_dense(gX, AT->m, ldgx, k, "spx_spmm_t", "gX"));
    return launch_spmm<true>(AT, perm, G, ldg, k, gX, ldgx, alpha, beta, plan, as_stream(stream), "spx_spmm_t");
}
