// Sparse triangular solve (Section 3.1.5) for a block-diagonal batch of lower-triangular
// systems, L x = b, and the transposed solve L^T y = v that its vector-Jacobian product
// needs (grad_b = L^-T v; grad_L = -(L^-T v) x^T on mask(L) is spx_masked_outer).
//
// Level scheduling instead of the paper's synchronisation-free solve: the levels of the
// lower pattern (spx_ic0_analyse) are walked by one thread block per system, rows of a level
// in parallel, one block barrier between levels -- no thread ever waits on a flag written by
// another block.  The transposed solve walks the same levels in reverse order on the CSR of
// L^T (upper triangular).  The rows of the next level are fetched while a level solves
// (trisolve.cuh); each row's sum is accumulated in double-float (FP32 pair) before the
// division by the pivot.  A zero, non-finite or missing pivot sets the system's status
// to SPX_BREAKDOWN (its solution is then not meaningful).
#include <math.h>

#include "common.cuh"
#include "trisolve.cuh"

namespace spx {
namespace {

constexpr int TRSV_THREADS = 512;

// upper = 0: T is lower with the diagonal last in each row, levels ascending;
// upper = 1: T is upper (the CSR of L^T) with the diagonal first, levels descending.
// The first TRSV_THREADS rows of the next level are fetched while the current level solves.
__global__ void __launch_bounds__(TRSV_THREADS) sptrsv_kernel(int32_t nsys, int32_t upper,
                                                              const int32_t* __restrict__ tp,
                                                              const int32_t* __restrict__ ti,
                                                              const float* __restrict__ tv,
                                                              const int32_t* __restrict__ off,
                                                              const int32_t* __restrict__ lev_ptr,
                                                              const int32_t* __restrict__ lev_rows,
                                                              const float* __restrict__ b, float* __restrict__ x,
                                                              int32_t* __restrict__ status) {
    const int s = blockIdx.x;
    if (s >= nsys) return;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int32_t* lp = lev_ptr + off[s];
    const int nl = off[s + 1] - off[s] - 1;
    const bool lower = upper == 0;
    const int tid = threadIdx.x;
    auto level = [&](int t) { return upper ? nl - 1 - t : t; };
    auto check = [&](const TriRow& r) {
        if (r.i >= 0 && (r.piv == 0.f || !isfinite(r.piv))) atomicOr(&bad, 1);
    };
    TriRow cur;
    if (nl > 0) cur = fetch_tri_row(lower, lp[level(0)] + tid, lp[level(0) + 1], lev_rows, tp, ti, tv, b);
    for (int t = 0; t < nl; ++t) {
        const int l = level(t);
        TriRow nxt;
        if (t + 1 < nl)
            nxt = fetch_tri_row(lower, lp[level(t + 1)] + tid, lp[level(t + 1) + 1], lev_rows, tp, ti, tv, b);
        check(cur);
        solve_tri_row_df(cur, ti, tv, x);
        for (int q = lp[l] + TRSV_THREADS + tid; q < lp[l + 1]; q += TRSV_THREADS) {
            const TriRow r = fetch_tri_row(lower, q, lp[l + 1], lev_rows, tp, ti, tv, b);
            check(r);
            solve_tri_row_df(r, ti, tv, x);
        }
        __syncthreads();
        cur = nxt;
    }
    if (threadIdx.x == 0 && status) status[s] = bad ? SPX_BREAKDOWN : SPX_OK;
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_sptrsv(const spx_csr* T, int32_t upper, int32_t nsys, const int32_t* sys_lev_off,
                                 const int32_t* lev_ptr, const int32_t* lev_rows,
                                 const float* b, float* x, int32_t* status, void* stream) {
    SPX_TRY(check_csr(T, true, "spx_sptrsv"));
    if (T->m != T->n) return set_error(SPX_INVALID_ARG, "spx_sptrsv: the matrix must be square");
    if (upper != 0 && upper != 1) return set_error(SPX_INVALID_ARG, "spx_sptrsv: upper is 0 or 1");
    if (nsys < 0 || (nsys > 0 && (!sys_lev_off || !lev_ptr || !lev_rows || !b || !x)))
        return set_error(SPX_INVALID_ARG, "spx_sptrsv: NULL argument");
    if (nsys == 0) return SPX_OK;
    sptrsv_kernel<<<(unsigned)nsys, TRSV_THREADS, 0, as_stream(stream)>>>(
        nsys, upper, T->indptr, T->indices, T->values, sys_lev_off, lev_ptr, lev_rows, b, x, status);
    SPX_CHECK_LAUNCH("spx_sptrsv");
    return SPX_OK;
}
