// Level-scheduled sparse triangular solves: one row of a level, fetched ahead of its level.
//
// Rows of one level depend only on rows of earlier levels, so everything a row needs except
// the solution entries it reads (row id, bounds, off-diagonal entries, pivot, right-hand side)
// can be loaded while the previous level is still being solved.  A level then costs one round
// trip for those solution entries plus the barrier that closes it.  Used by the IC(0)
// application inside the batched PCG and by the standalone batched solve (Section 3.1.5).
#pragma once

#include "common.cuh"

namespace spx {
namespace {

constexpr int TRI_PRE = 2;                      // off-diagonal entries held in registers (5-point IC(0): 2)

struct TriRow {
    int i = -1;                                 // row (-1: none)
    int e = 0, e_end = 0;                       // off-diagonal entries [e, e_end)
    int j[TRI_PRE];
    float v[TRI_PRE];
    float piv = 1.f, rhs = 0.f;
};

// lower = true: a lower-triangular CSR with the diagonal last in each row; lower = false: an
// upper-triangular CSR (the transpose of such a matrix) with the diagonal first.  A row whose
// pivot slot does not hold its diagonal gets pivot 0 (the caller reports the breakdown).
__device__ __forceinline__ TriRow fetch_tri_row(bool lower, int q, int q_end, const int32_t* __restrict__ rows,
                                                const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                                const float* __restrict__ val, const float* __restrict__ src) {
    TriRow t;
    if (q >= q_end) return t;
    const int i = rows[q];
    const int a = ptr[i], b = ptr[i + 1];
    t.i = i;
    t.rhs = src[i];
    if (b <= a) {
        t.piv = 0.f;
        return t;
    }
    const int d = lower ? b - 1 : a;
    t.e = lower ? a : a + 1;
    t.e_end = lower ? b - 1 : b;
    t.piv = idx[d] == i ? val[d] : 0.f;
#pragma unroll
    for (int u = 0; u < TRI_PRE; ++u) {
        const int k = t.e + u;
        const bool ok = k < t.e_end;
        t.j[u] = ok ? idx[k] : i;
        t.v[u] = ok ? val[k] : 0.f;
    }
    return t;
}

// x[i] = (rhs - sum of the row's off-diagonal entries times x) / pivot, FP32 accumulation.
__device__ __forceinline__ void solve_tri_row(const TriRow& t, const int32_t* __restrict__ idx,
                                              const float* __restrict__ val, float* __restrict__ x) {
    if (t.i < 0) return;
    float s = t.rhs;
#pragma unroll
    for (int u = 0; u < TRI_PRE; ++u) s = fmaf(-t.v[u], x[t.j[u]], s);
    for (int k = t.e + TRI_PRE; k < t.e_end; ++k) s = fmaf(-val[k], x[idx[k]], s);
    x[t.i] = s / t.piv;
}

// The same with the row's sum in double-float (an FP32 pair with exact products).
__device__ __forceinline__ void solve_tri_row_df(const TriRow& t, const int32_t* __restrict__ idx,
                                                 const float* __restrict__ val, float* __restrict__ x) {
    if (t.i < 0) return;
    float hi = t.rhs, lo = 0.f;
    auto add = [&](float a, float b) {
        const float ph = a * b;
        const float pl = fmaf(a, b, -ph);
        const float s = hi + ph;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (ph - bp);
        hi = s;
        lo += err + pl;
    };
#pragma unroll
    for (int u = 0; u < TRI_PRE; ++u) add(-t.v[u], x[t.j[u]]);
    for (int k = t.e + TRI_PRE; k < t.e_end; ++k) add(-val[k], x[idx[k]]);
    x[t.i] = (hi + lo) / t.piv;
}

}  // namespace
}  // namespace spx
