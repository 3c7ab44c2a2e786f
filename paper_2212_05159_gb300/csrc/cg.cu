// Batched preconditioned conjugate gradient on a block-diagonal CSR matrix (one SPD
// system per block), the differentiable sparse solve of Section 4.3 / Table 1 (SpSolve)
// with the direct solve replaced by PCG, and its adjoint.
//
// One persistent launch.  Each thread-block cluster (CL blocks on CL SMs) takes one
// system at a time from a queue (largest first when an order is given) and runs PCG on
// it to completion; its blocks split the system's rows.  Dot products are reduced inside
// each block and then across the cluster through distributed shared memory (one cluster
// barrier per reduction, partials double-buffered, summed in rank order: deterministic);
// the scalars of the iteration (alpha, beta, norms, stopping decisions) are then computed
// once per block by its thread 0 in FP64 and broadcast through shared memory.
//
// Every loop gives row i of a block's range to the same thread, so the vectors that are
// read only on a thread's own rows (x's FP32 partial, A p, z, D^-1, r unless M gathers it,
// and a copy of p) never cross threads: when a block's rows fit 8 per thread they live in
// the block's shared memory (192 KB at 1024 threads) instead of the workspace, and only p
// (and r for an explicit M), which the sparse products gather, goes through L2.  The
// arithmetic is the same either way.
//
// Precision (GB300 has ~1/60 of its FP32 rate in FP64): the iteration runs in FP32 with
// "reliable updates" -- the solution accumulates in an FP32 partial that is folded into
// the FP64 x whenever the recurrence residual has dropped by `delta` (and at the end);
// at every fold the residual is recomputed in FP64 as b - A x and that true residual
// decides convergence (||b - A x|| <= tol ||b||).  Inner products accumulate per thread
// in double-float (an FP32 pair with exact products, ~44 significant bits) and are
// combined in double-float up to the last cross-block sum, which is converted to FP64.  Preconditioners: none, Jacobi (z = D^-1 r), the factored
// approximate inverse M = L L^T of Section 4.3 (z = L (L^T r), two sparse products), and
// an explicit sparse M (z = M r, one product; e.g. L L^T formed once by SpGEMM),
// IC(0) (z = (L L^T)^-1 r by two level-scheduled triangular solves), and a symmetric M
// given by at most four lower diagonals (e.g. L L^T of a factor on tril(A) of a 5-point
// grid), kept in shared memory and applied in one pass (kind 5).
//
// Status per system: SPX_OK, SPX_MAXITER, SPX_BREAKDOWN (p^T A p <= 0 or r^T z <= 0),
// SPX_NONFINITE.  No spin waits: only cluster / block barriers.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <math.h>

#include <limits.h>

#include <atomic>
#include <vector>

#include "common.cuh"
#include "trisolve.cuh"

namespace cg = cooperative_groups;

namespace spx {
namespace {

constexpr int CG_MAX_WARPS = 32;
// Rows up to this long are multiplied two at a time (spmv_row2).  Five covers the 5-point
// stencil: 4-6 % faster PCG on 2D diffusion batches than one row at a time; wider paths
// spill under the 64-register cap (a 7-entry pair for the explicit M: 9 % slower).
constexpr int CG_ROW2_W = 5;

// Private vector rows per block kept in shared memory: 8 per thread (6 vectors, 192 bytes
// per thread: 192 KB for 1024 threads, within the 227 KB a block may use; with fewer
// threads the blocks that share an SM split the same budget).
constexpr int CG_SMEM_ROWS_PER_THREAD = 8;
constexpr int CG_SMEM_VECTORS = 6;
// Kind 5 keeps q, z, r and p's own entries in shared memory (4 vectors) and the block's rows of
// the at most CG_MDIA_MAX lower diagonals of the symmetric M = L L^T in BF16; x's FP32 partial
// stays in the workspace.  128 + 64 KB at 1024 threads.  L itself has at most CG_DIA_MAX
// diagonals (spx_dia_analyse / spx_dia_fill); spx_dia_square forms M's.
constexpr int CG_DIA_MAX = 3;
constexpr int CG_MDIA_MAX = 4;
constexpr int CG_DIA_VECTORS = 4;

struct CgArgs {
    int32_t nsys;
    const int32_t* sys_ptr;
    const int32_t* order;
    const int32_t* a_ptr;
    const int32_t* a_idx;
    const float* a_val;
    const float* b;
    double* x;
    int32_t pc;
    const float* dinv;
    const int32_t* l_ptr;
    const int32_t* l_idx;
    const float* l_val;
    const int32_t* lt_ptr;
    const int32_t* lt_idx;
    const float* lt_val;
    float* r;
    float* p;
    float* q;
    float* z;
    float* w;
    float* xp;
    double tol;
    double delta;
    int32_t maxit;
    int32_t* iters;
    int32_t* status;
    double* relres;
    int32_t* queue;
    const int32_t* lev_off;   // IC(0): per-system offsets into lev_ptr
    const int32_t* lev_ptr;   // IC(0): level l of a system = lev_rows[lev_ptr[l] .. lev_ptr[l+1])
    const int32_t* lev_rows;
    int32_t smem_rows;        // rows of a block's private vectors that fit in shared memory (0: none)
    // kind 5: the symmetric M by its lower diagonals, M_{i, i - off[d]} = M_{i - off[d], i} =
    // dia_val[d * n + i], per system
    const int32_t* dia_off;   // [nsys * CG_MDIA_MAX] distances (>= 0), ascending, the first 0
    const int32_t* dia_nd;    // [nsys] diagonals per system
    const __nv_bfloat16* dia_val;
    int32_t n;                // rows of the batch
};

// The vectors a thread reads only on its own rows, as seen by one system: in shared memory
// (element i at [i - off]) when the block's rows fit, else the global workspace (off = 0).
// p is written to both (other blocks gather it from global memory); r lives in global
// memory when the preconditioner gathers it (explicit M).
struct Vecs {
    float* xp;
    float* q;
    float* z;
    float* r;
    const float* di;
    float* po;        // the thread's own entries of p
    int off;
    bool sm;
    // kind 5 only (shared memory): the block's rows of M's lower diagonals
    const __nv_bfloat16* md = nullptr;
    int cap = 0;
};

// A system's M as a block sees it: lower diagonals at distances off[d] (d < nd, off[0] = 0),
// halo depth H = max off[d], the system's rows [R0, R1), the block's rows [lo, hi) and the
// row count of a block (chunk; the next block's rows start at hi, the previous block's at
// lo - chunk).
struct DiaSys {
    int nd, H, R0, R1, lo, hi, chunk;
    int off[CG_MDIA_MAX];
    bool ok;
};

// ---------------------------------------------------------------- double-float sums
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void df_add_prod(DF& s, float a, float b) {
    const float ph = a * b;
    const float pl = fmaf(a, b, -ph);          // exact: a*b = ph + pl
    const float t = s.hi + ph;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (ph - bp);
    s.hi = t;
    s.lo += err + pl;
}

// a + b in double-float (two-sum of the high parts, low parts added, renormalised)
__device__ __forceinline__ DF df_add(const DF& a, const DF& b) {
    const float t = a.hi + b.hi;
    const float bp = t - a.hi;
    const float err = (a.hi - (t - bp)) + (b.hi - bp) + (a.lo + b.lo);
    const float hi = t + err;
    return DF{hi, err - (hi - t)};
}

__device__ __forceinline__ DF df_of(double x) {
    const float hi = (float)x;
    return DF{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ DF df_shfl_down(const DF& v, int o) {
    return DF{__shfl_down_sync(FULL, v.hi, o), __shfl_down_sync(FULL, v.lo, o)};
}

// Sums NV double-float values over the cluster; the totals land in `out` of thread 0 of
// every block (all blocks add the same partials in the same order, so they agree).  All
// arithmetic before the last step is FP32 (double-float): GB300's FP64 rate is ~1/64 of its
// FP32 rate, and a reduction done in FP64 by every thread costs more than the sparse
// product it follows.  Warp: shuffle tree; block: warp 0 over the warp partials; cluster:
// lanes of warp 0 read the block partials through DSMEM (rank order), double-buffered so
// one cluster barrier per reduction suffices.
template <int NT, int NV>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, DF (&v)[NV], double (&out)[NV], float2 (*red)[4],
                                           float2 (*part)[4], int& slot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) v[k] = df_add(v[k], df_shfl_down(v[k], o));
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[warp][k] = make_float2(v[k].hi, v[k].lo);
    __syncthreads();
    const unsigned ncl = cl.num_blocks();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            DF t{0.f, 0.f};
            if (lane < NT / 32) t = DF{red[lane][k].x, red[lane][k].y};
#pragma unroll
            for (int o = NT / 64; o >= 1; o >>= 1) t = df_add(t, df_shfl_down(t, o));
            if (lane == 0) part[slot][k] = make_float2(t.hi, t.lo);
        }
    }
    cl.sync();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            DF t{0.f, 0.f};
            if (lane < (int)ncl) {
                const float2 pv = *cl.map_shared_rank(&part[slot][k], (unsigned)lane);
                t = DF{pv.x, pv.y};
            }
            for (int o = 16; o >= 1; o >>= 1)
                if (o < (int)ncl) t = df_add(t, df_shfl_down(t, o));
            out[k] = (double)t.hi + (double)t.lo;
        }
    }
    slot ^= 1;
}

// Scalars of the iteration, decided by thread 0 of each block and read by all its threads.
struct CgBcast {
    float alpha, beta;
    int action;                // ACT_* below
};
constexpr int ACT_GO = 0, ACT_STOP = 1, ACT_FOLD = 2;

// The FP64 state of one system, kept by thread 0 of each block in shared memory (no other
// thread reads it, so it holds no registers of the others through the iteration).
struct CgScal {
    double bnorm, rz, ref, last_true;
    int status;
};

// One row of a sparse product, entries in order; the loads of up to 8 entries are issued
// together (predicated tail) so that a row costs two dependent round trips, not one per
// entry.
__device__ __forceinline__ float spmv_row(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                          const float* __restrict__ val, const float* __restrict__ x, int i) {
    const int b = ptr[i], e = ptr[i + 1];
    float s = 0.f;
    int k = b;
    for (; k + 8 <= e; k += 8) {
        int j[8];
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            j[q] = idx[k + q];
            v[q] = val[k + q];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) s = fmaf(v[q], x[j[q]], s);
    }
    int j[8];
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const bool ok = k + q < e;
        j[q] = ok ? idx[k + q] : i;
        v[q] = ok ? val[k + q] : 0.f;
    }
    float t[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) t[q] = x[j[q]];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (k + q < e) s = fmaf(v[q], t[q], s);
    return s;
}

// spmv_row for rows i0 and (when has1) i1 together: with both rows at most W entries long
// their bounds, entries and gathered values are each loaded for both rows at once (three
// round trips for the pair instead of three per row); longer rows take spmv_row.  The
// products are the same, added in the same order.
template <int W>
__device__ __forceinline__ void spmv_row2(const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                          const float* __restrict__ val, const float* __restrict__ x, int i0, int i1,
                                          bool has1, float& s0, float& s1) {
    const int b0 = ptr[i0], e0 = ptr[i0 + 1];
    const int b1 = has1 ? ptr[i1] : 0, e1 = has1 ? ptr[i1 + 1] : 0;
    if (e0 - b0 > W || e1 - b1 > W) {
        s0 = spmv_row(ptr, idx, val, x, i0);
        s1 = has1 ? spmv_row(ptr, idx, val, x, i1) : 0.f;
        return;
    }
    int j0[W], j1[W];
    float v0[W], v1[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        const bool ok0 = b0 + q < e0, ok1 = b1 + q < e1;
        j0[q] = ok0 ? idx[b0 + q] : i0;
        v0[q] = ok0 ? val[b0 + q] : 0.f;
        j1[q] = ok1 ? idx[b1 + q] : i0;
        v1[q] = ok1 ? val[b1 + q] : 0.f;
    }
    float t0[W], t1[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
        t0[q] = x[j0[q]];
        t1[q] = x[j1[q]];
    }
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int q = 0; q < W; ++q) {
        if (b0 + q < e0) a0 = fmaf(v0[q], t0[q], a0);
        if (b1 + q < e1) a1 = fmaf(v1[q], t1[q], a1);
    }
    s0 = a0;
    s1 = a1;
}

// z = M r on rows [lo, hi) of the system (the caller barriers around LLT's two halves)
template <int NT, int PC>
__device__ __forceinline__ void apply_pc_local(const Vecs& v, int lo, int hi) {
    if constexpr (PC == 1) {
        for (int i = lo + threadIdx.x; i < hi; i += NT) v.z[i - v.off] = v.di[i - v.off] * v.r[i - v.off];
    } else if constexpr (PC == 0) {
        for (int i = lo + threadIdx.x; i < hi; i += NT) v.z[i - v.off] = v.r[i - v.off];
    }
}

// IC(0): z = L^-T L^-1 r with level-scheduled triangular solves, run by the cluster's
// first block (block barriers between levels) while the others wait at the cluster
// barrier.  L: lower CSR (diagonal last in each row); LT: its transpose (diagonal first).
// The first NT rows of the next level are fetched (row ids, bounds, entries, pivot, right-
// hand side) while the current level computes, so a level costs one round trip for the
// solution entries it reads plus the barrier; rows beyond NT in a level are fetched in place.
template <int NT>
__device__ __noinline__ void ic0_apply(const CgArgs& a, unsigned rank, int sid) {
    if (rank != 0) return;
    const int32_t* lp = a.lev_ptr + a.lev_off[sid];
    const int nl = a.lev_off[sid + 1] - a.lev_off[sid] - 1;
    const int tid = threadIdx.x;
    // forward: L w = r, levels ascending
    TriRow cur = nl > 0 ? fetch_tri_row(true, lp[0] + tid, lp[1], a.lev_rows, a.l_ptr, a.l_idx, a.l_val, a.r) : TriRow{};
    for (int l = 0; l < nl; ++l) {
        TriRow nxt;
        if (l + 1 < nl) nxt = fetch_tri_row(true, lp[l + 1] + tid, lp[l + 2], a.lev_rows, a.l_ptr, a.l_idx, a.l_val, a.r);
        solve_tri_row(cur, a.l_idx, a.l_val, a.w);
        for (int q = lp[l] + NT + tid; q < lp[l + 1]; q += NT)
            solve_tri_row(fetch_tri_row(true, q, lp[l + 1], a.lev_rows, a.l_ptr, a.l_idx, a.l_val, a.r), a.l_idx,
                          a.l_val, a.w);
        __syncthreads();
        cur = nxt;
    }
    // backward: L^T z = w, levels descending
    cur = nl > 0 ? fetch_tri_row(false, lp[nl - 1] + tid, lp[nl], a.lev_rows, a.lt_ptr, a.lt_idx, a.lt_val, a.w)
                 : TriRow{};
    for (int l = nl - 1; l >= 0; --l) {
        TriRow nxt;
        // the right-hand side of a row is w[i], final since the forward sweep ended
        if (l > 0) nxt = fetch_tri_row(false, lp[l - 1] + tid, lp[l], a.lev_rows, a.lt_ptr, a.lt_idx, a.lt_val, a.w);
        solve_tri_row(cur, a.lt_idx, a.lt_val, a.z);
        for (int q = lp[l] + NT + tid; q < lp[l + 1]; q += NT)
            solve_tri_row(fetch_tri_row(false, q, lp[l + 1], a.lev_rows, a.lt_ptr, a.lt_idx, a.lt_val, a.w), a.lt_idx,
                          a.lt_val, a.z);
        __syncthreads();
        cur = nxt;
    }
}

// Kind 5: the system's lower diagonals of M for the block's rows into shared memory (BF16).
template <int NT>
__device__ __forceinline__ void dia_load(const CgArgs& a, const Vecs& v, const DiaSys& ds) {
    __nv_bfloat16* md = const_cast<__nv_bfloat16*>(v.md);
    for (int d = 0; d < ds.nd; ++d)
        for (int i = ds.lo + threadIdx.x; i < ds.hi; i += NT)
            md[d * v.cap + (i - ds.lo)] = a.dia_val[(size_t)d * a.n + i];
}

// Kind 5: zs = scale * M xs on the block's rows (accumulate: zs += ...), M symmetric from its
// lower diagonals at distances o_d (o_0 = 0): with M_d[i] = M_{i, i - o_d},
//   (M x)_i = M_0[i] x_i + sum_{d >= 1} M_d[i] x_{i - o_d} + sum_{d >= 1} M_d[i + o_d] x_{i + o_d},
// summed in that order.  xs is complete over the whole cluster (a cluster barrier since it
// was written); xs, zs and M's rows are this block's shared memory (row i at [i - lo]).  A
// row whose reach [i - H, i + H] lies in the block reads only its own shared memory; the
// other rows read x (and M's rows below them) of the adjacent blocks through distributed
// shared memory (H <= chunk).  One pass, no barrier.
// FUSED (the iteration's step, xs = q, scale = -alpha): the pass also takes x_p += alpha p
// (xp, po) and r -= alpha q on the row, and adds <r, z> and <r, r> of the updated row to dots.
template <int NT, int NM, bool FUSED>
__device__ __forceinline__ void mdia_apply_nm(cg::cluster_group& cl, unsigned rank, const float* xs, float* zs,
                                              const __nv_bfloat16* md, int cap, int o1, int o2, int o3, int H, int R0,
                                              int R1, int lo, int hi, int chunk, float scale, bool accumulate,
                                              float* xp, const float* po, float* rs, DF (&dots)[2]) {
    const int od[4] = {0, o1, o2, o3};
    const float* xnext = hi < R1 ? cl.map_shared_rank(xs, rank + 1) : nullptr;
    const float* xprev = lo > R0 ? cl.map_shared_rank(xs, rank - 1) : nullptr;
    const __nv_bfloat16* mnext = hi < R1 ? cl.map_shared_rank(md, rank + 1) : nullptr;
    const int lo_prev = lo - chunk;
    if constexpr (FUSED) {
        // x_p += alpha p on the thread's rows: x_p lives in global memory, so its loads are all
        // issued at once (scale = -alpha)
#pragma unroll
        for (int k = 0; k < CG_SMEM_ROWS_PER_THREAD; ++k) {
            const int r = (int)threadIdx.x + k * NT;
            if (lo + r < hi) xp[r] = fmaf(-scale, po[r], xp[r]);
        }
    }
    for (int i = lo + threadIdx.x; i < hi; i += NT) {
        const int r = i - lo;
        if constexpr (FUSED) rs[r] = fmaf(scale, xs[r], rs[r]);  // r -= alpha q
        float t = __bfloat162float(md[r]) * xs[r];
        if (i - H >= lo && i + H < hi) {
#pragma unroll
            for (int d = 1; d < NM; ++d) t = fmaf(__bfloat162float(md[d * cap + r]), xs[r - od[d]], t);
#pragma unroll
            for (int d = 1; d < NM; ++d) t = fmaf(__bfloat162float(md[d * cap + r + od[d]]), xs[r + od[d]], t);
        } else {
#pragma unroll
            for (int d = 1; d < NM; ++d) {
                const int j = i - od[d];
                if (j >= R0) t = fmaf(__bfloat162float(md[d * cap + r]), j >= lo ? xs[j - lo] : xprev[j - lo_prev], t);
            }
#pragma unroll
            for (int d = 1; d < NM; ++d) {
                const int j = i + od[d];
                if (j < R1) {
                    const bool own = j < hi;
                    const float mv = __bfloat162float(own ? md[d * cap + (j - lo)] : mnext[d * cap + (j - hi)]);
                    t = fmaf(mv, own ? xs[j - lo] : xnext[j - hi], t);
                }
            }
        }
        const float zr = accumulate ? fmaf(scale, t, zs[r]) : scale * t;
        zs[r] = zr;
        if constexpr (FUSED) {
            const float rr = rs[r];
            df_add_prod(dots[0], rr, zr);
            df_add_prod(dots[1], rr, rr);
        }
    }
}

template <int NT, bool FUSED>
__device__ __forceinline__ void mdia_apply(cg::cluster_group& cl, unsigned rank, const DiaSys& ds, const float* xs,
                                           float* zs, const __nv_bfloat16* md, int cap, float scale, bool accumulate,
                                           float* xp, const float* po, float* rs, DF (&dots)[2]) {
    const int o1 = ds.off[1], o2 = ds.off[2], o3 = ds.off[3];
    const int H = ds.H, R0 = ds.R0, R1 = ds.R1, lo = ds.lo, hi = ds.hi, chunk = ds.chunk;
#define SPX_MDIA(NMv)                                                                                          \
    mdia_apply_nm<NT, NMv, FUSED>(cl, rank, xs, zs, md, cap, o1, o2, o3, H, R0, R1, lo, hi, chunk, scale,     \
                                  accumulate, xp, po, rs, dots)
    switch (ds.nd) {
        case 4: SPX_MDIA(4); break;
        case 3: SPX_MDIA(3); break;
        case 2: SPX_MDIA(2); break;
        default: SPX_MDIA(1); break;
    }
#undef SPX_MDIA
}

template <int NT, int PC>
__device__ void apply_pc(const CgArgs& a, const Vecs& v, cg::cluster_group& cl, int lo, int hi, unsigned rank,
                         int sid) {
    if constexpr (PC == 4) {
        cl.sync();                                               // r complete
        ic0_apply<NT>(a, rank, sid);
        cl.sync();                                               // z complete
    } else if constexpr (PC == 3) {
        cl.sync();                                               // r complete
#pragma unroll 2
        for (int i = lo + threadIdx.x; i < hi; i += NT)
            v.z[i - v.off] = spmv_row(a.l_ptr, a.l_idx, a.l_val, a.r, i);      // z = M r
    } else if constexpr (PC == 2) {
        cl.sync();                                               // r complete
#pragma unroll 2
        for (int i = lo + threadIdx.x; i < hi; i += NT)
            a.w[i] = spmv_row(a.lt_ptr, a.lt_idx, a.lt_val, a.r, i);   // w = L^T r
        cl.sync();                                               // w complete
#pragma unroll 2
        for (int i = lo + threadIdx.x; i < hi; i += NT)
            a.z[i] = spmv_row(a.l_ptr, a.l_idx, a.l_val, a.w, i);      // z = L w
    } else {
        apply_pc_local<NT, PC>(v, lo, hi);
    }
}

// r = b - A x in FP64 on [lo, hi); returns the thread's partial of ||r||^2 in FP64.
template <int NT>
__device__ __forceinline__ double true_residual(const CgArgs& a, const Vecs& v, int lo, int hi) {
    double s = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += NT) {
        double t = (double)a.b[i];
        for (int e = a.a_ptr[i]; e < a.a_ptr[i + 1]; ++e) t -= (double)a.a_val[e] * a.x[a.a_idx[e]];
        v.r[i - v.off] = (float)t;
        s += t * t;
    }
    return s;
}

// The vectors of one system for a block (shared memory when SM, else the workspace).
template <int NT, int PC, bool SM>
__device__ __forceinline__ Vecs make_vecs(const CgArgs& a, float* sv, int lo, int hi) {
    constexpr int cap = CG_SMEM_ROWS_PER_THREAD * NT;
    if constexpr (PC == 5) {
        // [q | z | r | po] (cap floats each), then M's BF16 diagonals (cap each)
        Vecs v{a.xp + lo, sv, sv + cap, sv + 2 * cap, nullptr, sv + 3 * cap, lo, true};
        v.md = reinterpret_cast<const __nv_bfloat16*>(sv + CG_DIA_VECTORS * cap);
        v.cap = cap;
        return v;
    } else if constexpr (SM) {
        if constexpr (PC == 1)
            for (int i = lo + threadIdx.x; i < hi; i += NT) sv[4 * cap + i - lo] = a.dinv[i];
        // element i of every view is at [i - lo]: the global r (gathered by M r) is shifted to match
        return Vecs{sv, sv + cap, sv + 2 * cap, PC <= 1 ? sv + 3 * cap : a.r + lo,
                    PC <= 1 ? sv + 4 * cap : nullptr, sv + 5 * cap, lo, true};
    } else {
        return Vecs{a.xp, a.q, a.z, a.r, a.dinv, a.p, 0, false};
    }
}

// PCG on rows [lo, hi) of system sid by this block (its cluster runs the other rows).
template <int NT, int PC, bool SM>
__device__ __forceinline__ void pcg_system(const CgArgs& a, cg::cluster_group& cl, unsigned rank, int sid, int lo,
                                           int hi, float* sv, float2 (&red)[CG_MAX_WARPS][4], float2 (&part)[2][4],
                                           CgBcast& bc, CgScal& sc, int& slot, const DiaSys& ds) {
    const bool t0 = threadIdx.x == 0;
    const Vecs v = make_vecs<NT, PC, SM>(a, sv, lo, hi);
    if constexpr (PC == 5) dia_load<NT>(a, v, ds);
    // z = M r applied directly (at the start and after a reliable update)
    auto precondition = [&]() {
        if constexpr (PC == 5) {
            cl.sync();                                           // r (and L's rows) complete
            DF unused[2] = {{0.f, 0.f}, {0.f, 0.f}};
            mdia_apply<NT, false>(cl, rank, ds, v.r, v.z, v.md, v.cap, 1.f, false, nullptr, nullptr, nullptr, unused);
        } else {
            apply_pc<NT, PC>(a, v, cl, lo, hi, rank, sid);
        }
    };
    // thread 0 of each block keeps the FP64 scalars; every block computes the same ones
    double& bnorm = sc.bnorm;
    double& rz = sc.rz;
    double& ref = sc.ref;
    double& last_true = sc.last_true;
    int& status = sc.status;
    if (t0) {
        bnorm = 0.0;
        rz = 0.0;
        ref = 0.0;
        last_true = 1.0;
        status = SPX_MAXITER;
    }

    // ---- x = 0, r = b, z = M r, p = z
    DF v2[2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (int i = lo + threadIdx.x; i < hi; i += NT) {
        const float bi = a.b[i];
        a.x[i] = 0.0;
        v.xp[i - v.off] = 0.f;
        v.r[i - v.off] = bi;
        df_add_prod(v2[0], bi, bi);
    }
    precondition();
    for (int i = lo + threadIdx.x; i < hi; i += NT) {
        const float zi = v.z[i - v.off];
        a.p[i] = zi;
        if (v.sm) v.po[i - v.off] = zi;
        df_add_prod(v2[1], v.r[i - v.off], zi);
    }
    {
        double o2[2];
        cluster_sum<NT, 2>(cl, v2, o2, red, part, slot);
        if (t0) {
            bnorm = sqrt(o2[0]);
            rz = o2[1];
            ref = bnorm;
            int act = ACT_GO;
            if (bnorm == 0.0) {
                status = SPX_OK;
                last_true = 0.0;
                act = ACT_STOP;
            } else if (!isfinite(rz) || !isfinite(bnorm)) {
                status = SPX_NONFINITE;
                act = ACT_STOP;
            } else if (!(rz > 0.0)) {
                status = SPX_BREAKDOWN;
                act = ACT_STOP;
            }
            bc.action = act;
        }
        __syncthreads();
    }
    int it = 0;
    bool dirty = false;                 // xp holds an unfolded part
    if (bc.action == ACT_GO) {
        while (it < a.maxit) {
            cl.sync();                                      // p complete (and bc read by all)
            {
                DF v1[1] = {{0.f, 0.f}};
                const float* __restrict__ Pv = a.p;
                for (int i = lo + threadIdx.x; i < hi; i += 2 * NT) {
                    const int i1 = i + NT;
                    const bool has1 = i1 < hi;
                    float q0, q1;
                    spmv_row2<CG_ROW2_W>(a.a_ptr, a.a_idx, a.a_val, Pv, i, i1, has1, q0, q1);
                    v.q[i - v.off] = q0;
                    df_add_prod(v1[0], v.po[i - v.off], q0);
                    if (has1) {
                        v.q[i1 - v.off] = q1;
                        df_add_prod(v1[0], v.po[i1 - v.off], q1);
                    }
                }
                double o1[1];
                cluster_sum<NT, 1>(cl, v1, o1, red, part, slot);
                if (t0) {
                    const double pq = o1[0];
                    int act = ACT_GO;
                    if (!isfinite(pq)) {
                        status = SPX_NONFINITE;
                        act = ACT_STOP;
                    } else if (!(pq > 0.0)) {
                        status = SPX_BREAKDOWN;
                        act = ACT_STOP;
                    } else {
                        bc.alpha = (float)(rz / pq);
                    }
                    bc.action = act;
                }
                __syncthreads();
            }
            if (bc.action == ACT_STOP) break;
            const float alpha = bc.alpha;
            dirty = true;
            ++it;
            DF v2n[2] = {{0.f, 0.f}, {0.f, 0.f}};
            if constexpr (PC <= 1) {
                // x_p += alpha p; r -= alpha q; z = M r (local); <r, z>, <r, r> -- one pass
                float* __restrict__ XP = v.xp - v.off;
                float* __restrict__ R = v.r - v.off;
                float* __restrict__ Z = v.z - v.off;
                const float* __restrict__ Pv = v.po - v.off;
                const float* __restrict__ Qv = v.q - v.off;
                const float* __restrict__ DI = v.di - v.off;
#pragma unroll 2
                for (int i = lo + threadIdx.x; i < hi; i += NT) {
                    XP[i] = fmaf(alpha, Pv[i], XP[i]);
                    const float ri = fmaf(-alpha, Qv[i], R[i]);
                    R[i] = ri;
                    const float zi = PC == 1 ? DI[i] * ri : ri;
                    Z[i] = zi;
                    df_add_prod(v2n[0], ri, zi);
                    df_add_prod(v2n[1], ri, ri);
                }
            } else if constexpr (PC == 3) {
                // explicit M: update, barrier, then z = M r with the dots in the same pass
                float* __restrict__ XP = v.xp - v.off;
                float* __restrict__ R = a.r;
                const float* __restrict__ Pv = v.po - v.off;
                const float* __restrict__ Qv = v.q - v.off;
#pragma unroll 2
                for (int i = lo + threadIdx.x; i < hi; i += NT) {
                    XP[i] = fmaf(alpha, Pv[i], XP[i]);
                    R[i] = fmaf(-alpha, Qv[i], R[i]);
                }
                cl.sync();                                  // r complete
                const float* __restrict__ Rc = a.r;
                float* __restrict__ Z = v.z - v.off;
#pragma unroll 2
                for (int i = lo + threadIdx.x; i < hi; i += NT) {
                    const float zi = spmv_row(a.l_ptr, a.l_idx, a.l_val, Rc, i);
                    Z[i] = zi;
                    const float ri = Rc[i];
                    df_add_prod(v2n[0], ri, zi);
                    df_add_prod(v2n[1], ri, ri);
                }
            } else if constexpr (PC == 5) {
                // x_p += alpha p; r -= alpha q; z -= alpha M q, with <r, z> and <r, r>: q = A p is
                // complete over the cluster since the reduction above, so M q needs no barrier
                mdia_apply<NT, true>(cl, rank, ds, v.q, v.z, v.md, v.cap, -alpha, true, v.xp, v.po, v.r, v2n);
            } else {
                float* __restrict__ XP = v.xp - v.off;
                float* __restrict__ R = v.r - v.off;
                const float* __restrict__ Pv = v.po - v.off;
                const float* __restrict__ Qv = v.q - v.off;
#pragma unroll 2
                for (int i = lo + threadIdx.x; i < hi; i += NT) {
                    XP[i] = fmaf(alpha, Pv[i], XP[i]);
                    R[i] = fmaf(-alpha, Qv[i], R[i]);
                }
                apply_pc<NT, PC>(a, v, cl, lo, hi, rank, sid);
                const float* __restrict__ Rc = v.r - v.off;
                const float* __restrict__ Zc = v.z - v.off;
#pragma unroll 2
                for (int i = lo + threadIdx.x; i < hi; i += NT) {
                    const float ri = Rc[i];
                    df_add_prod(v2n[0], ri, Zc[i]);
                    df_add_prod(v2n[1], ri, ri);
                }
            }
            double rz_new = 0.0;
            {
                double o2[2];
                cluster_sum<NT, 2>(cl, v2n, o2, red, part, slot);
                if (t0) {
                    rz_new = o2[0];
                    const double rnorm = sqrt(o2[1]);
                    int act = ACT_GO;
                    if (!isfinite(rz_new) || !isfinite(rnorm)) {
                        status = SPX_NONFINITE;
                        act = ACT_STOP;
                    } else if (rnorm <= a.delta * ref || rnorm <= a.tol * bnorm) {
                        act = ACT_FOLD;
                    } else if (!(rz_new > 0.0)) {
                        status = SPX_BREAKDOWN;
                        act = ACT_STOP;
                    } else {
                        bc.beta = (float)(rz_new / rz);
                        rz = rz_new;
                    }
                    bc.action = act;
                }
                __syncthreads();
            }
            if (bc.action == ACT_STOP) break;
            if (bc.action == ACT_FOLD) {
                // ---- reliable update: fold xp into x (FP64), true residual in FP64
                for (int i = lo + threadIdx.x; i < hi; i += NT) {
                    a.x[i] += (double)v.xp[i - v.off];
                    v.xp[i - v.off] = 0.f;
                }
                dirty = false;
                cl.sync();                                  // x complete
                {
                    DF v64[1] = {df_of(true_residual<NT>(a, v, lo, hi))};
                    double o1[1];
                    cluster_sum<NT, 1>(cl, v64, o1, red, part, slot);
                    if (t0) {
                        const double tn = sqrt(o1[0]);
                        last_true = tn / bnorm;
                        ref = tn;
                        int act = ACT_GO;
                        if (!isfinite(tn)) {
                            status = SPX_NONFINITE;
                            act = ACT_STOP;
                        } else if (tn <= a.tol * bnorm) {
                            status = SPX_OK;
                            act = ACT_STOP;
                        }
                        bc.action = act;
                    }
                    __syncthreads();
                }
                if (bc.action == ACT_STOP) break;
                precondition();
                DF vz[1] = {{0.f, 0.f}};
                for (int i = lo + threadIdx.x; i < hi; i += NT) df_add_prod(vz[0], v.r[i - v.off], v.z[i - v.off]);
                double o1[1];
                cluster_sum<NT, 1>(cl, vz, o1, red, part, slot);
                if (t0) {
                    rz_new = o1[0];
                    int act = ACT_GO;
                    if (!(rz_new > 0.0)) {
                        status = SPX_BREAKDOWN;
                        act = ACT_STOP;
                    } else {
                        bc.beta = (float)(rz_new / rz);
                        rz = rz_new;
                    }
                    bc.action = act;
                }
                __syncthreads();
                if (bc.action == ACT_STOP) break;
            }
            const float beta = bc.beta;
            if (v.sm) {
                float* __restrict__ Pg = a.p;
                float* __restrict__ PO = v.po - v.off;
                const float* __restrict__ Zc = v.z - v.off;
#pragma unroll 4
                for (int i = lo + threadIdx.x; i < hi; i += NT) {
                    const float pi = fmaf(beta, PO[i], Zc[i]);
                    PO[i] = pi;
                    Pg[i] = pi;
                }
            } else {
                float* __restrict__ Pv = a.p;
                const float* __restrict__ Zc = a.z;
#pragma unroll 4
                for (int i = lo + threadIdx.x; i < hi; i += NT) Pv[i] = fmaf(beta, Pv[i], Zc[i]);
            }
        }
    }
    if (dirty) {
        // fold the remainder and report the true residual of the returned x
        for (int i = lo + threadIdx.x; i < hi; i += NT) {
            a.x[i] += (double)v.xp[i - v.off];
            v.xp[i - v.off] = 0.f;
        }
        cl.sync();
        DF v64[1] = {df_of(true_residual<NT>(a, v, lo, hi))};
        double o1[1];
        cluster_sum<NT, 1>(cl, v64, o1, red, part, slot);
        if (t0) last_true = bnorm > 0.0 ? sqrt(o1[0]) / bnorm : 0.0;
    }
    if (rank == 0 && t0) {
        a.iters[sid] = it;
        a.status[sid] = status;
        a.relres[sid] = last_true;
    }
}

// Registers capped at 64 (1024 / NT blocks per SM): the launch sizes its grid for that many
// resident blocks.  A system whose rows per block fit CG_SMEM_ROWS_PER_THREAD x NT keeps
// the block's private vectors in shared memory (dynamic, 6 x that many floats).
template <int NT, int PC>
__global__ void __launch_bounds__(NT, 1024 / NT) pcg_kernel(CgArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const unsigned rank = cl.block_rank();
    const unsigned ncl = cl.num_blocks();
    __shared__ float2 red[CG_MAX_WARPS][4];
    __shared__ float2 part[2][4];
    __shared__ int sys_sh;
    __shared__ CgBcast bc;
    __shared__ CgScal sc;
    extern __shared__ float sv[];
    int slot = 0;
    const bool t0 = threadIdx.x == 0;

    for (;;) {
        if (rank == 0 && t0) sys_sh = atomicAdd(a.queue, 1);
        cl.sync();
        const int s = *cl.map_shared_rank(&sys_sh, 0);
        cl.sync();
        if (s >= a.nsys) break;
        const int sid = a.order ? a.order[s] : s;
        const int R0 = a.sys_ptr[sid], R1 = a.sys_ptr[sid + 1];
        const int chunk = (R1 - R0 + (int)ncl - 1) / (int)ncl;
        const int lo = min(R1, R0 + (int)rank * chunk), hi = min(R1, lo + chunk);
        bool in_smem = false;
        if constexpr (PC == 0 || PC == 1 || PC == 3 || PC == 5)
            in_smem = a.smem_rows >= CG_SMEM_ROWS_PER_THREAD * NT && chunk <= CG_SMEM_ROWS_PER_THREAD * NT;
        __shared__ DiaSys ds;                                   // block-uniform: kept out of registers
        if constexpr (PC == 5) {
            if (t0) {
                ds.nd = a.dia_nd[sid];
                ds.H = 0;
                bool offs_ok = true;
                for (int d = 0; d < CG_MDIA_MAX; ++d) {
                    ds.off[d] = d < ds.nd ? a.dia_off[sid * CG_MDIA_MAX + d] : 0;
                    if (d < ds.nd && ds.off[d] > ds.H) ds.H = ds.off[d];
                    if (d < ds.nd && (ds.off[d] < 0 || (d == 0) != (ds.off[d] == 0))) offs_ok = false;
                }
                ds.R0 = R0;
                ds.R1 = R1;
                ds.lo = lo;
                ds.hi = hi;
                ds.chunk = chunk;
                // the block holds its rows in shared memory and reaches only the adjacent blocks
                ds.ok = in_smem && offs_ok && ds.nd >= 1 && ds.nd <= CG_MDIA_MAX && (ds.H <= chunk || (int)ncl == 1);
            }
            __syncthreads();
            if (!ds.ok) {                                       // uniform across the cluster
                if (rank == 0 && t0) {
                    a.iters[sid] = 0;
                    a.status[sid] = SPX_NOT_SUPPORTED;
                    a.relres[sid] = -1.0;
                }
                cl.sync();
                continue;
            }
        }
        if (in_smem)                                            // uniform across the cluster
            pcg_system<NT, PC, true>(a, cl, rank, sid, lo, hi, sv, red, part, bc, sc, slot, ds);
        else
            pcg_system<NT, PC, false>(a, cl, rank, sid, lo, hi, sv, red, part, bc, sc, slot, ds);
        cl.sync();                                              // finish before the next system
    }
}

__global__ void diag_inverse_kernel(int32_t m, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                    const float* __restrict__ val, float* __restrict__ dinv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    float d = 0.f;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e)
        if (idx[e] == i) d = val[e];
    dinv[i] = d != 0.f ? 1.f / d : 0.f;
}

__global__ void masked_outer_f64_kernel(int32_t m, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                        const double* __restrict__ u, const double* __restrict__ v, double scale,
                                        float* __restrict__ out) {
    // one warp per row
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= m) return;
    const double ui = scale * u[row];
    for (int e = ptr[row] + lane; e < ptr[row + 1]; e += 32) out[e] = (float)(ui * v[idx[e]]);
}

// Diagonal form of a lower-triangular factor, per system: the distinct offsets j - i of its
// stored entries (at most CG_DIA_MAX, all <= 0), ascending in |offset|; nd = -1 when a system
// has more, or an entry above the diagonal.  One block per system; the set is the same
// whatever order the threads insert it in, and it is sorted at the end (deterministic).
__global__ void dia_analyse_kernel(int32_t nsys, const int32_t* __restrict__ sys_ptr,
                                   const int32_t* __restrict__ l_ptr, const int32_t* __restrict__ l_idx,
                                   int32_t* __restrict__ offs, int32_t* __restrict__ nd) {
    constexpr int SLOTS = CG_DIA_MAX + 1;
    __shared__ int tab[SLOTS];
    __shared__ int bad;
    const int sid = blockIdx.x;
    if (sid >= nsys) return;
    if (threadIdx.x < SLOTS) tab[threadIdx.x] = INT_MIN;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int i = sys_ptr[sid] + threadIdx.x; i < sys_ptr[sid + 1]; i += blockDim.x) {
        for (int e = l_ptr[i]; e < l_ptr[i + 1]; ++e) {
            const int off = l_idx[e] - i;
            if (off > 0) {
                bad = 1;
                continue;
            }
            int k = 0;
            for (; k < SLOTS; ++k) {
                const int cur = atomicCAS(&tab[k], INT_MIN, off);
                if (cur == INT_MIN || cur == off) break;
            }
            if (k == SLOTS) bad = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int o[SLOTS], c = 0;
        for (int k = 0; k < SLOTS; ++k)
            if (tab[k] != INT_MIN) o[c++] = tab[k];
        for (int x = 1; x < c; ++x)              // insertion sort, descending offset (ascending |offset|)
            for (int y = x; y > 0 && o[y] > o[y - 1]; --y) {
                const int t = o[y];
                o[y] = o[y - 1];
                o[y - 1] = t;
            }
        const bool ok = !bad && c <= CG_DIA_MAX;
        nd[sid] = ok ? c : -1;
        for (int d = 0; d < CG_DIA_MAX; ++d) offs[sid * CG_DIA_MAX + d] = ok && d < c ? o[d] : 0;
    }
}

// values[d * n + i] = L_{i, i + off_d} rounded to BF16 (zeros, written beforehand, elsewhere);
// one thread per row, its system by binary search in sys_ptr.
__global__ void dia_fill_kernel(int32_t n, int32_t nsys, const int32_t* __restrict__ sys_ptr,
                                const int32_t* __restrict__ l_ptr, const int32_t* __restrict__ l_idx,
                                const float* __restrict__ l_val, const int32_t* __restrict__ offs,
                                const int32_t* __restrict__ nd, __nv_bfloat16* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nsys;                       // the system s with sys_ptr[s] <= i < sys_ptr[s + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sys_ptr[mid] <= i) lo = mid;
        else hi = mid;
    }
    const int c = nd[lo];
    for (int e = l_ptr[i]; e < l_ptr[i + 1]; ++e) {
        const int off = l_idx[e] - (int)i;
        for (int d = 0; d < c; ++d)
            if (offs[lo * CG_DIA_MAX + d] == off) out[(int64_t)d * n + i] = __float2bfloat16(l_val[e]);
    }
}

// M = L L^T by its lower diagonals.  With L's diagonals at distances s_d = -off_d (values
// L_d[i] = L_{i, i - s_d}), M_{i, i - o} = sum over pairs (d, e) with s_d - s_e = o of
// L_d[i] L_e[i - o] (the common column is k = i - s_d = (i - o) - s_e).  The distances are 0
// and every positive s_d - s_e, ascending: at most CG_MDIA_MAX for CG_DIA_MAX diagonals.
// One thread per system.
__global__ void dia_square_offsets_kernel(int32_t nsys, const int32_t* __restrict__ l_offs,
                                          const int32_t* __restrict__ l_nd, int32_t* __restrict__ m_offs,
                                          int32_t* __restrict__ m_nd) {
    const int sid = blockIdx.x * blockDim.x + threadIdx.x;
    if (sid >= nsys) return;
    const int c = l_nd[sid];
    int o[CG_MDIA_MAX], cnt = 0;
    if (c >= 1 && c <= CG_DIA_MAX) {
        o[cnt++] = 0;
        for (int d = 0; d < c; ++d)
            for (int e = 0; e < c; ++e) {
                const int dist = l_offs[sid * CG_DIA_MAX + e] - l_offs[sid * CG_DIA_MAX + d];   // s_d - s_e
                if (dist <= 0) continue;
                bool seen = false;
                for (int q = 0; q < cnt; ++q) seen = seen || o[q] == dist;
                if (!seen && cnt < CG_MDIA_MAX) o[cnt++] = dist;
            }
        for (int x = 1; x < cnt; ++x)                // insertion sort, ascending
            for (int y = x; y > 0 && o[y] < o[y - 1]; --y) {
                const int t = o[y];
                o[y] = o[y - 1];
                o[y - 1] = t;
            }
    }
    m_nd[sid] = cnt > 0 ? cnt : -1;
    for (int q = 0; q < CG_MDIA_MAX; ++q) m_offs[sid * CG_MDIA_MAX + q] = q < cnt ? o[q] : 0;
}

// values of M's diagonals, one thread per row: FP32 sums of the exact products of L's BF16
// values in (d, e) order, rounded to BF16; zero where row i - o is outside the system.
__global__ void dia_square_kernel(int32_t n, int32_t nsys, const int32_t* __restrict__ sys_ptr,
                                  const int32_t* __restrict__ l_offs, const int32_t* __restrict__ l_nd,
                                  const __nv_bfloat16* __restrict__ l_val, const int32_t* __restrict__ m_offs,
                                  const int32_t* __restrict__ m_nd, __nv_bfloat16* __restrict__ m_val) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nsys;                       // the system s with sys_ptr[s] <= i < sys_ptr[s + 1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sys_ptr[mid] <= i) lo = mid;
        else hi = mid;
    }
    const int c = l_nd[lo], cm = m_nd[lo];
    const int64_t R0 = sys_ptr[lo];
    for (int q = 0; q < CG_MDIA_MAX; ++q) {
        float t = 0.f;
        if (q < cm && c >= 1) {
            const int o = m_offs[lo * CG_MDIA_MAX + q];
            if (i - o >= R0)
                for (int d = 0; d < c; ++d)
                    for (int e = 0; e < c; ++e)
                        if (l_offs[lo * CG_DIA_MAX + e] - l_offs[lo * CG_DIA_MAX + d] == o)
                            t = fmaf(__bfloat162float(l_val[(int64_t)d * n + i]),
                                     __bfloat162float(l_val[(int64_t)e * n + (i - o)]), t);
        }
        m_val[(int64_t)q * n + i] = __float2bfloat16(t);
    }
}

// Launch shape of the batched PCG (threads per block, blocks per cluster); 0 = default.
std::atomic<int> g_cg_threads{0};
std::atomic<int> g_cg_cluster{0};
std::atomic<int> g_cg_max_clusters{0};
std::atomic<int> g_cg_smem_vectors{1};


}  // namespace
}  // namespace spx

using namespace spx;

// The persistent launch of the batched PCG for preconditioner kind pc_kind (CgArgs filled).
static spx_status launch_pcg(CgArgs& a, int pc_kind, cudaStream_t st) {
    SPX_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(int32_t), st), "spx_cg_batched memset");

    const int nt = g_cg_threads.load() > 0 ? g_cg_threads.load() : 512;
    const int cl = g_cg_cluster.load() > 0 ? g_cg_cluster.load() : 8;
    const int blocks_per_sm = nt >= 1024 ? 1 : 1024 / nt;      // 64 registers per thread
    int clusters = blocks_per_sm * num_sms() / cl;
    const int maxc = g_cg_max_clusters.load();
    if (maxc > 0 && clusters > maxc) clusters = maxc;
    if (clusters < 1) clusters = 1;
    if (clusters > a.nsys) clusters = a.nsys;
    const bool smem_vecs = pc_kind == 5 ||
                           (g_cg_smem_vectors.load() != 0 && (pc_kind == 0 || pc_kind == 1 || pc_kind == 3));
    a.smem_rows = smem_vecs ? CG_SMEM_ROWS_PER_THREAD * nt : 0;
    const size_t smem = pc_kind == 5
        ? (size_t)a.smem_rows * (CG_DIA_VECTORS * sizeof(float) + CG_MDIA_MAX * sizeof(__nv_bfloat16))
        : (size_t)a.smem_rows * CG_SMEM_VECTORS * sizeof(float);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(clusters * cl));
    cfg.blockDim = dim3(nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto launch = [&](auto kern) -> spx_status {
        if (cl > 8)   // 16 blocks per cluster is beyond the portable size: opt in
            SPX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                     "spx_cg_batched cluster attribute");
        if (smem > 0)
            SPX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                     "spx_cg_batched shared memory attribute");
        SPX_CUDA(cudaLaunchKernelEx(&cfg, kern, a), "spx_cg_batched launch");
        return SPX_OK;
    };
    auto by_pc = [&](auto k0, auto k1, auto k2, auto k3, auto k4, auto k5) -> spx_status {
        switch (pc_kind) {
            case 0: return launch(k0);
            case 1: return launch(k1);
            case 2: return launch(k2);
            case 3: return launch(k3);
            case 4: return launch(k4);
            default: return launch(k5);
        }
    };
    if (nt == 256)
        return by_pc(pcg_kernel<256, 0>, pcg_kernel<256, 1>, pcg_kernel<256, 2>, pcg_kernel<256, 3>, pcg_kernel<256, 4>,
                     pcg_kernel<256, 5>);
    if (nt == 1024)
        return by_pc(pcg_kernel<1024, 0>, pcg_kernel<1024, 1>, pcg_kernel<1024, 2>, pcg_kernel<1024, 3>,
                     pcg_kernel<1024, 4>, pcg_kernel<1024, 5>);
    return by_pc(pcg_kernel<512, 0>, pcg_kernel<512, 1>, pcg_kernel<512, 2>, pcg_kernel<512, 3>, pcg_kernel<512, 4>,
                 pcg_kernel<512, 5>);
}

extern "C" spx_status spx_cg_workspace_size(int32_t n, size_t* bytes) {
    if (!bytes || n < 0) return set_error(SPX_INVALID_ARG, "spx_cg_workspace_size: bad arguments");
    const size_t v = ((size_t)n * 4 + 255) & ~size_t(255);
    *bytes = 6 * v + 256;
    return SPX_OK;
}

extern "C" spx_status spx_cg_batched(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys, const int32_t* order,
                                     const float* b, double* x, int32_t pc_kind, const float* pc_diag_inv,
                                     const spx_csr* L, const spx_csr* LT, const int32_t* const* ic0_levels,
                                     double tol, int32_t maxit, double delta, int32_t* iters, int32_t* status,
                                     double* relres, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_cg_batched"));
    if (A->m != A->n) return set_error(SPX_INVALID_ARG, "spx_cg_batched: A must be square");
    if (nsys < 0 || (nsys > 0 && (!sys_ptr || !b || !x || !iters || !status || !relres)))
        return set_error(SPX_INVALID_ARG, "spx_cg_batched: NULL argument");
    if (pc_kind < 0 || pc_kind > 4) return set_error(SPX_INVALID_ARG, "spx_cg_batched: unknown preconditioner");
    if (pc_kind == 4 && (!ic0_levels || !ic0_levels[0] || !ic0_levels[1] || !ic0_levels[2]))
        return set_error(SPX_INVALID_ARG, "spx_cg_batched: IC(0) needs its level schedule");
    if (pc_kind == 1 && !pc_diag_inv) return set_error(SPX_INVALID_ARG, "spx_cg_batched: Jacobi needs D^-1");
    if (pc_kind == 3) {
        SPX_TRY(check_csr(L, true, "spx_cg_batched (M)"));
        if (L->m != A->m) return set_error(SPX_INVALID_ARG, "spx_cg_batched: M shape");
    }
    if (pc_kind == 2 || pc_kind == 4) {
        SPX_TRY(check_csr(L, true, "spx_cg_batched (L)"));
        SPX_TRY(check_csr(LT, true, "spx_cg_batched (L^T)"));
        if (L->m != A->m || LT->m != A->m) return set_error(SPX_INVALID_ARG, "spx_cg_batched: L shape");
    }
    if (!(tol > 0.0) || maxit < 0 || !(delta > 0.0 && delta < 1.0))
        return set_error(SPX_INVALID_ARG, "spx_cg_batched: tol > 0, maxit >= 0, 0 < delta < 1 required");
    size_t need = 0;
    spx_cg_workspace_size(A->m, &need);
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_cg_batched: workspace %zu < %zu", ws_bytes, need);
    if (nsys == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    const size_t v = ((size_t)A->m * 4 + 255) & ~size_t(255);
    char* w = static_cast<char*>(ws);
    CgArgs a{};
    a.nsys = nsys;
    a.sys_ptr = sys_ptr;
    a.order = order;
    a.a_ptr = A->indptr;
    a.a_idx = A->indices;
    a.a_val = A->values;
    a.b = b;
    a.x = x;
    a.pc = pc_kind;
    a.dinv = pc_diag_inv;
    if (pc_kind == 3) {
        a.l_ptr = L->indptr; a.l_idx = L->indices; a.l_val = L->values;
    }
    if (pc_kind == 2 || pc_kind == 4) {
        a.l_ptr = L->indptr; a.l_idx = L->indices; a.l_val = L->values;
        a.lt_ptr = LT->indptr; a.lt_idx = LT->indices; a.lt_val = LT->values;
    }
    a.r = (float*)(w + 0 * v);
    a.p = (float*)(w + 1 * v);
    a.q = (float*)(w + 2 * v);
    a.z = (float*)(w + 3 * v);
    a.w = (float*)(w + 4 * v);
    a.xp = (float*)(w + 5 * v);
    a.queue = (int32_t*)(w + 6 * v);
    a.tol = tol;
    a.delta = delta;
    a.maxit = maxit;
    a.iters = iters;
    a.status = status;
    a.relres = relres;
    if (pc_kind == 4) {
        a.lev_off = ic0_levels[0];
        a.lev_ptr = ic0_levels[1];
        a.lev_rows = ic0_levels[2];
    }
    return launch_pcg(a, pc_kind, st);
}

extern "C" spx_status spx_diag_inverse(const spx_csr* A, float* dinv, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_diag_inverse"));
    if (A->m > 0 && !dinv) return set_error(SPX_INVALID_ARG, "spx_diag_inverse: NULL output");
    if (A->m == 0) return SPX_OK;
    diag_inverse_kernel<<<(unsigned)((A->m + 255) / 256), 256, 0, as_stream(stream)>>>(A->m, A->indptr, A->indices,
                                                                                       A->values, dinv);
    SPX_CHECK_LAUNCH("spx_diag_inverse");
    return SPX_OK;
}

extern "C" spx_status spx_masked_outer_f64(const spx_csr* A, const double* u, const double* v, double scale, float* out,
                                           void* stream) {
    SPX_TRY(check_csr(A, false, "spx_masked_outer_f64"));
    if (A->nnz > 0 && (!u || !v || !out)) return set_error(SPX_INVALID_ARG, "spx_masked_outer_f64: NULL operand");
    if (A->m == 0) return SPX_OK;
    const int64_t threads = (int64_t)A->m * 32;
    masked_outer_f64_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, as_stream(stream)>>>(
        A->m, A->indptr, A->indices, u, v, scale, out);
    SPX_CHECK_LAUNCH("spx_masked_outer_f64");
    return SPX_OK;
}

extern "C" spx_status spx_cg_set_launch(int32_t threads_per_block, int32_t cluster_size, int32_t max_clusters) {
    if (!(threads_per_block == 0 || threads_per_block == 256 || threads_per_block == 512 ||
          threads_per_block == 1024) ||
        !(cluster_size == 0 || cluster_size == 1 || cluster_size == 2 || cluster_size == 4 || cluster_size == 8 ||
          cluster_size == 16) ||
        max_clusters < 0)
        return set_error(SPX_INVALID_ARG,
                         "spx_cg_set_launch: threads in {256, 512, 1024}, cluster in {1, 2, 4, 8, 16}, "
                         "max_clusters >= 0");
    g_cg_threads.store(threads_per_block);
    g_cg_cluster.store(cluster_size);
    g_cg_max_clusters.store(max_clusters);
    return SPX_OK;
}

extern "C" spx_status spx_cg_set_vector_residency(int32_t shared_memory) {
    if (shared_memory != 0 && shared_memory != 1)
        return set_error(SPX_INVALID_ARG, "spx_cg_set_vector_residency: 0 or 1");
    g_cg_smem_vectors.store(shared_memory);
    return SPX_OK;
}

extern "C" spx_status spx_dia_analyse(const spx_csr* L, const int32_t* sys_ptr, int32_t nsys, int32_t* offsets,
                                      int32_t* nd, int32_t* supported_host, void* stream) {
    SPX_TRY(check_csr(L, false, "spx_dia_analyse"));
    if (nsys < 0 || (nsys > 0 && (!sys_ptr || !offsets || !nd)) || !supported_host)
        return set_error(SPX_INVALID_ARG, "spx_dia_analyse: bad arguments");
    *supported_host = 1;
    if (nsys == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    dia_analyse_kernel<<<(unsigned)nsys, 256, 0, st>>>(nsys, sys_ptr, L->indptr, L->indices, offsets, nd);
    SPX_CHECK_LAUNCH("spx_dia_analyse");
    // a system is unsupported when nd < 0: the minimum over the systems, read back once
    std::vector<int32_t> host((size_t)nsys);
    SPX_CUDA(cudaMemcpyAsync(host.data(), nd, (size_t)nsys * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
             "spx_dia_analyse copy");
    SPX_CUDA(cudaStreamSynchronize(st), "spx_dia_analyse sync");
    for (int32_t k = 0; k < nsys; ++k)
        if (host[(size_t)k] < 1) *supported_host = 0;
    return SPX_OK;
}

extern "C" spx_status spx_dia_fill(const spx_csr* L, const int32_t* sys_ptr, int32_t nsys, const int32_t* offsets,
                                   const int32_t* nd, void* values_bf16, void* stream) {
    SPX_TRY(check_csr(L, true, "spx_dia_fill"));
    if (nsys < 0 || (nsys > 0 && (!sys_ptr || !offsets || !nd || !values_bf16)))
        return set_error(SPX_INVALID_ARG, "spx_dia_fill: bad arguments");
    if (L->m == 0 || nsys == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    SPX_CUDA(cudaMemsetAsync(values_bf16, 0, (size_t)CG_DIA_MAX * L->m * sizeof(__nv_bfloat16), st),
             "spx_dia_fill memset");
    dia_fill_kernel<<<(unsigned)((L->m + 255) / 256), 256, 0, st>>>(L->m, nsys, sys_ptr, L->indptr, L->indices,
                                                                   L->values, offsets, nd,
                                                                   static_cast<__nv_bfloat16*>(values_bf16));
    SPX_CHECK_LAUNCH("spx_dia_fill");
    return SPX_OK;
}

extern "C" spx_status spx_dia_square(const int32_t* sys_ptr, int32_t nsys, int32_t n, const int32_t* l_offsets,
                                     const int32_t* l_nd, const void* l_values_bf16, int32_t* m_offsets,
                                     int32_t* m_nd, void* m_values_bf16, void* stream) {
    if (nsys < 0 || n < 0 ||
        (nsys > 0 && (!sys_ptr || !l_offsets || !l_nd || !l_values_bf16 || !m_offsets || !m_nd || !m_values_bf16)))
        return set_error(SPX_INVALID_ARG, "spx_dia_square: bad arguments");
    if (nsys == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    dia_square_offsets_kernel<<<(unsigned)((nsys + 127) / 128), 128, 0, st>>>(nsys, l_offsets, l_nd, m_offsets, m_nd);
    SPX_CHECK_LAUNCH("spx_dia_square offsets");
    if (n == 0) return SPX_OK;
    dia_square_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        n, nsys, sys_ptr, l_offsets, l_nd, static_cast<const __nv_bfloat16*>(l_values_bf16), m_offsets, m_nd,
        static_cast<__nv_bfloat16*>(m_values_bf16));
    SPX_CHECK_LAUNCH("spx_dia_square");
    return SPX_OK;
}

extern "C" spx_status spx_cg_batched_dia(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys, const int32_t* order,
                                         const float* b, double* x, const int32_t* dia_offsets, const int32_t* dia_nd,
                                         const void* dia_values_bf16, double tol, int32_t maxit, double delta,
                                         int32_t* iters, int32_t* status, double* relres, void* ws, size_t ws_bytes,
                                         void* stream) {
    SPX_TRY(check_csr(A, true, "spx_cg_batched_dia"));
    if (A->m != A->n) return set_error(SPX_INVALID_ARG, "spx_cg_batched_dia: A must be square");
    if (nsys < 0 || (nsys > 0 && (!sys_ptr || !b || !x || !iters || !status || !relres || !dia_offsets || !dia_nd ||
                                  !dia_values_bf16)))
        return set_error(SPX_INVALID_ARG, "spx_cg_batched_dia: NULL argument");
    if (!(tol > 0.0) || maxit < 0 || !(delta > 0.0 && delta < 1.0))
        return set_error(SPX_INVALID_ARG, "spx_cg_batched_dia: tol > 0, maxit >= 0, 0 < delta < 1 required");
    size_t need = 0;
    spx_cg_workspace_size(A->m, &need);
    if (!ws || ws_bytes < need)
        return set_error(SPX_OOM_WORKSPACE, "spx_cg_batched_dia: workspace %zu < %zu", ws_bytes, need);
    if (nsys == 0) return SPX_OK;
    const size_t v = ((size_t)A->m * 4 + 255) & ~size_t(255);
    char* w = static_cast<char*>(ws);
    CgArgs a{};
    a.nsys = nsys;
    a.sys_ptr = sys_ptr;
    a.order = order;
    a.a_ptr = A->indptr;
    a.a_idx = A->indices;
    a.a_val = A->values;
    a.b = b;
    a.x = x;
    a.pc = 5;
    a.dia_off = dia_offsets;
    a.dia_nd = dia_nd;
    a.dia_val = static_cast<const __nv_bfloat16*>(dia_values_bf16);
    a.n = A->m;
    a.r = (float*)(w + 0 * v);
    a.p = (float*)(w + 1 * v);
    a.q = (float*)(w + 2 * v);
    a.z = (float*)(w + 3 * v);
    a.w = (float*)(w + 4 * v);
    a.xp = (float*)(w + 5 * v);
    a.queue = (int32_t*)(w + 6 * v);
    a.tol = tol;
    a.delta = delta;
    a.maxit = maxit;
    a.iters = iters;
    a.status = status;
    a.relres = relres;
    return launch_pcg(a, 5, as_stream(stream));
}
