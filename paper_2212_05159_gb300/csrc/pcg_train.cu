// Loss and gradient of the unrolled PCG residual history w.r.t. the learned factor
// (Section 4.3):  M = L L^T,  N_it iterations from x0 = 0,
//   loss_s = sum_{i=1..N_it} w_i ||r_i|| / ||b||,  w_i = gamma^(N_it-i) / sum_j gamma^(N_it-j),
// for every system s of a block-diagonal batch, and d(mean_s loss_s) / d L.values on L's
// pattern (sparse gradient, Table 1: the SpMV VJP w.r.t. a matrix is a masked outer
// product).  The reverse pass is the chain rule (Section 2) applied statement by
// statement to the stored forward iterates, in reverse order.
//
// One thread block per system (training systems have up to ~16k rows); every stage is
// separated by a block barrier; vectors live in global memory (L2-resident for a batch);
// inner products accumulate per thread in double-float and across the block in FP64, in
// a fixed order (deterministic).  Masked outer products update each stored entry of L
// from the thread that owns its row: no atomics.
#include <math.h>

#include "common.cuh"

namespace spx {
namespace {

// 1024 threads: 28 % faster than 512 on a training batch of 32 systems (fewer rows per thread
// on the block's dependent passes; 64 registers, no spills)
constexpr int PT_THREADS = 1024;
constexpr int PT_WARPS = PT_THREADS / 32;
constexpr int PT_MAX_IT = 64;

struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_add_prod(DF& s, float a, float b) {
    const float ph = a * b;
    const float pl = fmaf(a, b, -ph);
    const float t = s.hi + ph;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (ph - bp);
    s.hi = t;
    s.lo += err + pl;
}

// Block-wide FP64 sum of one value per thread (fixed order); result in every thread.
__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    __syncthreads();                         // red free from the previous use
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < PT_WARPS; ++w) s += red[w];
    return s;
}

struct Mat {
    const int32_t* ptr;
    const int32_t* idx;
    const float* val;
};

__device__ __forceinline__ float row_dot(const Mat& M, const float* __restrict__ x, int i) {
    float s = 0.f;
    for (int e = M.ptr[i]; e < M.ptr[i + 1]; ++e) s = fmaf(M.val[e], x[M.idx[e]], s);
    return s;
}

struct TrainArgs {
    int32_t nsys;
    const int32_t* sys_ptr;
    Mat A, L, LT;
    const float* b;
    int32_t n_it;
    const float* wts;      // [n_it] loss weights
    float* store;          // 5 * (n_it + 1) * n floats: r, z, w, p, q per iteration
    float* tmp;            // 6 * n floats: RB, PB, PBn, ZB, WB, QB
    int64_t n;
    float* loss;           // [nsys]
    float* gL;             // [nnz(L)], overwritten
    float inv_nsys;        // gradient of the mean over systems
};

__global__ void __launch_bounds__(PT_THREADS) pcg_train_kernel(TrainArgs a) {
    __shared__ double red[PT_WARPS];
    __shared__ double sc[4 * (PT_MAX_IT + 1)];   // rz, s, alpha, beta per iteration
    const int sid = blockIdx.x;
    if (sid >= a.nsys) return;
    const int R0 = a.sys_ptr[sid], R1 = a.sys_ptr[sid + 1];
    const int N = a.n_it;
    const int64_t n = a.n;
    auto vec = [&](int which, int i) { return a.store + ((int64_t)which * (N + 1) + i) * n; };
    float* RB = a.tmp;
    float* PB = a.tmp + n;
    float* PBn = a.tmp + 2 * n;
    float* ZB = a.tmp + 3 * n;
    float* WB = a.tmp + 4 * n;
    float* QB = a.tmp + 5 * n;
    // per-iteration scalars: written by thread 0, read after a barrier
    double* rz = sc;
    double* sv = sc + (PT_MAX_IT + 1);
    double* al = sc + 2 * (PT_MAX_IT + 1);
    double* be = sc + 3 * (PT_MAX_IT + 1);
    __shared__ double rn[PT_MAX_IT + 1];
    double rzb[PT_MAX_IT + 1];           // identical in every thread

    // ------------------------------------------------------------- forward
    float* r0 = vec(0, 0);
    float* z0 = vec(1, 0);
    float* w0 = vec(2, 0);
    float* p0 = vec(3, 0);
    DF bb{0.f, 0.f};
    for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
        const float bi = a.b[i];
        r0[i] = bi;
        df_add_prod(bb, bi, bi);
    }
    const double bnorm = sqrt(block_sum((double)bb.hi + bb.lo, red));
    for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) w0[i] = row_dot(a.LT, r0, i);
    __syncthreads();
    DF t0{0.f, 0.f};
    for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
        const float zi = row_dot(a.L, w0, i);
        z0[i] = zi;
        p0[i] = zi;
        df_add_prod(t0, r0[i], zi);
    }
    double rz_cur = block_sum((double)t0.hi + t0.lo, red);
    if (threadIdx.x == 0) {
        rz[0] = rz_cur;
        rn[0] = bnorm;
    }
    double loss = 0.0;
    for (int it = 1; it <= N; ++it) {
        const float* pp = vec(3, it - 1);
        const float* rp = vec(0, it - 1);
        float* q = vec(4, it);
        float* r = vec(0, it);
        float* w = vec(2, it);
        float* z = vec(1, it);
        float* p = vec(3, it);
        __syncthreads();                                       // p_{it-1} complete
        DF s{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float qi = row_dot(a.A, pp, i);
            q[i] = qi;
            df_add_prod(s, pp[i], qi);
        }
        const double s_it = block_sum((double)s.hi + s.lo, red);
        const double a_it = rz_cur / s_it;
        const float alpha = (float)a_it;
        DF rr{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float ri = fmaf(-alpha, q[i], rp[i]);
            r[i] = ri;
            df_add_prod(rr, ri, ri);
        }
        const double rn_it = sqrt(block_sum((double)rr.hi + rr.lo, red));
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) w[i] = row_dot(a.LT, r, i);
        __syncthreads();
        DF t{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float zi = row_dot(a.L, w, i);
            z[i] = zi;
            df_add_prod(t, r[i], zi);
        }
        const double rz_it = block_sum((double)t.hi + t.lo, red);
        const double b_it = rz_it / rz_cur;
        if (threadIdx.x == 0) {
            sv[it] = s_it;
            al[it] = a_it;
            rn[it] = rn_it;
            rz[it] = rz_it;
            be[it] = b_it;
        }
        rz_cur = rz_it;
        loss += (double)a.wts[it - 1] * rn_it;
        const float beta = (float)b_it;
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) p[i] = fmaf(beta, pp[i], z[i]);
    }
    loss /= bnorm;
    if (threadIdx.x == 0) a.loss[sid] = (float)loss;
    __syncthreads();                                           // scalars visible

    // ------------------------------------------------------------- reverse
    const float gscale = a.inv_nsys;
    for (int k = 0; k <= N; ++k) rzb[k] = 0.0;
    for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
        RB[i] = (float)(a.wts[N - 1] / (bnorm * rn[N])) * vec(0, N)[i] * gscale;
        PB[i] = 0.f;
    }
    for (int e = a.L.ptr[R0] + threadIdx.x; e < a.L.ptr[R1]; e += PT_THREADS) a.gL[e] = 0.f;
    for (int it = N; it >= 1; --it) {
        const float* pp = vec(3, it - 1);
        const float* r = vec(0, it);
        const float* z = vec(1, it);
        const float* w = vec(2, it);
        const float* q = vec(4, it);
        __syncthreads();
        // p_it = z_it + beta p_{it-1}
        DF tb{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) df_add_prod(tb, PB[i], pp[i]);
        const double betab = block_sum((double)tb.hi + tb.lo, red);
        rzb[it] += betab / rz[it - 1];
        rzb[it - 1] -= betab * rz[it] / (rz[it - 1] * rz[it - 1]);
        const float fb = (float)be[it];
        const float frzb = (float)rzb[it];
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float pbi = PB[i];
            PBn[i] = fb * pbi;                                // pb_{it-1} starts here
            ZB[i] = fmaf(frzb, r[i], pbi);                    // zb = pb + rzb r
            RB[i] = fmaf(frzb, z[i], RB[i]);                  // rb += rzb z
        }
        __syncthreads();
        // z = L w:  gL += zb (x) w ; wb = L^T zb
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float zbi = ZB[i];
            for (int e = a.L.ptr[i]; e < a.L.ptr[i + 1]; ++e) a.gL[e] = fmaf(zbi, w[a.L.idx[e]], a.gL[e]);
            WB[i] = row_dot(a.LT, ZB, i);
        }
        __syncthreads();
        // w = L^T r:  gL += r (x) wb ; rb += L wb
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float ri = r[i];
            for (int e = a.L.ptr[i]; e < a.L.ptr[i + 1]; ++e) a.gL[e] = fmaf(ri, WB[a.L.idx[e]], a.gL[e]);
            RB[i] += row_dot(a.L, WB, i);
        }
        __syncthreads();
        // r_it = r_{it-1} - alpha q:  alphab = -<rb, q>
        DF ta{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) df_add_prod(ta, RB[i], q[i]);
        const double alphab = -block_sum((double)ta.hi + ta.lo, red);
        rzb[it - 1] += alphab / sv[it];
        const double sb = -alphab * rz[it - 1] / (sv[it] * sv[it]);
        const float fal = (float)al[it], fsb = (float)sb;
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            QB[i] = fmaf(-fal, RB[i], fsb * pp[i]);          // qb = -alpha rb + sb p
            PBn[i] = fmaf(fsb, q[i], PBn[i]);                 // pb_{it-1} += sb q
        }
        __syncthreads();
        // q = A p_{it-1}:  pb_{it-1} += A^T qb (A symmetric); rb_{it-1} = rb + loss term
        const float lw = it - 1 >= 1 ? (float)(a.wts[it - 2] / (bnorm * rn[it - 1])) * gscale : 0.f;
        const float* rprev = vec(0, it - 1);
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            PB[i] = PBn[i] + row_dot(a.A, QB, i);
            RB[i] = fmaf(lw, rprev[i], RB[i]);
        }
    }
    __syncthreads();
    // p_0 = z_0; rz_0 = <r_0, z_0>; z_0 = L w_0; w_0 = L^T r_0
    {
        const float* r = vec(0, 0);
        const float* w = vec(2, 0);
        const float frzb = (float)rzb[0];
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) ZB[i] = fmaf(frzb, r[i], PB[i]);
        __syncthreads();
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float zbi = ZB[i];
            for (int e = a.L.ptr[i]; e < a.L.ptr[i + 1]; ++e) a.gL[e] = fmaf(zbi, w[a.L.idx[e]], a.gL[e]);
            WB[i] = row_dot(a.LT, ZB, i);
        }
        __syncthreads();
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float ri = r[i];
            for (int e = a.L.ptr[i]; e < a.L.ptr[i + 1]; ++e) a.gL[e] = fmaf(ri, WB[a.L.idx[e]], a.gL[e]);
        }
    }
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_pcg_train_workspace_size(int32_t n, int32_t n_it, size_t* bytes) {
    if (!bytes || n < 0 || n_it < 1 || n_it > PT_MAX_IT)
        return set_error(SPX_INVALID_ARG, "spx_pcg_train_workspace_size: 1 <= n_it <= %d", PT_MAX_IT);
    *bytes = ((size_t)5 * (n_it + 1) + 6) * (size_t)n * 4 + 256;
    return SPX_OK;
}

extern "C" spx_status spx_pcg_train(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys, const spx_csr* L,
                                    const spx_csr* LT, const float* b, int32_t n_it, const float* weights,
                                    float* loss, float* grad_L, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_pcg_train"));
    SPX_TRY(check_csr(L, true, "spx_pcg_train (L)"));
    SPX_TRY(check_csr(LT, true, "spx_pcg_train (L^T)"));
    if (A->m != A->n || L->m != A->m || LT->m != A->m)
        return set_error(SPX_INVALID_ARG, "spx_pcg_train: shapes");
    if (nsys < 0 || (nsys > 0 && (!sys_ptr || !b || !weights || !loss || !grad_L)))
        return set_error(SPX_INVALID_ARG, "spx_pcg_train: NULL argument");
    size_t need = 0;
    SPX_TRY(spx_pcg_train_workspace_size(A->m, n_it, &need));
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_pcg_train: workspace %zu < %zu", ws_bytes, need);
    if (nsys == 0) return SPX_OK;
    TrainArgs t{};
    t.nsys = nsys;
    t.sys_ptr = sys_ptr;
    t.A = Mat{A->indptr, A->indices, A->values};
    t.L = Mat{L->indptr, L->indices, L->values};
    t.LT = Mat{LT->indptr, LT->indices, LT->values};
    t.b = b;
    t.n_it = n_it;
    t.wts = weights;
    t.n = A->m;
    t.store = static_cast<float*>(ws);
    t.tmp = t.store + (int64_t)5 * (n_it + 1) * A->m;
    t.loss = loss;
    t.gL = grad_L;
    t.inv_nsys = 1.0f / (float)nsys;
    pcg_train_kernel<<<nsys, PT_THREADS, 0, as_stream(stream)>>>(t);
    SPX_CHECK_LAUNCH("spx_pcg_train");
    return SPX_OK;
}
