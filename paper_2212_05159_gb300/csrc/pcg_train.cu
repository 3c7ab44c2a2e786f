// Loss and gradient of the unrolled PCG residual history w.r.t. the learned factor
// (Section 4.3):  M = L L^T,  N_it iterations from x0 = 0,
//   loss_s = sum_{i=1..N_it} w_i ||r_i|| / ||b||,  w_i = gamma^(N_it-i) / sum_j gamma^(N_it-j),
// for every system s of a block-diagonal batch, and d(mean_s loss_s) / d L.values on L's
// pattern (sparse gradient, Table 1: the SpMV VJP w.r.t. a matrix is a masked outer
// product).  The reverse pass is the chain rule (Section 2) applied statement by
// statement to the forward iterates, in reverse order -- all of them kept, or every
// s-th state kept and the iterates between recomputed (checkpoint interval s).
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
    int32_t seg;           // iterations per segment: the checkpoint interval (n_it: keep every iterate)
    const float* wts;      // [n_it] loss weights
    float* ck;             // 2 n floats per checkpoint after the first: r, p at iterations seg, 2 seg, ...
                           // (plus iteration 0), only when there is more than one segment
    float* store;          // 5 (seg + 1) n floats: r, z, w, p, q for the slots 0..seg of a segment
    float* tmp;            // 6 * n floats: RB, PB, PBn, ZB, WB, QB
    int64_t n;
    float* loss;           // [nsys]
    float* gL;             // [nnz(L)], overwritten
    float inv_nsys;        // gradient of the mean over systems
};

// Iterates are addressed by (kind, slot): slot t of the segment that starts at iteration c
// holds iteration c + t (slot 0: the state at c, r_c and p_c).  With one segment (seg =
// n_it) every iterate stays in the store, as a plain stored reverse pass needs.  With
// more, the forward keeps r and p at every segment start (a checkpoint) and the reverse
// pass runs the forward of each earlier segment again from its checkpoint before walking
// it backwards.  The recomputed iterates come out of the same code on the same inputs, in
// the same thread order, so they equal the first forward's bit for bit.
enum { V_R = 0, V_Z = 1, V_W = 2, V_P = 3, V_Q = 4 };

__global__ void __launch_bounds__(PT_THREADS) pcg_train_kernel(TrainArgs a) {
    __shared__ double red[PT_WARPS];
    __shared__ double sc[4 * (PT_MAX_IT + 1)];   // rz, s, alpha, beta per iteration
    const int sid = blockIdx.x;
    if (sid >= a.nsys) return;
    const int R0 = a.sys_ptr[sid], R1 = a.sys_ptr[sid + 1];
    const int N = a.n_it;
    const int S = a.seg;
    const int J = (N - 1) / S;                   // segments 0..J
    const int64_t n = a.n;
    auto vec = [&](int kind, int slot) { return a.store + ((int64_t)kind * (S + 1) + slot) * n; };
    auto ckr = [&](int k) { return a.ck + (int64_t)(2 * k) * n; };
    auto ckp = [&](int k) { return a.ck + (int64_t)(2 * k + 1) * n; };
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

    // One PCG iteration `it` of the segment starting at c (slot t = it - c): q = A p, alpha,
    // r -= alpha q, w = L^T r, z = L w, beta, p = z + beta p.  `first`: the forward proper
    // (records the scalars and returns ||r_it||); otherwise a recomputation.
    auto iterate = [&](int it, int c, double& rz_cur, bool first) -> double {
        const int t = it - c;
        const float* pp = vec(V_P, t - 1);
        const float* rp = vec(V_R, t - 1);
        float* q = vec(V_Q, t);
        float* r = vec(V_R, t);
        float* w = vec(V_W, t);
        float* z = vec(V_Z, t);
        float* p = vec(V_P, t);
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
        // (its barriers also complete r before w = L^T r gathers it)
        const double rn_it = sqrt(block_sum((double)rr.hi + rr.lo, red));
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) w[i] = row_dot(a.LT, r, i);
        __syncthreads();
        DF tt{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float zi = row_dot(a.L, w, i);
            z[i] = zi;
            df_add_prod(tt, r[i], zi);
        }
        const double rz_it = block_sum((double)tt.hi + tt.lo, red);
        const double b_it = rz_it / rz_cur;
        if (first && threadIdx.x == 0) {
            sv[it] = s_it;
            al[it] = a_it;
            rn[it] = rn_it;
            rz[it] = rz_it;
            be[it] = b_it;
        }
        rz_cur = rz_it;
        const float beta = (float)b_it;
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) p[i] = fmaf(beta, pp[i], z[i]);
        return rn_it;
    };

    // ------------------------------------------------------------- forward
    {
        float* r0 = vec(V_R, 0);
        float* z0 = vec(V_Z, 0);
        float* w0 = vec(V_W, 0);
        float* p0 = vec(V_P, 0);
        DF bb{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float bi = a.b[i];
            r0[i] = bi;
            df_add_prod(bb, bi, bi);
        }
        const double bn = sqrt(block_sum((double)bb.hi + bb.lo, red));
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) w0[i] = row_dot(a.LT, r0, i);
        __syncthreads();
        DF t0{0.f, 0.f};
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            const float zi = row_dot(a.L, w0, i);
            z0[i] = zi;
            p0[i] = zi;
            df_add_prod(t0, r0[i], zi);
            if (J > 0) {
                ckr(0)[i] = r0[i];
                ckp(0)[i] = zi;
            }
        }
        const double rz0 = block_sum((double)t0.hi + t0.lo, red);
        if (threadIdx.x == 0) {
            rz[0] = rz0;
            rn[0] = bn;
        }
    }
    __syncthreads();
    double rz_cur = rz[0];
    double loss = 0.0;
    for (int it = 1; it <= N; ++it) {
        const int k = (it - 1) / S;
        const int c = k * S;
        if (it > 1 && it - 1 == c) {
            // a new segment starts at c: the state at c (slot S of the last one) moves to
            // slot 0 and is kept as checkpoint k
            for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
                const float ri = vec(V_R, S)[i], pi = vec(V_P, S)[i];
                vec(V_R, 0)[i] = ri;
                vec(V_P, 0)[i] = pi;
                ckr(k)[i] = ri;
                ckp(k)[i] = pi;
            }
        }
        loss += (double)a.wts[it - 1] * iterate(it, c, rz_cur, true);
    }
    __syncthreads();                                           // scalars visible
    const double bnorm_v = rn[0];
    loss /= bnorm_v;
    if (threadIdx.x == 0) a.loss[sid] = (float)loss;

    // ------------------------------------------------------------- reverse
    const float gscale = a.inv_nsys;
    for (int k = 0; k <= N; ++k) rzb[k] = 0.0;
    {
        const float* rN = vec(V_R, N - J * S);                 // the last segment is still in the store
        for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
            RB[i] = (float)(a.wts[N - 1] / (bnorm_v * rn[N])) * rN[i] * gscale;
            PB[i] = 0.f;
        }
    }
    for (int e = a.L.ptr[R0] + threadIdx.x; e < a.L.ptr[R1]; e += PT_THREADS) a.gL[e] = 0.f;
    for (int k = J; k >= 0; --k) {
        const int c = k * S;
        const int e_it = min(c + S, N);
        if (k < J) {
            // segment k again from its checkpoint
            __syncthreads();                                   // the later segment's reverse is done with the store
            for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
                vec(V_R, 0)[i] = ckr(k)[i];
                vec(V_P, 0)[i] = ckp(k)[i];
            }
            double rzc = rz[c];
            for (int it = c + 1; it <= e_it; ++it) iterate(it, c, rzc, false);
        }
        for (int it = e_it; it >= c + 1; --it) {
            const int t = it - c;
            const float* pp = vec(V_P, t - 1);
            const float* r = vec(V_R, t);
            const float* z = vec(V_Z, t);
            const float* w = vec(V_W, t);
            const float* q = vec(V_Q, t);
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
            const float lw = it - 1 >= 1 ? (float)(a.wts[it - 2] / (bnorm_v * rn[it - 1])) * gscale : 0.f;
            const float* rprev = vec(V_R, t - 1);
            for (int i = R0 + threadIdx.x; i < R1; i += PT_THREADS) {
                PB[i] = PBn[i] + row_dot(a.A, QB, i);
                RB[i] = fmaf(lw, rprev[i], RB[i]);
            }
        }
    }
    __syncthreads();
    // p_0 = z_0; rz_0 = <r_0, z_0>; z_0 = L w_0; w_0 = L^T r_0 (slot 0 of segment 0: r_0 restored,
    // w_0 written by the forward's iteration 0 and never overwritten)
    {
        const float* r = vec(V_R, 0);
        const float* w = vec(V_W, 0);
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

static int train_segment(int32_t n_it, int32_t interval) {
    return (interval <= 0 || interval >= n_it) ? n_it : interval;
}

extern "C" spx_status spx_pcg_train_workspace_size(int32_t n, int32_t n_it, int32_t ckpt_interval, size_t* bytes) {
    if (!bytes || n < 0 || n_it < 1 || n_it > PT_MAX_IT)
        return set_error(SPX_INVALID_ARG, "spx_pcg_train_workspace_size: 1 <= n_it <= %d", PT_MAX_IT);
    const int seg = train_segment(n_it, ckpt_interval);
    const int segments = (n_it - 1) / seg + 1;
    const size_t ck_vectors = segments > 1 ? (size_t)2 * segments : 0;
    *bytes = (ck_vectors + (size_t)5 * (seg + 1) + 6) * (size_t)n * 4 + 256;
    return SPX_OK;
}

extern "C" spx_status spx_pcg_train(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys, const spx_csr* L,
                                    const spx_csr* LT, const float* b, int32_t n_it, int32_t ckpt_interval,
                                    const float* weights,
                                    float* loss, float* grad_L, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_pcg_train"));
    SPX_TRY(check_csr(L, true, "spx_pcg_train (L)"));
    SPX_TRY(check_csr(LT, true, "spx_pcg_train (L^T)"));
    if (A->m != A->n || L->m != A->m || LT->m != A->m)
        return set_error(SPX_INVALID_ARG, "spx_pcg_train: shapes");
    if (nsys < 0 || (nsys > 0 && (!sys_ptr || !b || !weights || !loss || !grad_L)))
        return set_error(SPX_INVALID_ARG, "spx_pcg_train: NULL argument");
    size_t need = 0;
    SPX_TRY(spx_pcg_train_workspace_size(A->m, n_it, ckpt_interval, &need));
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
    t.seg = train_segment(n_it, ckpt_interval);
    t.wts = weights;
    t.n = A->m;
    t.store = static_cast<float*>(ws);
    t.tmp = t.store + (int64_t)5 * (t.seg + 1) * A->m;
    t.ck = t.tmp + (int64_t)6 * A->m;                          // used only with more than one segment
    t.loss = loss;
    t.gL = grad_L;
    t.inv_nsys = 1.0f / (float)nsys;
    pcg_train_kernel<<<nsys, PT_THREADS, 0, as_stream(stream)>>>(t);
    SPX_CHECK_LAUNCH("spx_pcg_train");
    return SPX_OK;
}
