// Kernels of the message-passing network that emits the learned factor L on tril(A)
// (the learned preconditioner M = L L^T of Section 4.3):
//   features      d_i = a_ii^-1/2, e_ij = d_i a_ij d_j, node inputs [1, sum, min, max]
//   dense layers  Y = [X1 X2] W + b with fused epilogues (relu, residual), their data and
//                 weight gradients (BF16 weights, FP32 accumulation)
//   edge head     o_e = relu(P_i + Q_j + e_ij u + c) . v + bias, L_e = d_i lhat(o_e),
//                 and its reverse (recomputing the hidden edge activations)
//   tril          the pattern of tril(A) with the position of each entry in A
//   adam          the optimizer step, refreshing the BF16 copy of the weights
// Reductions over rows / edges write per-block partials that a second pass adds in a
// fixed order: every result is deterministic.  Message passing itself (E h and its
// transpose) runs on the library's SpMM kernels.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "scan.cuh"

namespace spx {
namespace {

constexpr int HID = 64;
constexpr int DT = 256;            // threads of the dense kernels
constexpr int DROWS = 16;          // rows per dense tile (16 threads per row, 4 columns each)
constexpr int KMAX = 128;          // max inner dimension of a dense layer
constexpr int NMAX = 128;          // max output width of a dense layer

__device__ __forceinline__ float softplus(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid(float x) { return 1.f / (1.f + expf(-x)); }

// ---------------------------------------------------------------- features
__global__ void diag_rsqrt_kernel(int32_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                  const float* __restrict__ val, float* __restrict__ d) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = 0.f;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e)
        if (idx[e] == i) a = val[e];
    d[i] = a > 0.f ? rsqrtf(a) : 0.f;
}

__global__ void features_kernel(int32_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                const float* __restrict__ val, const float* __restrict__ d, float* __restrict__ ev,
                                float* __restrict__ f) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f, mn = INFINITY, mx = -INFINITY;
    bool any = false;
    const float di = d[i];
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
        const int j = idx[e];
        const float v = di * val[e] * d[j];
        ev[e] = v;
        if (j != i) {
            s += v;
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
            any = true;
        }
    }
    f[i * 4 + 0] = 1.f;
    f[i * 4 + 1] = s;
    f[i * 4 + 2] = any ? mn : 0.f;
    f[i * 4 + 3] = any ? mx : 0.f;
}

// ---------------------------------------------------------------- dense forward
// Y = [X1 X2] W + b (W: (K1+K2) x N, BF16).  mode 0: Y = pre; 1: Y = relu(pre);
// 2: U = pre and Y = Hin + relu(pre).
__global__ void __launch_bounds__(DT) dense_fwd_kernel(int64_t n, const float* __restrict__ X1, int K1,
                                                       const float* __restrict__ X2, int K2,
                                                       const __nv_bfloat16* __restrict__ W,
                                                       const float* __restrict__ bias, int N, int mode,
                                                       const float* __restrict__ Hin, float* __restrict__ Y,
                                                       float* __restrict__ U) {
    __shared__ float Ws[KMAX * 64];      // one 64-column panel of W at a time
    __shared__ float Xs[DROWS][KMAX + 1];
    const int K = K1 + K2;
    const int64_t r0 = (int64_t)blockIdx.x * DROWS;
    for (int t = threadIdx.x; t < DROWS * K; t += DT) {
        const int rr = t / K, k = t % K;
        const int64_t row = r0 + rr;
        float x = 0.f;
        if (row < n) x = k < K1 ? X1[row * K1 + k] : X2[row * K2 + (k - K1)];
        Xs[rr][k] = x;
    }
    for (int c0 = 0; c0 < N; c0 += 64) {
        __syncthreads();
        for (int t = threadIdx.x; t < K * 64; t += DT) {
            const int k = t / 64, c = t % 64;
            Ws[t] = c0 + c < N ? __bfloat162float(W[k * N + c0 + c]) : 0.f;
        }
        __syncthreads();
        // thread -> (row, 4 columns): 16 threads per row, 16 rows
        const int rr = threadIdx.x / 16;
        const int cc = (threadIdx.x % 16) * 4;
        float acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = 0.f;
        for (int k = 0; k < K; ++k) {
            const float x = Xs[rr][k];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(x, Ws[k * 64 + cc + q], acc[q]);
        }
        const int64_t row = r0 + rr;
        if (row < n) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = c0 + cc + q;
                if (c >= N) continue;
                const float pre = acc[q] + (bias ? bias[c] : 0.f);
                if (mode == 0) {
                    Y[row * N + c] = pre;
                } else if (mode == 1) {
                    Y[row * N + c] = fmaxf(pre, 0.f);
                } else {
                    U[row * N + c] = pre;
                    Y[row * N + c] = Hin[row * N + c] + fmaxf(pre, 0.f);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- dense backward (data)
// [dX1 dX2] (+)= G W^T, G: n x N, W: (K1+K2) x N (BF16).
__global__ void __launch_bounds__(DT) dense_bwd_data_kernel(int64_t n, const float* __restrict__ G, int N,
                                                            const __nv_bfloat16* __restrict__ W, int K1, int K2,
                                                            float* __restrict__ dX1, float* __restrict__ dX2,
                                                            int accumulate) {
    __shared__ float Wt[NMAX * 64];       // W^T panel: [N][64 rows of W]
    __shared__ float Gs[DROWS][NMAX + 1];
    const int K = K1 + K2;
    const int64_t r0 = (int64_t)blockIdx.x * DROWS;
    for (int t = threadIdx.x; t < DROWS * N; t += DT) {
        const int rr = t / N, c = t % N;
        const int64_t row = r0 + rr;
        Gs[rr][c] = row < n ? G[row * N + c] : 0.f;
    }
    for (int k0 = 0; k0 < K; k0 += 64) {
        __syncthreads();
        for (int t = threadIdx.x; t < N * 64; t += DT) {
            const int c = t / 64, k = t % 64;
            Wt[t] = k0 + k < K ? __bfloat162float(W[(k0 + k) * N + c]) : 0.f;
        }
        __syncthreads();
        const int rr = threadIdx.x / 16;
        const int kk = (threadIdx.x % 16) * 4;
        float acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = 0.f;
        for (int c = 0; c < N; ++c) {
            const float g = Gs[rr][c];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(g, Wt[c * 64 + kk + q], acc[q]);
        }
        const int64_t row = r0 + rr;
        if (row < n) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k0 + kk + q;
                if (k >= K) continue;
                float* dst = k < K1 ? dX1 + row * K1 + k : dX2 + row * K2 + (k - K1);
                if (k >= K1 && !dX2) continue;
                *dst = accumulate ? *dst + acc[q] : acc[q];
            }
        }
    }
}

// ---------------------------------------------------------------- dense backward (weights)
// partial[b] = sum over the block's rows of [X1 X2]^T G (and, in row K, sum of G).
constexpr int WROWS = 256;         // rows per block of the weight gradient
constexpr int WOUT_MAX = 33 * DT;  // (K + 1) * N outputs at most (e.g. 129 x 64, 65 x 128)
__global__ void __launch_bounds__(DT) dense_bwd_weight_kernel(int64_t n, const float* __restrict__ X1, int K1,
                                                              const float* __restrict__ X2, int K2,
                                                              const float* __restrict__ G, int N,
                                                              float* __restrict__ partial) {
    __shared__ float Xs[16][KMAX + 1];
    __shared__ float Gs[16][NMAX];
    const int K = K1 + K2;
    const int KB = K + 1;                          // + bias row
    const int outs = KB * N;
    constexpr int PER = WOUT_MAX / DT;             // outputs per thread
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.f;
    const int64_t rb = (int64_t)blockIdx.x * WROWS;
    for (int r0 = 0; r0 < WROWS; r0 += 16) {
        __syncthreads();
        for (int t = threadIdx.x; t < 16 * K; t += DT) {
            const int rr = t / K, k = t % K;
            const int64_t row = rb + r0 + rr;
            float x = 0.f;
            if (row < n) x = k < K1 ? X1[row * K1 + k] : X2[row * K2 + (k - K1)];
            Xs[rr][k] = x;
        }
        for (int t = threadIdx.x; t < 16 * N; t += DT) {
            const int rr = t / N, c = t % N;
            const int64_t row = rb + r0 + rr;
            Gs[rr][c] = row < n ? G[row * N + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int o = threadIdx.x + q * DT;
            if (o < outs) {
                const int k = o / N, c = o % N;
                float s = acc[q];
                for (int rr = 0; rr < 16; ++rr) s = fmaf(k < K ? Xs[rr][k] : 1.f, Gs[rr][c], s);
                acc[q] = s;
            }
        }
    }
    float* out = partial + (int64_t)blockIdx.x * outs;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int o = threadIdx.x + q * DT;
        if (o < outs) out[o] = acc[q];
    }
}

__global__ void sum_partials_kernel(int nparts, int outs, const float* __restrict__ partial, int K, int N,
                                    float* __restrict__ dW, float* __restrict__ db) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= outs) return;
    float s = 0.f;
    for (int b = 0; b < nparts; ++b) s += partial[(int64_t)b * outs + o];
    const int k = o / N, c = o % N;
    if (k < K) dW[o] = s;
    else if (db) db[c] = s;
}

__global__ void relu_backward_kernel(int64_t count, const float* __restrict__ gh, const float* __restrict__ u,
                                     float* __restrict__ gu) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += stride)
        gu[t] = u[t] > 0.f ? gh[t] : 0.f;
}

// ---------------------------------------------------------------- tril(A)
__global__ void tril_count_kernel(int32_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                  int32_t* __restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) c += idx[e] <= i;
    cnt[i] = c;
}

__global__ void tril_fill_kernel(int32_t n, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                 const int32_t* __restrict__ lptr, int32_t* __restrict__ lidx,
                                 int32_t* __restrict__ src) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = lptr[i];
    for (int e = ptr[i]; e < ptr[i + 1]; ++e)
        if (idx[e] <= i) {
            lidx[o] = idx[e];
            src[o] = e;
            ++o;
        }
}

// ---------------------------------------------------------------- edge head
struct EdgeParams {
    const float* u;
    const float* c;
    const float* v;
    const float* bd;
    const float* bo;
};

// warp per row of tril(A); lanes hold hidden units lane and lane + 32
__global__ void edge_fwd_kernel(int32_t n, const int32_t* __restrict__ lptr, const int32_t* __restrict__ lidx,
                                const float* __restrict__ el, const float* __restrict__ d,
                                const float* __restrict__ P, const float* __restrict__ Q, EdgeParams pr,
                                float* __restrict__ L) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const float p0 = P[i * HID + lane], p1 = P[i * HID + lane + 32];
    const float u0 = pr.u[lane], u1 = pr.u[lane + 32];
    const float c0 = pr.c[lane], c1 = pr.c[lane + 32];
    const float v0 = pr.v[lane], v1 = pr.v[lane + 32];
    for (int e = lptr[i]; e < lptr[i + 1]; ++e) {
        const int j = lidx[e];
        const float ee = el[e];
        const float t0 = fmaxf(p0 + Q[(int64_t)j * HID + lane] + ee * u0 + c0, 0.f);
        const float t1 = fmaxf(p1 + Q[(int64_t)j * HID + lane + 32] + ee * u1 + c1, 0.f);
        float o = fmaf(t0, v0, t1 * v1);
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) o += __shfl_xor_sync(FULL, o, off);
        if (lane == 0) {
            const bool dg = j == i;
            o += dg ? pr.bd[0] : pr.bo[0];
            L[e] = d[i] * (dg ? softplus(o) : o);
        }
    }
}

// Recomputes the hidden activations of edge e = (i, j) and returns (gt0, gt1) for the
// lane's two hidden units, plus go and t (for the parameter gradients).
__device__ __forceinline__ void edge_back(int i, int j, float ee, float gl, const float* __restrict__ d,
                                          const float* __restrict__ P, const float* __restrict__ Q,
                                          const EdgeParams& pr, int lane, float& gt0, float& gt1, float& go,
                                          float& t0, float& t1) {
    const float pre0 = P[(int64_t)i * HID + lane] + Q[(int64_t)j * HID + lane] + ee * pr.u[lane] + pr.c[lane];
    const float pre1 = P[(int64_t)i * HID + lane + 32] + Q[(int64_t)j * HID + lane + 32] + ee * pr.u[lane + 32] +
                       pr.c[lane + 32];
    t0 = fmaxf(pre0, 0.f);
    t1 = fmaxf(pre1, 0.f);
    float o = fmaf(t0, pr.v[lane], t1 * pr.v[lane + 32]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) o += __shfl_xor_sync(FULL, o, off);
    const bool dg = j == i;
    o += dg ? pr.bd[0] : pr.bo[0];
    const float glh = gl * d[i];
    go = dg ? glh * sigmoid(o) : glh;
    gt0 = pre0 > 0.f ? go * pr.v[lane] : 0.f;
    gt1 = pre1 > 0.f ? go * pr.v[lane + 32] : 0.f;
}

constexpr int EB_ROWS = 16;        // tril rows per warp in the row pass
constexpr int EB_PART = 3 * HID + 2;

// Row pass: gP_i = sum over row i's edges of gt; per-warp partials of gv, gc, gu, gbd, gbo.
__global__ void edge_bwd_rows_kernel(int32_t n, const int32_t* __restrict__ lptr, const int32_t* __restrict__ lidx,
                                     const float* __restrict__ el, const float* __restrict__ d,
                                     const float* __restrict__ P, const float* __restrict__ Q, EdgeParams pr,
                                     const float* __restrict__ gL, float* __restrict__ gP,
                                     float* __restrict__ partial) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t i0 = w * EB_ROWS;
    if (i0 >= n) return;
    float gv0 = 0.f, gv1 = 0.f, gc0 = 0.f, gc1 = 0.f, gu0 = 0.f, gu1 = 0.f, gbd = 0.f, gbo = 0.f;
    for (int64_t i = i0; i < i0 + EB_ROWS && i < n; ++i) {
        float gp0 = 0.f, gp1 = 0.f;
        for (int e = lptr[i]; e < lptr[i + 1]; ++e) {
            const int j = lidx[e];
            float gt0, gt1, go, t0, t1;
            edge_back((int)i, j, el[e], gL[e], d, P, Q, pr, lane, gt0, gt1, go, t0, t1);
            gp0 += gt0;
            gp1 += gt1;
            gv0 = fmaf(go, t0, gv0);
            gv1 = fmaf(go, t1, gv1);
            gc0 += gt0;
            gc1 += gt1;
            gu0 = fmaf(gt0, el[e], gu0);
            gu1 = fmaf(gt1, el[e], gu1);
            if (j == i) gbd += go;
            else gbo += go;
        }
        gP[i * HID + lane] = gp0;
        gP[i * HID + lane + 32] = gp1;
    }
    float* pp = partial + w * EB_PART;
    pp[lane] = gv0;
    pp[lane + 32] = gv1;
    pp[HID + lane] = gc0;
    pp[HID + lane + 32] = gc1;
    pp[2 * HID + lane] = gu0;
    pp[2 * HID + lane + 32] = gu1;
    if (lane == 0) {
        pp[3 * HID] = gbd;
        pp[3 * HID + 1] = gbo;
    }
}

// Column pass: gQ_j = sum over the edges (i, j) of gt, through tril's transpose.
__global__ void edge_bwd_cols_kernel(int32_t n, const int32_t* __restrict__ tptr, const int32_t* __restrict__ tidx,
                                     const int32_t* __restrict__ tperm, const float* __restrict__ el,
                                     const float* __restrict__ d, const float* __restrict__ P,
                                     const float* __restrict__ Q, EdgeParams pr, const float* __restrict__ gL,
                                     float* __restrict__ gQ) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    float gq0 = 0.f, gq1 = 0.f;
    for (int t = tptr[j]; t < tptr[j + 1]; ++t) {
        const int i = tidx[t];
        const int e = tperm[t];
        float gt0, gt1, go, t0, t1;
        edge_back(i, (int)j, el[e], gL[e], d, P, Q, pr, lane, gt0, gt1, go, t0, t1);
        gq0 += gt0;
        gq1 += gt1;
    }
    gQ[j * HID + lane] = gq0;
    gQ[j * HID + lane + 32] = gq1;
}

__global__ void edge_sum_partials_kernel(int64_t nparts, const float* __restrict__ partial, float* __restrict__ out) {
    const int o = threadIdx.x + blockIdx.x * blockDim.x;
    if (o >= EB_PART) return;
    float s = 0.f;
    for (int64_t b = 0; b < nparts; ++b) s += partial[b * EB_PART + o];
    out[o] = s;
}

// ---------------------------------------------------------------- adam
__global__ void adam_kernel(int64_t count, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16* __restrict__ p16) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += stride) {
        const float gt = g[t];
        const float mt = fmaf(b1, m[t], (1.f - b1) * gt);
        const float vt = fmaf(b2, v[t], (1.f - b2) * gt * gt);
        m[t] = mt;
        v[t] = vt;
        const float upd = lr * (mt / c1) / (sqrtf(vt / c2) + eps);
        const float np = p[t] - upd;
        p[t] = np;
        if (p16) p16[t] = __float2bfloat16(np);
    }
}

__global__ void to_bf16_kernel(int64_t count, const float* __restrict__ p, __nv_bfloat16* __restrict__ p16) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count; t += stride)
        p16[t] = __float2bfloat16(p[t]);
}

unsigned grid1(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 32;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

unsigned warp_grid(int64_t warps) { return (unsigned)((warps * 32 + 255) / 256); }

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_mpnn_features(const spx_csr* A, float* d, float* e_vals, float* feats, void* stream) {
    SPX_TRY(check_csr(A, true, "spx_mpnn_features"));
    if (A->m != A->n) return set_error(SPX_INVALID_ARG, "spx_mpnn_features: A must be square");
    if (A->m == 0) return SPX_OK;
    if (!d || !feats || (A->nnz > 0 && !e_vals)) return set_error(SPX_INVALID_ARG, "spx_mpnn_features: NULL output");
    cudaStream_t st = as_stream(stream);
    const unsigned g = (unsigned)((A->m + 255) / 256);
    diag_rsqrt_kernel<<<g, 256, 0, st>>>(A->m, A->indptr, A->indices, A->values, d);
    SPX_CHECK_LAUNCH("mpnn diag");
    features_kernel<<<g, 256, 0, st>>>(A->m, A->indptr, A->indices, A->values, d, e_vals, feats);
    SPX_CHECK_LAUNCH("mpnn features");
    return SPX_OK;
}

extern "C" spx_status spx_dense_forward(int64_t n, const float* X1, int32_t K1, const float* X2, int32_t K2,
                                        const void* W_bf16, const float* bias, int32_t N, int32_t mode,
                                        const float* Hin, float* Y, float* U, void* stream) {
    if (n < 0 || K1 < 1 || K2 < 0 || K1 + K2 > KMAX || N < 1 || N > NMAX || mode < 0 || mode > 2)
        return set_error(SPX_INVALID_ARG, "spx_dense_forward: sizes (K <= %d, N <= %d)", KMAX, NMAX);
    if (n > 0 && (!X1 || (K2 > 0 && !X2) || !W_bf16 || !Y || (mode == 2 && (!Hin || !U))))
        return set_error(SPX_INVALID_ARG, "spx_dense_forward: NULL operand");
    if (n == 0) return SPX_OK;
    dense_fwd_kernel<<<(unsigned)((n + DROWS - 1) / DROWS), DT, 0, as_stream(stream)>>>(
        n, X1, K1, X2, K2, static_cast<const __nv_bfloat16*>(W_bf16), bias, N, mode, Hin, Y, U);
    SPX_CHECK_LAUNCH("spx_dense_forward");
    return SPX_OK;
}

extern "C" spx_status spx_dense_backward_data(int64_t n, const float* G, int32_t N, const void* W_bf16, int32_t K1,
                                              int32_t K2, float* dX1, float* dX2, int32_t accumulate, void* stream) {
    if (n < 0 || K1 < 1 || K2 < 0 || K1 + K2 > KMAX || N < 1 || N > NMAX)
        return set_error(SPX_INVALID_ARG, "spx_dense_backward_data: sizes");
    if (n > 0 && (!G || !W_bf16 || !dX1)) return set_error(SPX_INVALID_ARG, "spx_dense_backward_data: NULL operand");
    if (n == 0) return SPX_OK;
    dense_bwd_data_kernel<<<(unsigned)((n + DROWS - 1) / DROWS), DT, 0, as_stream(stream)>>>(
        n, G, N, static_cast<const __nv_bfloat16*>(W_bf16), K1, K2, dX1, dX2, accumulate);
    SPX_CHECK_LAUNCH("spx_dense_backward_data");
    return SPX_OK;
}

extern "C" spx_status spx_dense_backward_weight_workspace_size(int64_t n, int32_t K, int32_t N, size_t* bytes) {
    if (!bytes || n < 0 || K < 1 || K > KMAX || N < 1 || N > NMAX || (K + 1) * N > WOUT_MAX)
        return set_error(SPX_INVALID_ARG, "spx_dense_backward_weight_workspace_size: sizes ((K+1)*N <= %d)",
                         WOUT_MAX);
    const int64_t parts = (n + WROWS - 1) / WROWS;
    *bytes = (size_t)(parts > 0 ? parts : 1) * (size_t)(K + 1) * N * 4 + 256;
    return SPX_OK;
}

extern "C" spx_status spx_dense_backward_weight(int64_t n, const float* X1, int32_t K1, const float* X2, int32_t K2,
                                                const float* G, int32_t N, float* dW, float* db, void* ws,
                                                size_t ws_bytes, void* stream) {
    const int32_t K = K1 + K2;
    size_t need = 0;
    SPX_TRY(spx_dense_backward_weight_workspace_size(n, K, N, &need));
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_dense_backward_weight: workspace too small");
    if (!dW || (n > 0 && (!X1 || (K2 > 0 && !X2) || !G)))
        return set_error(SPX_INVALID_ARG, "spx_dense_backward_weight: NULL operand");
    cudaStream_t st = as_stream(stream);
    const int64_t parts = (n + WROWS - 1) / WROWS;
    const int outs = (K + 1) * N;
    if (parts == 0) {
        SPX_CUDA(cudaMemsetAsync(dW, 0, sizeof(float) * (size_t)K * N, st), "dense_bwd_weight memset");
        if (db) SPX_CUDA(cudaMemsetAsync(db, 0, sizeof(float) * (size_t)N, st), "dense_bwd_weight memset");
        return SPX_OK;
    }
    float* partial = static_cast<float*>(ws);
    dense_bwd_weight_kernel<<<(unsigned)parts, DT, 0, st>>>(n, X1, K1, X2, K2, G, N, partial);
    SPX_CHECK_LAUNCH("spx_dense_backward_weight");
    sum_partials_kernel<<<(unsigned)((outs + 255) / 256), 256, 0, st>>>((int)parts, outs, partial, K, N, dW, db);
    SPX_CHECK_LAUNCH("spx_dense_backward_weight sum");
    return SPX_OK;
}

extern "C" spx_status spx_relu_backward(int64_t count, const float* gh, const float* u, float* gu, void* stream) {
    if (count < 0 || (count > 0 && (!gh || !u || !gu))) return set_error(SPX_INVALID_ARG, "spx_relu_backward");
    if (count == 0) return SPX_OK;
    relu_backward_kernel<<<grid1(count, 256), 256, 0, as_stream(stream)>>>(count, gh, u, gu);
    SPX_CHECK_LAUNCH("spx_relu_backward");
    return SPX_OK;
}

extern "C" spx_status spx_tril_workspace_size(int32_t n, size_t* bytes) {
    if (!bytes || n < 0) return set_error(SPX_INVALID_ARG, "spx_tril_workspace_size");
    *bytes = (((size_t)n * 4 + 255) & ~size_t(255)) + scan_workspace_bytes<int32_t>(n);
    return SPX_OK;
}

extern "C" spx_status spx_tril_pattern(const spx_csr* A, int32_t* l_indptr, int32_t* l_indices, int32_t* l_src,
                                       int64_t* nnz_host, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, false, "spx_tril_pattern"));
    size_t need = 0;
    spx_tril_workspace_size(A->m, &need);
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_tril_pattern: workspace too small");
    if (!l_indptr || !nnz_host) return set_error(SPX_INVALID_ARG, "spx_tril_pattern: NULL output");
    cudaStream_t st = as_stream(stream);
    int32_t* cnt = static_cast<int32_t*>(ws);
    int32_t* sws = (int32_t*)(static_cast<char*>(ws) + (((size_t)A->m * 4 + 255) & ~size_t(255)));
    const unsigned g = (unsigned)((A->m + 255) / 256);
    if (A->m > 0) {
        tril_count_kernel<<<g, 256, 0, st>>>(A->m, A->indptr, A->indices, cnt);
        SPX_CHECK_LAUNCH("tril count");
    }
    SPX_TRY((scan_counts<int32_t, int32_t>(cnt, l_indptr, A->m, sws, st)));
    int32_t nnz = 0;
    SPX_CUDA(cudaMemcpyAsync(&nnz, l_indptr + A->m, sizeof(int32_t), cudaMemcpyDeviceToHost, st), "tril copy");
    SPX_CUDA(cudaStreamSynchronize(st), "tril sync");
    *nnz_host = nnz;
    if (l_indices && l_src && A->m > 0) {
        tril_fill_kernel<<<g, 256, 0, st>>>(A->m, A->indptr, A->indices, l_indptr, l_indices, l_src);
        SPX_CHECK_LAUNCH("tril fill");
    }
    return SPX_OK;
}

extern "C" spx_status spx_edge_forward(const spx_csr* Lpat, const float* e_low, const float* d, const float* P,
                                       const float* Q, const float* u, const float* c, const float* v,
                                       const float* bd, const float* bo, float* L_values, void* stream) {
    SPX_TRY(check_csr(Lpat, false, "spx_edge_forward"));
    if (Lpat->m == 0) return SPX_OK;
    if (!e_low || !d || !P || !Q || !u || !c || !v || !bd || !bo || !L_values)
        return set_error(SPX_INVALID_ARG, "spx_edge_forward: NULL operand");
    EdgeParams pr{u, c, v, bd, bo};
    edge_fwd_kernel<<<warp_grid(Lpat->m), 256, 0, as_stream(stream)>>>(Lpat->m, Lpat->indptr, Lpat->indices, e_low,
                                                                        d, P, Q, pr, L_values);
    SPX_CHECK_LAUNCH("spx_edge_forward");
    return SPX_OK;
}

extern "C" spx_status spx_edge_backward_workspace_size(int32_t n, size_t* bytes) {
    if (!bytes || n < 0) return set_error(SPX_INVALID_ARG, "spx_edge_backward_workspace_size");
    const int64_t warps = ((int64_t)n + EB_ROWS - 1) / EB_ROWS;
    *bytes = (size_t)(warps > 0 ? warps : 1) * EB_PART * 4 + 256;
    return SPX_OK;
}

// gparams: device float[3*64 + 2] = [gv (64), gc (64), gu (64), gbd, gbo]
extern "C" spx_status spx_edge_backward(const spx_csr* Lpat, const int32_t* lt_indptr, const int32_t* lt_indices,
                                        const int32_t* lt_perm, const float* e_low, const float* d, const float* P,
                                        const float* Q, const float* u, const float* c, const float* v,
                                        const float* bd, const float* bo, const float* gL, float* gP, float* gQ,
                                        float* gparams, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(Lpat, false, "spx_edge_backward"));
    size_t need = 0;
    spx_edge_backward_workspace_size(Lpat->m, &need);
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_edge_backward: workspace too small");
    if (Lpat->m == 0) return SPX_OK;
    if (!lt_indptr || !e_low || !d || !P || !Q || !gL || !gP || !gQ || !gparams)
        return set_error(SPX_INVALID_ARG, "spx_edge_backward: NULL operand");
    cudaStream_t st = as_stream(stream);
    EdgeParams pr{u, c, v, bd, bo};
    const int64_t warps = ((int64_t)Lpat->m + EB_ROWS - 1) / EB_ROWS;
    float* partial = static_cast<float*>(ws);
    edge_bwd_rows_kernel<<<warp_grid(warps), 256, 0, st>>>(Lpat->m, Lpat->indptr, Lpat->indices, e_low, d, P, Q, pr,
                                                            gL, gP, partial);
    SPX_CHECK_LAUNCH("edge bwd rows");
    edge_bwd_cols_kernel<<<warp_grid(Lpat->m), 256, 0, st>>>(Lpat->m, lt_indptr, lt_indices, lt_perm, e_low, d, P, Q,
                                                              pr, gL, gQ);
    SPX_CHECK_LAUNCH("edge bwd cols");
    edge_sum_partials_kernel<<<1, 256, 0, st>>>(warps, partial, gparams);
    SPX_CHECK_LAUNCH("edge bwd sum");
    return SPX_OK;
}

extern "C" spx_status spx_adam_step(int64_t count, float* params, const float* grads, float* m, float* v,
                                    int32_t step, float lr, float beta1, float beta2, float eps, void* params_bf16,
                                    void* stream) {
    if (count < 0 || step < 1 || (count > 0 && (!params || !grads || !m || !v)))
        return set_error(SPX_INVALID_ARG, "spx_adam_step: bad arguments");
    if (count == 0) return SPX_OK;
    // Bias corrections in double on the host, rounded once: 1 - beta2^t is small for small t,
    // so a float power would carry its rounding error into every update at 1/(1 - beta2^t).
    const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
    adam_kernel<<<grid1(count, 256), 256, 0, as_stream(stream)>>>(count, params, grads, m, v, lr, beta1, beta2, eps, c1,
                                                                   c2, static_cast<__nv_bfloat16*>(params_bf16));
    SPX_CHECK_LAUNCH("spx_adam_step");
    return SPX_OK;
}

extern "C" spx_status spx_to_bf16(int64_t count, const float* src, void* dst, void* stream) {
    if (count < 0 || (count > 0 && (!src || !dst))) return set_error(SPX_INVALID_ARG, "spx_to_bf16");
    if (count == 0) return SPX_OK;
    to_bf16_kernel<<<grid1(count, 256), 256, 0, as_stream(stream)>>>(count, src, static_cast<__nv_bfloat16*>(dst));
    SPX_CHECK_LAUNCH("spx_to_bf16");
    return SPX_OK;
}
