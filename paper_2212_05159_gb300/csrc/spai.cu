// Pieces of the sparse approximate inverse by gradient descent (Section 4.6):
//   loss(M) = ||I - M A||_F^2 over the stored entries of M (mask(M) = mask(A)),
//   grad    = -2 mask_M((I - M A) A^T)   (Table 1, SpSpMM w.r.t. the first operand),
// with C = M A, the gradient and d A all formed by the library's SpGEMM kernels.  This file
// adds what is specific to the method:
//   * spx_spai_residual: scale * (I - C) on C's pattern (scale = -2 gives the upstream
//     gradient of the loss with respect to C's values), and the number of diagonal entries
//     present in C's pattern;
//   * spx_dot: a deterministic inner product (FP32 inputs, double-float per thread, FP64
//     across threads and blocks, fixed order), result left on the device;
//   * spx_spai_update: the exact line-search step along -grad, m -= (1/2) (g.g) / (gA.gA) g,
//     with both inner products read on the device (no host round trip).
#include "common.cuh"

namespace spx {
namespace {

constexpr int DOT_THREADS = 256;
constexpr int DOT_BLOCKS_PER_SM = 4;

struct DFs {
    float hi, lo;
};

__device__ __forceinline__ void dfs_add_prod(DFs& s, float a, float b) {
    const float ph = a * b;
    const float pl = fmaf(a, b, -ph);          // a*b = ph + pl exactly
    const float t = s.hi + ph;
    const float bp = t - s.hi;
    const float err = (s.hi - (t - bp)) + (ph - bp);
    s.hi = t;
    s.lo += err + pl;
}

// One warp per row: out_e = scale * ([i == j] - c_e); diagonal entries counted per warp.
__global__ void spai_residual_kernel(int32_t m, const int32_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                                     const float* __restrict__ c, float scale, float* __restrict__ out,
                                     int* __restrict__ diag_count) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int found = 0;
    for (int64_t i = warp; i < m; i += nwarps) {
        const int a = indptr[i], b = indptr[i + 1];
        for (int e = a + lane; e < b; e += 32) {
            const bool d = indices[e] == (int32_t)i;
            found += d ? 1 : 0;
            out[e] = scale * ((d ? 1.f : 0.f) - c[e]);
        }
    }
    if (diag_count) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) found += __shfl_xor_sync(FULL, found, o);
        if (lane == 0 && found) atomicAdd(diag_count, found);      // integer: order-independent
    }
}

// Stage 1: block b sums a fixed grid-stride subset in double-float, then FP64 over its warps.
__global__ void __launch_bounds__(DOT_THREADS) dot_partial_kernel(int64_t n, const float* __restrict__ x,
                                                                  const float* __restrict__ y, double* __restrict__ part) {
    __shared__ double red[DOT_THREADS / 32];
    DFs s{0.f, 0.f};
    const int64_t stride = (int64_t)gridDim.x * DOT_THREADS;
    for (int64_t i = blockIdx.x * (int64_t)DOT_THREADS + threadIdx.x; i < n; i += stride)
        dfs_add_prod(s, x[i], y[i]);
    double v = (double)s.hi + (double)s.lo;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < DOT_THREADS / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Stage 2: one thread adds the block partials in block order.
__global__ void dot_final_kernel(int nb, const double* __restrict__ part, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += part[b];
        *out = t;
    }
}

int dot_blocks(int64_t n) {
    const int64_t want = (n + DOT_THREADS * 8 - 1) / (DOT_THREADS * 8);
    const int64_t cap = (int64_t)DOT_BLOCKS_PER_SM * num_sms();
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

__global__ void spai_update_kernel(int64_t nnz, float* __restrict__ m, const float* __restrict__ g,
                                   const double* __restrict__ gg, const double* __restrict__ dada) {
    const double num = *gg, den = *dada;
    if (!(den > 0.0) || !isfinite(num) || !isfinite(den)) return;      // no step along a null direction
    const float eta = (float)(0.5 * num / den);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += stride)
        m[i] = fmaf(-eta, g[i], m[i]);
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_spai_residual(const spx_csr* C, float scale, float* out, int32_t* diag_count,
                                        void* stream) {
    SPX_TRY(check_csr(C, true, "spx_spai_residual"));
    if (C->nnz > 0 && !out) return set_error(SPX_INVALID_ARG, "spx_spai_residual: NULL output");
    cudaStream_t st = as_stream(stream);
    if (diag_count) SPX_CUDA(cudaMemsetAsync(diag_count, 0, sizeof(int32_t), st), "spx_spai_residual memset");
    if (C->m == 0) return SPX_OK;
    const int64_t warps = C->m;
    int64_t blocks = (warps * 32 + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    spai_residual_kernel<<<(unsigned)blocks, 256, 0, st>>>(C->m, C->indptr, C->indices, C->values, scale, out,
                                                           reinterpret_cast<int*>(diag_count));
    SPX_CHECK_LAUNCH("spx_spai_residual");
    return SPX_OK;
}

extern "C" spx_status spx_dot_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 0) return set_error(SPX_INVALID_ARG, "spx_dot_workspace_size: bad arguments");
    *bytes = (size_t)dot_blocks(n) * sizeof(double);
    return SPX_OK;
}

extern "C" spx_status spx_dot(int64_t n, const float* x, const float* y, double* out, void* ws, size_t ws_bytes,
                              void* stream) {
    if (n < 0 || !out || (n > 0 && (!x || !y))) return set_error(SPX_INVALID_ARG, "spx_dot: bad arguments");
    const int nb = dot_blocks(n);
    if (!ws || ws_bytes < (size_t)nb * sizeof(double))
        return set_error(SPX_OOM_WORKSPACE, "spx_dot: workspace %zu < %zu", ws_bytes, (size_t)nb * sizeof(double));
    cudaStream_t st = as_stream(stream);
    double* part = static_cast<double*>(ws);
    dot_partial_kernel<<<nb, DOT_THREADS, 0, st>>>(n, x, y, part);
    SPX_CHECK_LAUNCH("spx_dot partial");
    dot_final_kernel<<<1, 32, 0, st>>>(nb, part, out);
    SPX_CHECK_LAUNCH("spx_dot final");
    return SPX_OK;
}

extern "C" spx_status spx_spai_update(int64_t nnz, float* m, const float* g, const double* gg, const double* dada,
                                      void* stream) {
    if (nnz < 0 || !gg || !dada || (nnz > 0 && (!m || !g)))
        return set_error(SPX_INVALID_ARG, "spx_spai_update: bad arguments");
    if (nnz == 0) return SPX_OK;
    int64_t blocks = (nnz + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    spai_update_kernel<<<(unsigned)blocks, 256, 0, as_stream(stream)>>>(nnz, m, g, gg, dada);
    SPX_CHECK_LAUNCH("spx_spai_update");
    return SPX_OK;
}
