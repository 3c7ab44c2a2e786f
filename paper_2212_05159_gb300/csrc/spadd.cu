// Sparse + sparse (Section 3.1.4):  C = alpha A + beta B with mask(C) = mask(A) U mask(B),
// and its gradients alpha V on mask(A), beta V on mask(B) (Table 1, Sp + Sp).
//
// The pattern of C depends on the patterns only, so it is built once per pair:
//   symbolic  one thread per row merges the two sorted rows and counts the union; a
//             device-wide scan (64-bit, checked against the int32 index range) gives
//             C's row offsets;
//   fill      the same merge writes C's columns and two maps in each direction: for every
//             entry of C the entry of A (and of B) it takes its value from (-1 if none),
//             and for every entry of A (of B) its position in C.
// Then, per call, every value is written once by exactly one thread, in a fixed order:
//   numeric   c[e] = alpha a[src_a[e]] + beta b[src_b[e]]   (absent terms skipped)
//   backward  ga[e] = alpha gc[pos_a[e]],  gb[e] = beta gc[pos_b[e]]
// Structural union: an entry stored in A or B stays in C even when its value cancels.
#include <limits.h>

#include "common.cuh"
#include "scan.cuh"

namespace spx {
namespace {

__global__ void spadd_count_kernel(int32_t m, const int32_t* __restrict__ ap, const int32_t* __restrict__ ai,
                                   const int32_t* __restrict__ bp, const int32_t* __restrict__ bi,
                                   int32_t* __restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    int ea = ap[i], eb = bp[i];
    const int fa = ap[i + 1], fb = bp[i + 1];
    int c = 0;
    while (ea < fa && eb < fb) {
        const int ja = ai[ea], jb = bi[eb];
        ea += ja <= jb;
        eb += jb <= ja;
        ++c;
    }
    cnt[i] = c + (fa - ea) + (fb - eb);
}

__global__ void spadd_fill_kernel(int32_t m, const int32_t* __restrict__ ap, const int32_t* __restrict__ ai,
                                  const int32_t* __restrict__ bp, const int32_t* __restrict__ bi,
                                  const int32_t* __restrict__ cp, int32_t* __restrict__ ci,
                                  int32_t* __restrict__ src_a, int32_t* __restrict__ src_b,
                                  int32_t* __restrict__ pos_a, int32_t* __restrict__ pos_b) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    int ea = ap[i], eb = bp[i], ec = cp[i];
    const int fa = ap[i + 1], fb = bp[i + 1];
    while (ea < fa || eb < fb) {
        const int ja = ea < fa ? ai[ea] : INT_MAX;
        const int jb = eb < fb ? bi[eb] : INT_MAX;
        const int j = ja < jb ? ja : jb;
        ci[ec] = j;
        if (ja == j) {
            src_a[ec] = ea;
            pos_a[ea] = ec;
            ++ea;
        } else {
            src_a[ec] = -1;
        }
        if (jb == j) {
            src_b[ec] = eb;
            pos_b[eb] = ec;
            ++eb;
        } else {
            src_b[ec] = -1;
        }
        ++ec;
    }
}

__global__ void to_int32_kernel(int64_t n, const int64_t* __restrict__ in, int32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)in[i];
}

__global__ void spadd_numeric_kernel(int64_t nnz, float alpha, const float* __restrict__ av,
                                     const int32_t* __restrict__ sa, float beta, const float* __restrict__ bv,
                                     const int32_t* __restrict__ sb, float* __restrict__ cv) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t a = sa[e], b = sb[e];
        float v = 0.f;
        if (a >= 0) v = alpha * av[a];
        if (b >= 0) v += beta * bv[b];
        cv[e] = v;
    }
}

__global__ void gather_scaled_kernel(int64_t n, float s, const float* __restrict__ g, const int32_t* __restrict__ pos,
                                     float* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += stride) out[e] = s * g[pos[e]];
}

unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

size_t spadd_ws(int32_t m) {
    const size_t cnt = ((size_t)m * 4 + 255) & ~size_t(255);
    const size_t off = (((size_t)m + 1) * 8 + 255) & ~size_t(255);
    return cnt + off + scan_workspace_bytes<int64_t>(m);
}

spx_status check_pair(const spx_csr* A, const spx_csr* B, const char* who) {
    SPX_TRY(check_csr(A, false, who));
    SPX_TRY(check_csr(B, false, who));
    if (A->m != B->m || A->n != B->n) return set_error(SPX_INVALID_ARG, "%s: shapes differ", who);
    return SPX_OK;
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_spadd_workspace_size(int32_t m, size_t* bytes) {
    if (!bytes || m < 0) return set_error(SPX_INVALID_ARG, "spx_spadd_workspace_size: bad arguments");
    *bytes = spadd_ws(m);
    return SPX_OK;
}

extern "C" spx_status spx_spadd_symbolic(const spx_csr* A, const spx_csr* B, int32_t* c_indptr, int64_t* nnz_c,
                                         void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_pair(A, B, "spx_spadd_symbolic"));
    if (!c_indptr || !nnz_c) return set_error(SPX_INVALID_ARG, "spx_spadd_symbolic: NULL output");
    const size_t need = spadd_ws(A->m);
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_spadd_symbolic: workspace %zu < %zu", ws_bytes, need);
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    int32_t* cnt = reinterpret_cast<int32_t*>(w);
    int64_t* off = reinterpret_cast<int64_t*>(w + (((size_t)A->m * 4 + 255) & ~size_t(255)));
    int64_t* sws = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(off) + ((((size_t)A->m + 1) * 8 + 255) & ~size_t(255)));
    *nnz_c = 0;
    if (A->m == 0) {
        SPX_CUDA(cudaMemsetAsync(c_indptr, 0, sizeof(int32_t), st), "spx_spadd_symbolic memset");
        return SPX_OK;
    }
    spadd_count_kernel<<<(unsigned)((A->m + 255) / 256), 256, 0, st>>>(A->m, A->indptr, A->indices, B->indptr,
                                                                        B->indices, cnt);
    SPX_CHECK_LAUNCH("spx_spadd_symbolic count");
    SPX_TRY((scan_counts<int32_t, int64_t>(cnt, off, A->m, sws, st)));
    int64_t tot = 0;
    SPX_CUDA(cudaMemcpyAsync(&tot, off + A->m, sizeof(int64_t), cudaMemcpyDeviceToHost, st), "spx_spadd_symbolic copy");
    SPX_CUDA(cudaStreamSynchronize(st), "spx_spadd_symbolic sync");
    if (tot >= (int64_t(1) << 31))
        return set_error(SPX_INVALID_ARG, "spx_spadd_symbolic: nnz(C) = %lld exceeds the int32 index range",
                         (long long)tot);
    to_int32_kernel<<<(unsigned)((A->m + 1 + 255) / 256), 256, 0, st>>>(A->m + 1, off, c_indptr);
    SPX_CHECK_LAUNCH("spx_spadd_symbolic offsets");
    *nnz_c = tot;
    return SPX_OK;
}

extern "C" spx_status spx_spadd_fill(const spx_csr* A, const spx_csr* B, const int32_t* c_indptr, int32_t* c_indices,
                                     int32_t* src_a, int32_t* src_b, int32_t* pos_a, int32_t* pos_b, void* stream) {
    SPX_TRY(check_pair(A, B, "spx_spadd_fill"));
    if (!c_indptr || (A->m > 0 && (A->nnz + B->nnz > 0) && (!c_indices || !src_a || !src_b)) ||
        (A->nnz > 0 && !pos_a) || (B->nnz > 0 && !pos_b))
        return set_error(SPX_INVALID_ARG, "spx_spadd_fill: NULL output");
    if (A->m == 0) return SPX_OK;
    spadd_fill_kernel<<<(unsigned)((A->m + 255) / 256), 256, 0, as_stream(stream)>>>(
        A->m, A->indptr, A->indices, B->indptr, B->indices, c_indptr, c_indices, src_a, src_b, pos_a, pos_b);
    SPX_CHECK_LAUNCH("spx_spadd_fill");
    return SPX_OK;
}

extern "C" spx_status spx_spadd_numeric(int64_t nnz_c, float alpha, const float* a_vals, const int32_t* src_a,
                                        float beta, const float* b_vals, const int32_t* src_b, float* c_vals,
                                        void* stream) {
    if (nnz_c < 0 || (nnz_c > 0 && (!src_a || !src_b || !c_vals)))
        return set_error(SPX_INVALID_ARG, "spx_spadd_numeric: bad arguments");
    if (nnz_c == 0) return SPX_OK;
    spadd_numeric_kernel<<<grid_for(nnz_c), 256, 0, as_stream(stream)>>>(nnz_c, alpha, a_vals, src_a, beta, b_vals,
                                                                         src_b, c_vals);
    SPX_CHECK_LAUNCH("spx_spadd_numeric");
    return SPX_OK;
}

extern "C" spx_status spx_spadd_backward(int64_t nnz_a, int64_t nnz_b, float alpha, float beta, const float* gc,
                                         const int32_t* pos_a, const int32_t* pos_b, float* ga, float* gb,
                                         void* stream) {
    if (nnz_a < 0 || nnz_b < 0 || ((nnz_a > 0 || nnz_b > 0) && !gc))
        return set_error(SPX_INVALID_ARG, "spx_spadd_backward: bad arguments");
    cudaStream_t st = as_stream(stream);
    if (ga && nnz_a > 0) {
        if (!pos_a) return set_error(SPX_INVALID_ARG, "spx_spadd_backward: NULL pos_a");
        gather_scaled_kernel<<<grid_for(nnz_a), 256, 0, st>>>(nnz_a, alpha, gc, pos_a, ga);
        SPX_CHECK_LAUNCH("spx_spadd_backward A");
    }
    if (gb && nnz_b > 0) {
        if (!pos_b) return set_error(SPX_INVALID_ARG, "spx_spadd_backward: NULL pos_b");
        gather_scaled_kernel<<<grid_for(nnz_b), 256, 0, st>>>(nnz_b, beta, gc, pos_b, gb);
        SPX_CHECK_LAUNCH("spx_spadd_backward B");
    }
    return SPX_OK;
}
