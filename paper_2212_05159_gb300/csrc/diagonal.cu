// The diagonal of a CSR matrix as a differentiable read (the paper's A.diagonal(), used to
// build Jacobi-type operators from sparse values, Section 4.1): d_i = a_ii (0 where row i
// stores no diagonal entry), and its vector-Jacobian product, which puts g_i on the
// stored entry (i, i) of the values gradient -- a gradient on A's own pattern.
#include "common.cuh"

namespace spx {
namespace {

// One thread per row; the row's columns are sorted, so the diagonal is found by binary
// search.  pos[i] = index of entry (i, i) in indices / values, or -1.
__global__ void csr_diagonal_kernel(int32_t nd, const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                                    const float* __restrict__ val, float* __restrict__ diag,
                                    int32_t* __restrict__ pos) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nd) return;
    int lo = ptr[i], hi = ptr[i + 1];
    int at = -1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int j = idx[mid];
        if (j == (int)i) {
            at = mid;
            break;
        }
        if (j < (int)i) lo = mid + 1;
        else hi = mid;
    }
    if (pos) pos[i] = at;
    if (diag) diag[i] = at >= 0 ? val[at] : 0.f;
}

__global__ void diagonal_backward_kernel(int32_t nd, const int32_t* __restrict__ pos, const float* __restrict__ g,
                                         float* __restrict__ gv) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nd) return;
    const int p = pos[i];
    if (p >= 0) gv[p] += g[i];
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_csr_diagonal(const spx_csr* A, float* diag, int32_t* pos, void* stream) {
    SPX_TRY(check_csr(A, diag != nullptr, "spx_csr_diagonal"));
    const int32_t nd = A->m < A->n ? A->m : A->n;
    if (nd == 0 || (!diag && !pos)) return SPX_OK;
    csr_diagonal_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, as_stream(stream)>>>(nd, A->indptr, A->indices,
                                                                                    A->values, diag, pos);
    SPX_CHECK_LAUNCH("spx_csr_diagonal");
    return SPX_OK;
}

extern "C" spx_status spx_diagonal_backward(int32_t nd, const int32_t* pos, const float* g_diag, float* g_values,
                                            void* stream) {
    if (nd < 0 || (nd > 0 && (!pos || !g_diag || !g_values)))
        return set_error(SPX_INVALID_ARG, "spx_diagonal_backward: bad arguments");
    if (nd == 0) return SPX_OK;
    diagonal_backward_kernel<<<(unsigned)((nd + 255) / 256), 256, 0, as_stream(stream)>>>(nd, pos, g_diag, g_values);
    SPX_CHECK_LAUNCH("spx_diagonal_backward");
    return SPX_OK;
}
