// Boundary conveniences around the solver and the row-wise products:
//   spx_precond_apply   z = M r for the preconditioners of spx_cg_batched, outside the solver
//                       (Jacobi, L L^T, an explicit M, IC(0) by two triangular solves);
//   spx_cg_adjoint      the SpSolve VJP of Table 1 in one call: lambda = A^-T g by the same
//                       PCG (A symmetric), grad_A = -(lambda x^T) on mask(A);
//   spx_spmm_autotune   the launch parameters of spx_spmm chosen by timing on the device;
//   spx_sync_status     per-system status words read back to the host.
// Each is composed from the library's own entry points and kernels.
#include <float.h>
#include <string.h>

#include "common.cuh"

namespace spx {
namespace {

__global__ void scale_copy_kernel(int64_t n, const float* __restrict__ d, const float* __restrict__ r,
                                  float* __restrict__ z) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) z[i] = d ? d[i] * r[i] : r[i];
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_precond_apply(int32_t pc_kind, int64_t n, const float* r, float* z, const float* pc_diag_inv,
                                        const spx_csr* L, const spx_csr* LT, int32_t nsys,
                                        const int32_t* const* ic0_levels, float* tmp, void* stream) {
    if (n < 0 || (n > 0 && (!r || !z))) return set_error(SPX_INVALID_ARG, "spx_precond_apply: NULL vector");
    if (n == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    switch (pc_kind) {
        case 0:
        case 1: {
            if (pc_kind == 1 && !pc_diag_inv) return set_error(SPX_INVALID_ARG, "spx_precond_apply: Jacobi needs D^-1");
            int64_t blocks = (n + 255) / 256;
            const int64_t cap = (int64_t)num_sms() * 16;
            scale_copy_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, st>>>(
                n, pc_kind == 1 ? pc_diag_inv : nullptr, r, z);
            SPX_CHECK_LAUNCH("spx_precond_apply");
            return SPX_OK;
        }
        case 2:                                            // z = L (L^T r)
            if (!L || !LT || !tmp) return set_error(SPX_INVALID_ARG, "spx_precond_apply: L L^T needs L, L^T and tmp");
            SPX_TRY(spx_spmm(LT, r, 1, 1, tmp, 1, 1.f, 0.f, nullptr, nullptr, 0, stream));
            return spx_spmm(L, tmp, 1, 1, z, 1, 1.f, 0.f, nullptr, nullptr, 0, stream);
        case 3:                                            // z = M r, M passed as L
            if (!L) return set_error(SPX_INVALID_ARG, "spx_precond_apply: an explicit M is passed as L");
            return spx_spmm(L, r, 1, 1, z, 1, 1.f, 0.f, nullptr, nullptr, 0, stream);
        case 4:                                            // z = L^-T (L^-1 r)
            if (!L || !LT || !tmp || !ic0_levels || !ic0_levels[0] || !ic0_levels[1] || !ic0_levels[2])
                return set_error(SPX_INVALID_ARG, "spx_precond_apply: IC(0) needs L, L^T, levels and tmp");
            SPX_TRY(spx_sptrsv(L, 0, nsys, ic0_levels[0], ic0_levels[1], ic0_levels[2], r, tmp, nullptr, stream));
            return spx_sptrsv(LT, 1, nsys, ic0_levels[0], ic0_levels[1], ic0_levels[2], tmp, z, nullptr, stream);
        default:
            return set_error(SPX_INVALID_ARG, "spx_precond_apply: unknown preconditioner %d", pc_kind);
    }
}

extern "C" spx_status spx_cg_adjoint(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys, const int32_t* order,
                                     const double* x, const float* g, double* lambda, float* grad_A, int32_t pc_kind,
                                     const float* pc_diag_inv, const spx_csr* L, const spx_csr* LT,
                                     const int32_t* const* ic0_levels, double tol, int32_t maxit, double delta,
                                     int32_t* iters, int32_t* status, double* relres, void* ws, size_t ws_bytes,
                                     void* stream) {
    if (grad_A && A && A->nnz > 0 && !x) return set_error(SPX_INVALID_ARG, "spx_cg_adjoint: grad_A needs x");
    SPX_TRY(spx_cg_batched(A, sys_ptr, nsys, order, g, lambda, pc_kind, pc_diag_inv, L, LT, ic0_levels, tol, maxit,
                           delta, iters, status, relres, ws, ws_bytes, stream));
    if (grad_A) SPX_TRY(spx_masked_outer_f64(A, lambda, x, -1.0, grad_A, stream));
    return SPX_OK;
}

extern "C" spx_status spx_spmm_autotune(const spx_csr* A, const float* X, int64_t ldx, int32_t k, float* Y,
                                        int64_t ldy, spx_rowplan* plan, float* best_ms, void* stream) {
    if (!plan || !best_ms) return set_error(SPX_INVALID_ARG, "spx_spmm_autotune: NULL plan or output");
    SPX_TRY(check_csr(A, true, "spx_spmm_autotune"));
    cudaStream_t st = as_stream(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPX_CUDA(cudaEventCreate(&e0), "spx_spmm_autotune event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(SPX_CUDA_ERROR, "spx_spmm_autotune: event");
    }
    const int rpgs[] = {1, 2, 4, 8};
    const bool vec4 = k % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
    float best = FLT_MAX;
    spx_rowplan keep = *plan;
    spx_status rc = SPX_OK;
    for (int eng = 0; eng < (vec4 ? 2 : 1) && rc == SPX_OK; ++eng) {
        for (int rpg : rpgs) {
            spx_rowplan p = *plan;
            p.col_block = 0;                               // one pass over all k (the measured best)
            p.rows_per_group = rpg;
            p.engine = eng;
            rc = spx_spmm(A, X, ldx, k, Y, ldy, 1.f, 0.f, &p, nullptr, 0, stream);   // warm-up
            if (rc != SPX_OK) break;
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < 3 && rc == SPX_OK; ++rep)
                rc = spx_spmm(A, X, ldx, k, Y, ldy, 1.f, 0.f, &p, nullptr, 0, stream);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = set_error(SPX_CUDA_ERROR, "spx_spmm_autotune: timing");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            if (rc == SPX_OK && ms < best) {
                best = ms;
                keep = p;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPX_OK) return rc;
    *plan = keep;
    *best_ms = best;
    return SPX_OK;
}

extern "C" spx_status spx_sync_status(const int32_t* status_dev, int32_t n, int32_t* status_host, void* stream) {
    if (n < 0 || (n > 0 && (!status_dev || !status_host)))
        return set_error(SPX_INVALID_ARG, "spx_sync_status: bad arguments");
    cudaStream_t st = as_stream(stream);
    if (n > 0)
        SPX_CUDA(cudaMemcpyAsync(status_host, status_dev, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
                 "spx_sync_status copy");
    SPX_TRY(spx_check_device(stream));                     // synchronizes; reports an expired device wait
    for (int32_t i = 0; i < n; ++i)
        if (status_host[i] != SPX_OK)
            return set_error((spx_status)status_host[i], "spx_sync_status: entry %d is %s", i,
                             spx_status_name(status_host[i]));
    return SPX_OK;
}
