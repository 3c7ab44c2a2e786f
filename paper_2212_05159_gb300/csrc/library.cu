// Library-wide entry points: error reporting, status names, version, CSR validation.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "common.cuh"

namespace spx {

__device__ int g_spx_device_error = 0;

int* device_error_word() {
    static int* cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!cached[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_spx_device_error) != cudaSuccess) return nullptr;
        cached[dev] = static_cast<int*>(p);
    }
    return cached[dev];
}

static thread_local char g_msg[512] = "";

spx_status set_error(spx_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
    return st;
}

spx_status cuda_error(cudaError_t err, const char* where) {
    return set_error(SPX_CUDA_ERROR, "%s: %s (%s)", where, cudaGetErrorName(err),
                     cudaGetErrorString(err));
}

int num_sms() {
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            n > 0)
            cached = n;
        else
            cached = NUM_SMS_GB300;
    }
    return cached;
}

spx_status check_csr(const spx_csr* A, bool need_values, const char* who) {
    if (!A) return set_error(SPX_INVALID_ARG, "%s: NULL matrix", who);
    if (A->m < 0 || A->n < 0 || A->nnz < 0 || A->nnz >= (int64_t(1) << 31))
        return set_error(SPX_INVALID_ARG, "%s: bad sizes m=%d n=%d nnz=%lld", who, A->m, A->n,
                         (long long)A->nnz);
    if (!A->indptr) return set_error(SPX_INVALID_ARG, "%s: NULL indptr", who);
    if (A->nnz > 0 && !A->indices) return set_error(SPX_INVALID_ARG, "%s: NULL indices", who);
    if (need_values && A->nnz > 0 && !A->values)
        return set_error(SPX_INVALID_ARG, "%s: NULL values", who);
    return SPX_OK;
}

// Bit 0: pattern error (range / monotonicity); bit 1: unsorted or duplicate columns.
__global__ void validate_kernel(int32_t m, int32_t n, int64_t nnz, const int32_t* __restrict__ indptr,
                                const int32_t* __restrict__ indices, int* __restrict__ flags) {
    int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        if (indptr[0] != 0 || (int64_t)indptr[m] != nnz) atomicOr(flags, 1);
    }
    for (int64_t i = tid; i < m; i += stride) {
        int a = indptr[i], b = indptr[i + 1];
        if (a > b || a < 0 || (int64_t)b > nnz) {
            atomicOr(flags, 1);
            continue;
        }
        int prev = -1;
        for (int e = a; e < b; ++e) {
            int j = indices[e];
            if (j < 0 || j >= n) {
                atomicOr(flags, 1);
                break;
            }
            if (j <= prev) atomicOr(flags, 2);
            prev = j;
        }
    }
}

}  // namespace spx

using namespace spx;

extern "C" const char* spx_last_error(void) { return g_msg; }

extern "C" const char* spx_status_name(int s) {
    switch (s) {
        case SPX_OK: return "SPX_OK";
        case SPX_INVALID_ARG: return "SPX_INVALID_ARG";
        case SPX_BAD_PATTERN: return "SPX_BAD_PATTERN";
        case SPX_UNSORTED: return "SPX_UNSORTED";
        case SPX_OOM_WORKSPACE: return "SPX_OOM_WORKSPACE";
        case SPX_MAXITER: return "SPX_MAXITER";
        case SPX_BREAKDOWN: return "SPX_BREAKDOWN";
        case SPX_NONFINITE: return "SPX_NONFINITE";
        case SPX_DEVICE_TIMEOUT: return "SPX_DEVICE_TIMEOUT";
        case SPX_CUDA_ERROR: return "SPX_CUDA_ERROR";
        case SPX_NOT_SUPPORTED: return "SPX_NOT_SUPPORTED";
        default: return "SPX_UNKNOWN";
    }
}

extern "C" int32_t spx_version(void) { return 200; }

extern "C" spx_status spx_csr_validate(const spx_csr* A, void* ws, size_t ws_bytes,
                                       void* stream) {
    SPX_TRY(check_csr(A, false, "spx_csr_validate"));
    if (!ws || ws_bytes < 16) return set_error(SPX_OOM_WORKSPACE, "spx_csr_validate: workspace < 16 B");
    cudaStream_t st = as_stream(stream);
    int* flags = static_cast<int*>(ws);
    SPX_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), st), "spx_csr_validate memset");
    int threads = 256;
    int64_t blocks = ((int64_t)A->m + threads - 1) / threads;
    if (blocks < 1) blocks = 1;
    if (blocks > 4 * num_sms() * 8) blocks = 4 * num_sms() * 8;
    validate_kernel<<<(unsigned)blocks, threads, 0, st>>>(A->m, A->n, A->nnz, A->indptr,
                                                          A->indices, flags);
    SPX_CHECK_LAUNCH("spx_csr_validate");
    int h = 0;
    SPX_CUDA(cudaMemcpyAsync(&h, flags, sizeof(int), cudaMemcpyDeviceToHost, st),
             "spx_csr_validate copy");
    SPX_CUDA(cudaStreamSynchronize(st), "spx_csr_validate sync");
    if (h & 1) return set_error(SPX_BAD_PATTERN, "spx_csr_validate: indptr/indices out of range");
    if (h & 2) return set_error(SPX_UNSORTED, "spx_csr_validate: columns not strictly increasing");
    return SPX_OK;
}

extern "C" spx_status spx_check_device(void* stream) {
    cudaStream_t st = as_stream(stream);
    SPX_CUDA(cudaStreamSynchronize(st), "spx_check_device sync");
    int h = 0, zero = 0;
    SPX_CUDA(cudaMemcpyFromSymbol(&h, g_spx_device_error, sizeof(int)), "spx_check_device read");
    if (h) {
        SPX_CUDA(cudaMemcpyToSymbol(g_spx_device_error, &zero, sizeof(int)), "spx_check_device clear");
        return set_error(SPX_DEVICE_TIMEOUT, "a bounded device-side wait ran out (flags 0x%x)", h);
    }
    return SPX_OK;
}
