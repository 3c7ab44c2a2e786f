// Column-block slabs of a row-major dense operand.
//
// A gather kernel that reads rows of a dense n x k operand at random keeps the touched
// data in L2 only if the data is dense in cache lines: L2 allocates whole 128-byte lines,
// so a column block of a row-major array (a few sectors per row) costs as much L2 as the
// full array.  When a caller asks for column blocks narrower than k, the operand is
// repacked once into column-block-major slabs -- slab b holds columns [b*cb, b*cb + cb) of
// every row, contiguously, row stride cb -- and each pass of the gather kernel reads one
// slab.  On GB300 one pass over all k columns was the fastest choice on every workload
// measured (power-law and stencil matrices, k = 32 to 128), so blocks are opt-in: the
// default is one pass.
#pragma once

#include "common.cuh"

namespace spx {
namespace {  // internal linkage: every translation unit gets its own copy

// Number of slabs and bytes of the repacked copy (0 when no repacking applies).
inline int32_t slab_count(int32_t k, int32_t cb) { return (k + cb - 1) / cb; }
inline size_t slab_bytes(int64_t rows, int32_t k, int32_t cb) {
    if (cb >= k || cb % 4 != 0 || k % 4 != 0) return 0;
    return (size_t)slab_count(k, cb) * (size_t)rows * (size_t)cb * 4;
}

// Xb[b][j][0..cb) = X[j][b*cb .. b*cb + cb) (float4 copies; k, cb, ldx multiples of 4).
__global__ void __launch_bounds__(256) slab_repack_kernel(int64_t rows, const float* __restrict__ X, int64_t ldx,
                                                          int32_t k, int32_t cb, float* __restrict__ Xb) {
    const int64_t k4 = k / 4;
    const int64_t total = rows * k4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += stride) {
        const int64_t j = t / k4;
        const int32_t col = (int32_t)(t - j * k4) * 4;
        const int32_t b = col / cb;
        const int32_t cc = col - b * cb;
        float4 v = __ldcs(reinterpret_cast<const float4*>(X + j * ldx + col));
        *reinterpret_cast<float4*>(Xb + ((int64_t)b * rows + j) * cb + cc) = v;
    }
}

inline spx_status slab_repack(int64_t rows, const float* X, int64_t ldx, int32_t k, int32_t cb, float* Xb,
                              cudaStream_t st) {
    const int64_t total = rows * (k / 4);
    if (total == 0) return SPX_OK;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    slab_repack_kernel<<<(unsigned)blocks, 256, 0, st>>>(rows, X, ldx, k, cb, Xb);
    SPX_CHECK_LAUNCH("slab_repack");
    return SPX_OK;
}

}  // namespace
}  // namespace spx
