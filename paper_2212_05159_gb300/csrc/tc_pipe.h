// Internal interface of the pipelined tensor-core kernel (tc_pipe.cu) for the entry points
// of tc_dense.cu.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spx.h"

namespace spx {

// True while the pipelined kernel is enabled (spx_tc_set_pipeline; on by default).
bool tc_pipe_enabled();

// Launch the pipelined kernel when the shapes suit it; *launched tells whether it did.
// Shapes it takes: K1 (and K2, if any) multiples of 32 with K1 + K2 <= 128, N a multiple
// of 32 in 32..128 (mode 4: N / 2 a multiple of 32), n < 2^31 - 128.  Arguments as in
// spx_dense_forward_tc, already validated.
spx_status tc_pipe_forward(int64_t n, const float* X1, int K1, const float* X2, int K2, const __nv_bfloat16* W,
                           const float* bias, int N, int mode, const float* Hin, float* Y, float* U, cudaStream_t st,
                           bool* launched);

// As above for the data gradient [dX1 dX2] (+)= G W^T: N, K1 and K2 (if any) multiples of
// 32, N <= 128, K1 + K2 <= 128.  Arguments as in spx_dense_backward_data_tc, validated.
spx_status tc_pipe_bwd_data(int64_t n, const float* G, int N, const __nv_bfloat16* W, int K1, int K2, float* dX1,
                            float* dX2, int accumulate, cudaStream_t st, bool* launched);

}  // namespace spx
