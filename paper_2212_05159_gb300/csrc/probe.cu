// Gather-bound probe: a measurement instrument for the products that gather dense rows
// through a sparse column stream (spx_spmm, spx_sddmm, spx_spmm_t).  It is not an
// operation of the paper.
//
// For every entry e of a column stream it reads row indices[e] of X -- k float32 columns,
// k / 4 lanes per row with 16-byte loads, the index stream evict-first and X evict-last
// in L2, exactly as the SpMM kernel's gathers -- and adds it to a per-lane sum.  There
// are no values, no row boundaries and no output rows, so its time is the floor for any
// kernel that gathers the same rows in the same order on this GPU: the rate at which the
// memory system delivers that access pattern.  Each lane group keeps U batches of 8
// entries in flight (8 U independent 16-byte loads per lane), and the next chunk's
// indices are loaded while the current chunk's rows are in flight.
#include "common.cuh"

namespace spx {
namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BATCH = 8;

template <int LPR, int U>
__global__ void __launch_bounds__(PROBE_THREADS) gather_probe_kernel(int64_t nnz, const int32_t* __restrict__ idx,
                                                                     int32_t n, const float* __restrict__ X,
                                                                     int64_t ldx, float* __restrict__ out) {
    constexpr int G = 32 / LPR;                         // lane groups per warp
    constexpr int CH = G * PROBE_BATCH * U;             // entries per warp chunk
    const int lane = threadIdx.x & 31;
    const int g = lane / LPR;
    const int c = lane % LPR;
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    const int64_t nwarps = (int64_t)gridDim.x * (PROBE_THREADS / 32);
    const int64_t w = ((int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x) >> 5;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int jn[U * PROBE_BATCH];
    int64_t base = w * CH;
#pragma unroll
    for (int t = 0; t < U * PROBE_BATCH; ++t) {
        const int64_t e = base + (int64_t)((t / PROBE_BATCH) * G + g) * PROBE_BATCH + t % PROBE_BATCH;
        jn[t] = e < nnz ? ld_hint(idx + e, pol_stream) : -1;
    }
    for (; base < nnz; base += nwarps * CH) {
        int jc[U * PROBE_BATCH];
#pragma unroll
        for (int t = 0; t < U * PROBE_BATCH; ++t) jc[t] = jn[t];
        const int64_t nb = base + nwarps * CH;
#pragma unroll
        for (int t = 0; t < U * PROBE_BATCH; ++t) {
            const int64_t e = nb + (int64_t)((t / PROBE_BATCH) * G + g) * PROBE_BATCH + t % PROBE_BATCH;
            jn[t] = e < nnz ? ld_hint(idx + e, pol_stream) : -1;
        }
#pragma unroll
        for (int t = 0; t < U * PROBE_BATCH; ++t) {
            const int j = jc[t];
            if (j >= 0 && j < n) {
                const float4 x = ld_hint4(X + (int64_t)j * ldx + 4 * c, pol_keep);
                acc.x += x.x;
                acc.y += x.y;
                acc.z += x.z;
                acc.w += x.w;
            }
        }
    }
    out[(int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x] = (acc.x + acc.y) + (acc.z + acc.w);
}

template <int LPR>
spx_status launch_probe(int unroll, unsigned grid, cudaStream_t st, int64_t nnz, const int32_t* idx, int32_t n,
                        const float* X, int64_t ldx, float* out) {
    switch (unroll) {
        case 1: gather_probe_kernel<LPR, 1><<<grid, PROBE_THREADS, 0, st>>>(nnz, idx, n, X, ldx, out); break;
        case 2: gather_probe_kernel<LPR, 2><<<grid, PROBE_THREADS, 0, st>>>(nnz, idx, n, X, ldx, out); break;
        default: gather_probe_kernel<LPR, 4><<<grid, PROBE_THREADS, 0, st>>>(nnz, idx, n, X, ldx, out); break;
    }
    SPX_CHECK_LAUNCH("spx_gather_probe");
    return SPX_OK;
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_gather_probe(const int32_t* indices, int64_t nnz, int32_t n, const float* X, int64_t ldx,
                                       int32_t k, int32_t unroll, int32_t blocks_per_sm, float* out, int64_t out_len,
                                       void* stream) {
    if (nnz < 0 || n < 0 || (nnz > 0 && (!indices || !X)) || !out)
        return set_error(SPX_INVALID_ARG, "spx_gather_probe: bad arguments");
    if (k != 4 && k != 8 && k != 16 && k != 32 && k != 64 && k != 128)
        return set_error(SPX_NOT_SUPPORTED, "spx_gather_probe: k = %d (4, 8, 16, 32, 64 or 128)", k);
    if (unroll != 1 && unroll != 2 && unroll != 4)
        return set_error(SPX_INVALID_ARG, "spx_gather_probe: unroll = %d (1, 2 or 4)", unroll);
    if (blocks_per_sm < 1 || blocks_per_sm > 16)
        return set_error(SPX_INVALID_ARG, "spx_gather_probe: blocks_per_sm = %d (1..16)", blocks_per_sm);
    if (ldx < k || (ldx % 4) != 0 || (reinterpret_cast<uintptr_t>(X) & 15) != 0)
        return set_error(SPX_INVALID_ARG, "spx_gather_probe: X must be 16-byte aligned with ldx >= k, ldx %% 4 == 0");
    const int64_t grid = (int64_t)blocks_per_sm * num_sms();
    if (out_len < grid * PROBE_THREADS)
        return set_error(SPX_INVALID_ARG, "spx_gather_probe: out_len %lld < %lld", (long long)out_len,
                         (long long)(grid * PROBE_THREADS));
    cudaStream_t st = as_stream(stream);
    const unsigned gr = (unsigned)grid;
    switch (k / 4) {
        case 1: return launch_probe<1>(unroll, gr, st, nnz, indices, n, X, ldx, out);
        case 2: return launch_probe<2>(unroll, gr, st, nnz, indices, n, X, ldx, out);
        case 4: return launch_probe<4>(unroll, gr, st, nnz, indices, n, X, ldx, out);
        case 8: return launch_probe<8>(unroll, gr, st, nnz, indices, n, X, ldx, out);
        case 16: return launch_probe<16>(unroll, gr, st, nnz, indices, n, X, ldx, out);
        default: return launch_probe<32>(unroll, gr, st, nnz, indices, n, X, ldx, out);
    }
}
