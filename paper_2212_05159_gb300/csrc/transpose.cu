// Sparse transpose of a CSR pattern (Section 3.1.3 forms A^T to compute A^T V).
//
// The entries of A are in row-major order, so A^T's order -- by column, then by row --
// is a *stable* sort of the entries by column index.  We run a least-significant-digit
// radix sort (8-bit digits) of (column, entry id) pairs:
//   upsweep:   per 4096-key tile, a 256-bin digit histogram           -> hist[digit][tile]
//   scan:      exclusive scan of hist in digit-major order             -> global offsets
//   downsweep: stable in-tile ranks (warp match_any per 32-key round, warps in order)
//              and scatter.
// Then t_indices[p] = row(entry[p]) and perm[p] = entry[p].  Integer work only, so
// the result is bit-exact and deterministic.
#include "common.cuh"
#include "scan.cuh"

namespace spx {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                        // 32-key rounds per warp
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;      // 4096 keys per tile
constexpr int RS_BITS = 8;
constexpr int RS_BINS = 1 << RS_BITS;

__global__ void __launch_bounds__(256) expand_rows_kernel(int32_t m, const int32_t* __restrict__ indptr,
                                                          int32_t* __restrict__ rows) {
    // one warp per row, lanes write the row id of each entry
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m) return;
    int a = indptr[warp], b = indptr[warp + 1];
    for (int e = a + lane; e < b; e += 32) rows[e] = (int32_t)warp;
}

__global__ void __launch_bounds__(256) column_count_kernel(int64_t nnz, const int32_t* __restrict__ indices,
                                                           int32_t* __restrict__ count) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride)
        atomicAdd(count + indices[e], 1);
}

__device__ __forceinline__ int64_t key_index(int64_t tile_base, int warp, int round, int lane) {
    return tile_base + (int64_t)warp * (RS_ROUNDS * 32) + round * 32 + lane;
}

__global__ void __launch_bounds__(RS_THREADS) radix_upsweep_kernel(const int32_t* __restrict__ keys, int64_t nnz,
                                                                   int shift, int64_t num_tiles,
                                                                   int32_t* __restrict__ hist) {
    __shared__ int32_t h[RS_BINS];
    for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = key_index(base, warp, r, lane);
        if (i < nnz) atomicAdd(&h[(keys[i] >> shift) & (RS_BINS - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) hist[(int64_t)d * num_tiles + blockIdx.x] = h[d];
}

// vals_in == nullptr means the identity (entry ids) for the first pass.
__global__ void __launch_bounds__(RS_THREADS) radix_downsweep_kernel(
    const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int64_t nnz, int shift,
    int64_t num_tiles, const int32_t* __restrict__ offsets, int32_t* __restrict__ keys_out,
    int32_t* __restrict__ vals_out) {
    __shared__ int32_t wh[RS_WARPS][RS_BINS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wh[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    int32_t key[RS_ROUNDS], val[RS_ROUNDS], rank[RS_ROUNDS];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = key_index(base, warp, r, lane);
        bool valid = i < nnz;
        key[r] = valid ? keys_in[i] : 0;
        val[r] = valid ? (vals_in ? vals_in[i] : (int32_t)i) : 0;
        int d = valid ? ((key[r] >> shift) & (RS_BINS - 1)) : RS_BINS;   // RS_BINS: no bin
        unsigned peers = __match_any_sync(FULL, d);
        int before = __popc(peers & lt);
        int cnt = __popc(peers);
        int cur = valid ? wh[warp][d] : 0;
        rank[r] = cur + before;
        __syncwarp();
        if (valid && before == 0) wh[warp][d] = cur + cnt;
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, plus the tile's global offset
    for (int d = threadIdx.x; d < RS_BINS; d += RS_THREADS) {
        int32_t run = offsets[(int64_t)d * num_tiles + blockIdx.x];
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            int32_t c = wh[w][d];
            wh[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t i = key_index(base, warp, r, lane);
        if (i < nnz) {
            int d = (key[r] >> shift) & (RS_BINS - 1);
            int32_t pos = wh[warp][d] + rank[r];
            keys_out[pos] = key[r];
            vals_out[pos] = val[r];
        }
    }
}

__global__ void __launch_bounds__(256) transpose_finish_kernel(int64_t nnz, const int32_t* __restrict__ sorted_vals,
                                                               const int32_t* __restrict__ rows,
                                                               int32_t* __restrict__ t_indices,
                                                               int32_t* __restrict__ perm) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += stride) {
        int32_t e = sorted_vals ? sorted_vals[p] : (int32_t)p;
        perm[p] = e;
        t_indices[p] = rows[e];
    }
}

struct TransposeLayout {
    size_t rows, keys_a, keys_b, vals_a, vals_b, hist, offsets, count, scan_ws, total;
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

TransposeLayout transpose_layout(int32_t m, int32_t n, int64_t nnz) {
    (void)m;
    TransposeLayout L{};
    int64_t tiles = (nnz + RS_TILE - 1) / RS_TILE;
    int64_t hist_n = (int64_t)RS_BINS * (tiles > 0 ? tiles : 1);
    size_t o = 0;
    L.rows = o;     o = align256(o + sizeof(int32_t) * (size_t)nnz);
    L.keys_a = o;   o = align256(o + sizeof(int32_t) * (size_t)nnz);
    L.keys_b = o;   o = align256(o + sizeof(int32_t) * (size_t)nnz);
    L.vals_a = o;   o = align256(o + sizeof(int32_t) * (size_t)nnz);
    L.vals_b = o;   o = align256(o + sizeof(int32_t) * (size_t)nnz);
    L.hist = o;     o = align256(o + sizeof(int32_t) * (size_t)hist_n);
    L.offsets = o;  o = align256(o + sizeof(int32_t) * (size_t)(hist_n + 1));
    L.count = o;    o = align256(o + sizeof(int32_t) * (size_t)n);
    int64_t scan_n = hist_n > n ? hist_n : (int64_t)n;
    L.scan_ws = o;  o = align256(o + scan_workspace_bytes<int32_t>(scan_n));
    L.total = o;
    return L;
}

int grid_for(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_transpose_workspace_size(int32_t m, int32_t n, int64_t nnz, size_t* bytes) {
    if (!bytes || m < 0 || n < 0 || nnz < 0)
        return set_error(SPX_INVALID_ARG, "spx_transpose_workspace_size: bad arguments");
    *bytes = transpose_layout(m, n, nnz).total;
    return SPX_OK;
}

extern "C" spx_status spx_csr_transpose(const spx_csr* A, int32_t* t_indptr, int32_t* t_indices,
                                        int32_t* perm, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(A, false, "spx_csr_transpose"));
    if (!t_indptr || (A->nnz > 0 && (!t_indices || !perm)))
        return set_error(SPX_INVALID_ARG, "spx_csr_transpose: NULL output");
    TransposeLayout L = transpose_layout(A->m, A->n, A->nnz);
    if (!ws || ws_bytes < L.total)
        return set_error(SPX_OOM_WORKSPACE, "spx_csr_transpose: workspace %zu < %zu", ws_bytes, L.total);
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    int32_t* rows = (int32_t*)(w + L.rows);
    int32_t* count = (int32_t*)(w + L.count);
    int32_t* scan_ws = (int32_t*)(w + L.scan_ws);
    const int64_t nnz = A->nnz;

    // column counts -> t_indptr
    if (A->n > 0) SPX_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)A->n, st), "transpose memset");
    if (nnz > 0) {
        column_count_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, A->indices, count);
        SPX_CHECK_LAUNCH("column_count");
    }
    SPX_TRY((scan_counts<int32_t, int32_t>(count, t_indptr, A->n, scan_ws, st)));
    if (nnz == 0) return SPX_OK;

    int64_t rows_threads = (int64_t)A->m * 32;
    expand_rows_kernel<<<(unsigned)((rows_threads + 255) / 256), 256, 0, st>>>(A->m, A->indptr, rows);
    SPX_CHECK_LAUNCH("expand_rows");

    int bits = 0;
    while (bits < 31 && (int64_t(1) << bits) < (int64_t)A->n) ++bits;
    const int passes = (bits + RS_BITS - 1) / RS_BITS;
    const int64_t tiles = (nnz + RS_TILE - 1) / RS_TILE;
    int32_t* hist = (int32_t*)(w + L.hist);
    int32_t* offs = (int32_t*)(w + L.offsets);
    const int32_t* kin = A->indices;
    const int32_t* vin = nullptr;
    int32_t* kbuf[2] = {(int32_t*)(w + L.keys_a), (int32_t*)(w + L.keys_b)};
    int32_t* vbuf[2] = {(int32_t*)(w + L.vals_a), (int32_t*)(w + L.vals_b)};
    for (int p = 0; p < passes; ++p) {
        int shift = p * RS_BITS;
        radix_upsweep_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(kin, nnz, shift, tiles, hist);
        SPX_CHECK_LAUNCH("radix_upsweep");
        SPX_TRY((scan_counts<int32_t, int32_t>(hist, offs, (int64_t)RS_BINS * tiles, scan_ws, st)));
        radix_downsweep_kernel<<<(unsigned)tiles, RS_THREADS, 0, st>>>(kin, vin, nnz, shift, tiles, offs,
                                                                       kbuf[p & 1], vbuf[p & 1]);
        SPX_CHECK_LAUNCH("radix_downsweep");
        kin = kbuf[p & 1];
        vin = vbuf[p & 1];
    }
    transpose_finish_kernel<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, vin, rows, t_indices, perm);
    SPX_CHECK_LAUNCH("transpose_finish");
    return SPX_OK;
}
