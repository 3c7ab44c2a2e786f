// Sparse x sparse product C = A B, all CSR (Section 3.1.2), and its reverse mode
// (Table 1, SpSpMM rows): gA = (V B^T) masked to A, gB = (A^T V) masked to B, with V
// given on C's pattern.
//
// Forward, expand / sort / compress per row (the ESC scheme the paper follows):
//   analyse   products P_i = sum_{k in A_i} |B_k|, their prefix sums, and the list of
//             "big" rows (P_i > WARP_CAP, appended by an atomic counter: their order in
//             the list varies, no result depends on it);
//   symbolic  per row: expand the P_i product columns, sort, keep the unique ones; the
//             sorted unique columns go to a products-sized scratch at offset Pptr[i] and
//             their count to row_nnz[i]; C_indptr = scan(row_nnz).  Rows of at most 8
//             entries of A and 64 products: one 8-lane group each (four rows per warp),
//             the products in eight registers per lane, sorted by a bitonic network whose
//             short strides stay in a lane and long ones are shuffles, its first levels
//             skipped when B's rows can be laid out as aligned sorted runs.  Other rows of
//             at most 64 products: one warp, two registers per lane, the same network;
//             rows of 65..512 products sort in shared memory; a big row takes a whole block
//             and a shared bitmap of the column space (chunked), which yields the columns
//             already sorted.  mask(C) is structural: no numerical-zero dropping.
//   fill      copies the unique columns into C_indices (8 lanes per row).
//   numeric   per row, C_ij = sum over k in A_i of A_ik B_kj.  Rows of at most 8 entries of
//             A and 64 columns of C: one 8-lane group each (four rows per warp), every B_k's
//             first 8 entries loaded at once, products placed by binary search in C's row and
//             summed over A's entries in order.  Other rows with at most 128
//             columns: four 8-lane groups, group g takes the entries k = g, g+4, ... of A_i
//             (in A's order) into a private slice of the row's accumulator (the four slices
//             fit the space one wide row needs), its lanes over B_k's columns (distinct within
//             a k, so lanes never collide); the slices are added in group order.  Wider rows:
//             the whole warp on one k at a time.  Every sum has a fixed order.
// Reverse.  gA on small rows (at most 8 entries of A and 64 columns of C): one 8-lane group per
// row, four rows per warp, C_i staged in shared memory and lane w owning A's entry w.  Other
// rows of gA, and gB (8-lane groups as well, four stored entries of the output in flight per
// warp):
//   gA[(i,k)] = sum_{j in B_k} V[i,j] B[k,j]: one warp per row i, C_i's columns and V's
//             values staged in shared memory; a group per stored (i,k), its lanes over
//             B_k's entries (binary search of j in C_i), then a fixed shuffle tree.
//   gB[(k,j)] = sum_{i in A^T_k} A[i,k] V[i,j]: the "SpGEMM on the columns of A" of
//             Section 3.1.2 -- one warp per row k of B over the transposed pattern of A; a
//             group per stored (k,j), its lanes over A^T_k (binary search of j in C_i),
//             then a fixed shuffle tree; when A^T_k and B_k have at most 8 entries, a lane's
//             entry of A^T_k and C_i's bounds are loaded once and both rounds of B_k search
//             together.
// All integer work is exact; every floating-point sum has a fixed order.
#include <limits.h>

#include "common.cuh"
#include "scan.cuh"

namespace spx {
namespace {

constexpr int WARP_CAP = 512;          // products per row handled by one warp
constexpr int SYM_WARPS = 8;           // warps per block, symbolic / fill
constexpr int NUM_WARPS = 4;           // warps per block, numeric
constexpr int GRP = 8;                 // lanes per group in the value kernels
constexpr int NGRP = 32 / GRP;         // groups per warp
constexpr int BIG_THREADS = 512;
constexpr int FILL_LANES = 8;         // lanes per row, fill
constexpr int BITMAP_WORDS = 8192;     // 32 KB shared bitmap: 262144 columns per chunk

inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

struct GemmLayout {
    size_t prod, pptr, row_nnz, big_pos, big_rows, scan64, scan32, total;
};

GemmLayout gemm_layout(int32_t m) {
    GemmLayout L{};
    size_t o = 0;
    L.prod = o;     o = al(o + 4 * (size_t)m);
    L.pptr = o;     o = al(o + 8 * ((size_t)m + 1));
    L.row_nnz = o;  o = al(o + 4 * (size_t)m);
    L.big_pos = o;  o = al(o + 4 * ((size_t)m + 1));
    L.big_rows = o; o = al(o + 4 * ((size_t)m + 1));
    L.scan64 = o;   o = al(o + scan_workspace_bytes<int64_t>(m));
    L.scan32 = o;   o = al(o + scan_workspace_bytes<int32_t>(m));
    L.total = o;
    return L;
}

// ------------------------------------------------------------------ analyse
// Products per row, and the rows with more than WARP_CAP of them appended to big_rows (their
// order in the list varies from run to run; each is computed whole by one block, so no result
// depends on it).  *n_big must be zero before the launch.
__global__ void products_kernel(int32_t m, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx,
                                const int32_t* __restrict__ b_ptr, int32_t* __restrict__ prod,
                                int32_t* __restrict__ big_rows, int32_t* __restrict__ n_big) {
    // 8 lanes per row
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = t >> 3;
    const int sub = threadIdx.x & 7;
    int64_t s = 0;
    if (row < m) {
        for (int e = a_ptr[row] + sub; e < a_ptr[row + 1]; e += 8) {
            const int k = a_idx[e];
            s += b_ptr[k + 1] - b_ptr[k];
        }
    }
#pragma unroll
    for (int o = 4; o >= 1; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (row < m && sub == 0) {
        const int32_t p = s > INT_MAX ? INT_MAX : (int32_t)s;
        prod[row] = p;
        if (p > WARP_CAP) big_rows[atomicAdd(n_big, 1)] = (int32_t)row;
    }
}

// ------------------------------------------------------------------ symbolic (warp rows)
__device__ __forceinline__ void warp_bitonic_sort(int* keys, int Q, int lane) {
    for (int size = 2; size <= Q; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (Q >> 1); t += 32) {
                const int i = 2 * stride * (t / stride) + (t % stride);
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const int a = keys[i], b = keys[j];
                if ((a > b) == up) {
                    keys[i] = b;
                    keys[j] = a;
                }
            }
            __syncwarp();
        }
    }
}

// Bitonic sort of a warp's 32 * NS keys held in registers, key e = lane + 32 s in v[s]:
// compare-exchanges with a partner in another lane go through shuffles, those between the
// two slots of a lane (stride 32) stay local.  Ascending.  Levels below `start` are
// skipped: the caller guarantees that every aligned block of start / 2 keys is already
// sorted, ascending where its block index is even and descending where it is odd (the
// state the network itself leaves after those levels).
template <int NS>
__device__ __forceinline__ void warp_bitonic_sort_regs(int (&v)[NS], int lane, int start) {
    constexpr int Q = 32 * NS;
#pragma unroll
    for (int size = 2; size <= Q; size <<= 1) {
        if (size < start) continue;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {                              // NS == 2: slots 0 and 1 of the lane
                const int e = lane;                          // the lower element of the pair
                const bool up = (e & size) == 0;
                const int a = v[0], b = v[1];
                v[0] = up ? min(a, b) : max(a, b);
                v[1] = up ? max(a, b) : min(a, b);
            } else {
#pragma unroll
                for (int s2 = 0; s2 < NS; ++s2) {
                    const int e = lane + 32 * s2;
                    const int p = __shfl_xor_sync(FULL, v[s2], stride);
                    const bool lower = (e & stride) == 0;
                    const bool up = (e & size) == 0;
                    v[s2] = (lower == up) ? min(v[s2], p) : max(v[s2], p);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ symbolic (small rows)
// Rows with at most SYG_A entries of A and at most SYG_P products: one 8-lane group per row,
// so a warp keeps four rows in flight.  A row's 64 slots are laid out lane-major (slot
// i = 8 c + s is register s of lane c): the bitonic network's strides 1..4 compare registers
// of one lane, strides 8..32 exchange register s with lane c ^ (stride / 8) by a shuffle.  When
// the aligned-run layout fits (|A_i| R <= 64, R the smallest power of two >= every |B_k|),
// entry e's columns fill slots [e R, e R + R), ascending for even e and reversed (pads first)
// for odd e, and the levels up to R are skipped; with R = 8 a lane's run is its own registers.
// Otherwise the products are packed in entry order and sorted in full.  The first of each
// run is kept, in order.  symbolic_warp_kernel skips these rows.
constexpr int SYG_THREADS = 256;
constexpr int SYG_A = GRP;             // entries of A per small row: one per lane of the group
constexpr int SYG_P = 8 * GRP;         // products per small row: eight registers per lane

__device__ __forceinline__ bool small_symbolic_row(int na, int p) { return na <= SYG_A && p <= SYG_P; }

__global__ void __launch_bounds__(SYG_THREADS) symbolic_group_kernel(
    int32_t m, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const int32_t* __restrict__ prod, const int64_t* __restrict__ pptr,
    int32_t* __restrict__ tmp, int32_t* __restrict__ row_nnz) {
    const int lane = threadIdx.x & 31;
    const int c = lane % GRP;
    const unsigned gmask = ((1u << GRP) - 1u) << ((lane / GRP) * GRP);
    const int64_t row = ((int64_t)blockIdx.x * SYG_THREADS + threadIdx.x) / GRP;
    if (row >= m) return;                                  // the whole group leaves
    const int P = prod[row];
    const int a0 = a_ptr[row], nA = a_ptr[row + 1] - a0;
    if (!small_symbolic_row(nA, P)) return;                // group-uniform
    int32_t* out = tmp + pptr[row];                        // loaded now, off the row's chain
    int b0 = 0, len = 0;
    if (c < nA) {
        const int k = a_idx[a0 + c];
        b0 = b_ptr[k];
        len = b_ptr[k + 1] - b0;
    }
    int lmax = len;
#pragma unroll
    for (int o = 1; o < GRP; o <<= 1) lmax = max(lmax, __shfl_xor_sync(gmask, lmax, o, GRP));
    int R = 1;
    while (R < lmax) R <<= 1;
    int v[8];
    int start;
    if (R == 8) {                                          // entry c's run is lane c's registers
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            int key = INT_MAX;
            if ((c & 1) == 0) {
                if (s < len) key = b_idx[b0 + s];
            } else {
                const int q = s - (8 - len);                   // descending: pads first
                if (q >= 0) key = b_idx[b0 + len - 1 - q];
            }
            v[s] = key;                                        // lanes c >= nA have len 0: pads
        }
        start = 16;
    } else if (nA * R <= SYG_P) {
        const int lg = __ffs(R) - 1;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int i = 8 * c + s;
            const int e = i >> lg, pos = i & (R - 1);
            const int bb = __shfl_sync(gmask, b0, e & (GRP - 1), GRP);
            const int ll = __shfl_sync(gmask, len, e & (GRP - 1), GRP);
            int key = INT_MAX;
            if (e < nA) {
                if ((e & 1) == 0) {
                    if (pos < ll) key = b_idx[bb + pos];
                } else {
                    const int q = pos - (R - ll);              // descending: pads first
                    if (q >= 0) key = b_idx[bb + ll - 1 - q];
                }
            }
            v[s] = key;
        }
        start = 2 * R;
    } else {
        // packed: product t lies in the entry whose inclusive scan of the lengths first exceeds t
        int incl = len;
#pragma unroll
        for (int o = 1; o < GRP; o <<= 1) {
            const int y = __shfl_up_sync(gmask, incl, o, GRP);
            if (c >= o) incl += y;
        }
        const int excl = incl - len;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int t = 8 * c + s;
            int e = 0;                                       // lanes with incl <= t
#pragma unroll
            for (int step = GRP / 2; step >= 1; step >>= 1) {
                const int cc = __shfl_sync(gmask, incl, e + step - 1, GRP);
                if (cc <= t) e += step;
            }
            e = min(e, GRP - 1);
            const int src = __shfl_sync(gmask, b0, e, GRP) + t - __shfl_sync(gmask, excl, e, GRP);
            v[s] = t < P ? b_idx[src] : INT_MAX;
        }
        start = 2;
    }
#pragma unroll
    for (int size = 2; size <= SYG_P; size <<= 1) {
        if (size < start) continue;
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 8) {                               // partner: register s of lane c ^ (stride / 8)
                const int lm = stride >> 3;
                const bool lower = (c & lm) == 0;
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const bool up = ((8 * c + s) & size) == 0;
                    const int p = __shfl_xor_sync(gmask, v[s], lm, GRP);
                    v[s] = (lower == up) ? min(v[s], p) : max(v[s], p);
                }
            } else {                                         // both keys in this lane
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    if (s & stride) continue;
                    const bool up = ((8 * c + s) & size) == 0;
                    const int a = v[s], b = v[s | stride];
                    v[s] = up ? min(a, b) : max(a, b);
                    v[s | stride] = up ? max(a, b) : min(a, b);
                }
            }
        }
    }
    // the first of each run among the P real keys (pads, INT_MAX, sort last)
    const int prev7 = __shfl_up_sync(gmask, v[7], 1, GRP);
    unsigned keep = 0;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int i = 8 * c + s;
        const int prev = s ? v[s - 1] : prev7;
        if (i < P && (i == 0 || v[s] != prev)) keep |= 1u << s;
    }
    const int cnt = __popc(keep);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < GRP; o <<= 1) {
        const int y = __shfl_up_sync(gmask, incl, o, GRP);
        if (c >= o) incl += y;
    }
    out += incl - cnt;
#pragma unroll
    for (int s = 0; s < 8; ++s)
        if (keep & (1u << s)) *out++ = v[s];
    if (c == GRP - 1) row_nnz[row] = incl;
}

// ------------------------------------------------------------------ symbolic (other warp rows)
// Sorted unique product columns of row i -> tmp + pptr[i]; count -> row_nnz[i].
__device__ __forceinline__ void symbolic_warp_row(
    int64_t row, int lane, int* keys, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx,
    const int32_t* __restrict__ b_ptr, const int32_t* __restrict__ b_idx, const int32_t* __restrict__ prod,
    const int64_t* __restrict__ pptr, int32_t* __restrict__ tmp, int32_t* __restrict__ row_nnz) {
    __syncwarp();                                   // the previous row's reads of keys are done
    const int P = prod[row];
    const int a0 = a_ptr[row], nA = a_ptr[row + 1] - a0;
    int32_t* out = tmp + pptr[row];
    if (P <= 64 && nA <= 32) {
        // at most 64 products from at most 32 entries of A, every product column fetched
        // straight into a register (two per lane, INT_MAX pads).  Lane e holds B_k's range
        // for entry e.  When R (the smallest power of two >= every |B_k|) times |A_i| fits
        // the 64 slots, entry e's sorted columns go to the aligned slots [e R, e R + R),
        // ascending for even e and reversed for odd e, which is the state of the bitonic
        // network after its levels up to R, so those levels are skipped.  Otherwise the
        // products are packed: product t lies in the entry whose inclusive scan of the
        // lengths first exceeds t (a binary search over the lanes).
        int b0 = 0, len = 0;
        if (lane < nA) {
            const int k = a_idx[a0 + lane];
            b0 = b_ptr[k];
            len = b_ptr[k + 1] - b0;
        }
        const int lmax = __reduce_max_sync(FULL, (unsigned)len);
        int R = 1;
        while (R < lmax) R <<= 1;
        int v[2];
        int start, used;
        if (nA * R <= 64) {
            const int lg = __ffs(R) - 1;
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int sl = lane + 32 * s2;
                const int e = sl >> lg, pos = sl & (R - 1);
                const int bb = __shfl_sync(FULL, b0, e & 31);
                const int ll = __shfl_sync(FULL, len, e & 31);
                int key = INT_MAX;
                if (e < nA) {
                    if ((e & 1) == 0) {
                        if (pos < ll) key = b_idx[bb + pos];
                    } else {
                        const int q = pos - (R - ll);          // descending: pads first
                        if (q >= 0) key = b_idx[bb + ll - 1 - q];
                    }
                }
                v[s2] = key;
            }
            start = 2 * R;
            used = nA * R;
        } else {
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const int excl = incl - len;
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
                const int t = lane + 32 * s2;
                int e = 0;                                   // lanes with incl <= t
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int c = __shfl_sync(FULL, incl, e + step - 1);
                    if (c <= t) e += step;
                }
                e = min(e, 31);
                const int src = __shfl_sync(FULL, b0, e) + t - __shfl_sync(FULL, excl, e);
                v[s2] = t < P ? b_idx[src] : INT_MAX;
            }
            start = 2;
            used = P;
        }
        // sorted in registers, then the first of each run kept in order with ballots
        if (used <= 32) {                                // slots 32..63 hold pads only
            int w1[1] = {v[0]};
            warp_bitonic_sort_regs<1>(w1, lane, start);
            v[0] = w1[0];
        } else {
            warp_bitonic_sort_regs<2>(v, lane, start);
        }
        int base = 0;
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            const int t = lane + 32 * s2;
            int prev = __shfl_up_sync(FULL, v[s2], 1);
            const int last_lo = __shfl_sync(FULL, v[0], 31);    // key 31, before key 32
            if (lane == 0) prev = s2 == 0 ? INT_MIN : last_lo;
            const bool keep = t < P && (t == 0 || v[s2] != prev);
            const unsigned bal = __ballot_sync(FULL, keep);
            if (keep) out[base + __popc(bal & lanemask_lt())] = v[s2];
            base += __popc(bal);
        }
        if (lane == 0) row_nnz[row] = base;
        return;
    }
    // expand
    int pos = 0;
    for (int e = a0; e < a0 + nA; ++e) {
        const int k = a_idx[e];
        const int b0 = b_ptr[k], len = b_ptr[k + 1] - b0;
        for (int t = lane; t < len; t += 32) keys[pos + t] = b_idx[b0 + t];
        pos += len;
    }
    __syncwarp();
    int Q = 1;
    while (Q < P) Q <<= 1;
    for (int t = P + lane; t < Q; t += 32) keys[t] = INT_MAX;
    __syncwarp();
    warp_bitonic_sort(keys, Q, lane);
    // compress: keep the first of each run, in order
    int base = 0;
    for (int t0 = 0; t0 < P; t0 += 32) {
        const int t = t0 + lane;
        const bool keep = t < P && (t == 0 || keys[t] != keys[t - 1]);
        const unsigned bal = __ballot_sync(FULL, keep);
        if (keep) out[base + __popc(bal & lanemask_lt())] = keys[t];
        base += __popc(bal);
    }
    if (lane == 0) row_nnz[row] = base;
}

// The rows neither symbolic_group_kernel (small rows) nor symbolic_big_kernel (more than
// WARP_CAP products) takes: each warp checks 32 rows at once (lane r: row base + r), then runs
// the ones that are its, one at a time.  Grid-strided over the rows.
__global__ void __launch_bounds__(SYM_WARPS * 32) symbolic_warp_kernel(
    int32_t m, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const int32_t* __restrict__ prod, const int64_t* __restrict__ pptr,
    int32_t* __restrict__ tmp, int32_t* __restrict__ row_nnz) {
    __shared__ int keys_all[SYM_WARPS][WARP_CAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * SYM_WARPS;
    for (int64_t base = ((int64_t)blockIdx.x * SYM_WARPS + warp) * 32; base < m; base += nw * 32) {
        const int64_t r = base + lane;
        bool mine = false;
        if (r < m) {
            const int p = prod[r];
            mine = p <= WARP_CAP && !small_symbolic_row(a_ptr[r + 1] - a_ptr[r], p);
        }
        unsigned todo = __ballot_sync(FULL, mine);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            symbolic_warp_row(base + b, lane, keys_all[warp], a_ptr, a_idx, b_ptr, b_idx, prod, pptr, tmp, row_nnz);
        }
    }
}

// ------------------------------------------------------------------ symbolic (big rows)
// One block per big row; the column space is visited in chunks of BITMAP_WORDS*32.
__global__ void __launch_bounds__(BIG_THREADS) symbolic_big_kernel(
    const int32_t* __restrict__ big_rows, const int32_t* __restrict__ n_big_dev, int32_t p,
    const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const int64_t* __restrict__ pptr, int32_t* __restrict__ tmp,
    int32_t* __restrict__ row_nnz) {
    __shared__ unsigned bits[BITMAP_WORDS];
    __shared__ int warp_sums[BIG_THREADS / 32 + 1];
    const int n_big = *n_big_dev;
    constexpr int WPT = BITMAP_WORDS / BIG_THREADS;           // words per thread
    for (int q = blockIdx.x; q < n_big; q += gridDim.x) {
        const int row = big_rows[q];
        const int ea = a_ptr[row], eb = a_ptr[row + 1];
        int32_t* out = tmp + pptr[row];
        int written = 0;
        for (int64_t c0 = 0; c0 < p; c0 += (int64_t)BITMAP_WORDS * 32) {
            for (int w = threadIdx.x; w < BITMAP_WORDS; w += BIG_THREADS) bits[w] = 0u;
            __syncthreads();
            for (int e = ea + threadIdx.x; e < eb; e += BIG_THREADS) {
                const int k = a_idx[e];
                for (int f = b_ptr[k]; f < b_ptr[k + 1]; ++f) {
                    const int64_t j = (int64_t)b_idx[f] - c0;
                    if (j >= 0 && j < (int64_t)BITMAP_WORDS * 32) atomicOr(&bits[j >> 5], 1u << (j & 31));
                }
            }
            __syncthreads();
            // thread t owns words [t*WPT, (t+1)*WPT): exclusive scan of their popcounts
            int cnt = 0;
#pragma unroll
            for (int u = 0; u < WPT; ++u) cnt += __popc(bits[threadIdx.x * WPT + u]);
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(FULL, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) warp_sums[warp] = inc;
            __syncthreads();
            if (threadIdx.x == 0) {
                int run = 0;
                for (int w = 0; w < BIG_THREADS / 32; ++w) {
                    int v = warp_sums[w];
                    warp_sums[w] = run;
                    run += v;
                }
                warp_sums[BIG_THREADS / 32] = run;
            }
            __syncthreads();
            int wpos = written + warp_sums[warp] + inc - cnt;
#pragma unroll
            for (int u = 0; u < WPT; ++u) {
                unsigned word = bits[threadIdx.x * WPT + u];
                while (word) {
                    const int bpos = __ffs(word) - 1;
                    word &= word - 1;
                    out[wpos++] = (int32_t)(c0 + (int64_t)(threadIdx.x * WPT + u) * 32 + bpos);
                }
            }
            written += warp_sums[BIG_THREADS / 32];
            __syncthreads();
        }
        if (threadIdx.x == 0) row_nnz[row] = written;
    }
}

__global__ void fill_kernel(int32_t m, const int64_t* __restrict__ pptr, const int32_t* __restrict__ tmp,
                            const int32_t* __restrict__ c_ptr, int32_t* __restrict__ c_idx) {
    // FILL_LANES lanes per row, four loads in flight per lane
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / FILL_LANES;
    const int sub = threadIdx.x % FILL_LANES;
    if (row >= m) return;
    const int32_t* src = tmp + pptr[row];
    const int a = c_ptr[row], n = c_ptr[row + 1] - a;
    int32_t* dst = c_idx + a;
    int t = sub;
    for (; t + 3 * FILL_LANES < n; t += 4 * FILL_LANES) {
        const int v0 = src[t], v1 = src[t + FILL_LANES], v2 = src[t + 2 * FILL_LANES], v3 = src[t + 3 * FILL_LANES];
        dst[t] = v0;
        dst[t + FILL_LANES] = v1;
        dst[t + 2 * FILL_LANES] = v2;
        dst[t + 3 * FILL_LANES] = v3;
    }
    for (; t < n; t += FILL_LANES) dst[t] = src[t];
}

// ------------------------------------------------------------------ numeric
__device__ __forceinline__ int lower_bound_i32(const int* __restrict__ a, int n, int key) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Small rows: at most SG_A entries of A, at most SG_C columns of C and at most WARP_CAP
// products.  One 8-lane group per row, so a warp keeps four rows in flight.  Lane e loads A's
// entry e and B_k's bounds, then lane w the first 8 entries of every B_k (entry w of each),
// so a row costs four dependent round trips (its bounds; A's entries and C's columns; B's
// bounds; B's entries).  Every product's place in C's row comes from a binary search over
// C's columns in shared memory, all searches before any sum; the sums then run over A's
// entries in order, one fixed-order FMA per product into the group's accumulator (the
// columns of one B_k are distinct, so the lanes never collide).  numeric_warp_kernel
// skips these rows.
constexpr int SG_THREADS = 256;
constexpr int SG_A = 8;                // A entries per small row
constexpr int SG_C = 64;               // C columns per small row

__device__ __forceinline__ bool small_row(int na, int nc, int p) {
    return na <= SG_A && nc <= SG_C && p <= WARP_CAP;
}

__global__ void __launch_bounds__(SG_THREADS, 5) numeric_group_kernel(
    int32_t m, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const float* __restrict__ a_val,
    const int32_t* __restrict__ b_ptr, const int32_t* __restrict__ b_idx, const float* __restrict__ b_val,
    const int32_t* __restrict__ c_ptr, const int32_t* __restrict__ c_idx, const int32_t* __restrict__ prod,
    float* __restrict__ c_val) {
    // each group's rows padded by 8 words: the four groups of a warp start 8 banks apart, so
    // their searches and sums at equal offsets do not meet in one bank
    __shared__ int scol[SG_THREADS / GRP][SG_C + 8];
    __shared__ float sacc[SG_THREADS / GRP][SG_C + 8];
    const int lane = threadIdx.x & 31;
    const int gid = threadIdx.x / GRP;
    const int w = lane % GRP;
    const unsigned gmask = ((1u << GRP) - 1u) << ((lane / GRP) * GRP);
    const int64_t row = (int64_t)blockIdx.x * (SG_THREADS / GRP) + gid;
    if (row >= m) return;                                  // the whole group leaves
    const int a0 = a_ptr[row], na = a_ptr[row + 1] - a0;
    const int c0 = c_ptr[row], nc = c_ptr[row + 1] - c0;
    if (!small_row(na, nc, prod[row])) return;
    int* cols = scol[gid];
    float* acc = sacc[gid];
    int k = -1;
    float av = 0.f;
    if (w < na) {
        k = a_idx[a0 + w];
        av = a_val[a0 + w];
    }
    {                                                      // C's columns: all loads in flight at once
        int cv[SG_C / GRP];
#pragma unroll
        for (int q = 0; q < SG_C / GRP; ++q) cv[q] = w + q * GRP < nc ? c_idx[c0 + w + q * GRP] : 0;
#pragma unroll
        for (int q = 0; q < SG_C / GRP; ++q)
            if (w + q * GRP < nc) {
                cols[w + q * GRP] = cv[q];
                acc[w + q * GRP] = 0.f;
            }
    }
    int bs = 0, be = 0;
    if (k >= 0) {
        bs = b_ptr[k];
        be = b_ptr[k + 1];
    }
    int jt[SG_A];
    float vt[SG_A];
#pragma unroll
    for (int t = 0; t < SG_A; ++t) {
        const int s_t = __shfl_sync(gmask, bs, t, GRP), e_t = __shfl_sync(gmask, be, t, GRP);
        jt[t] = -1;
        vt[t] = 0.f;
        if (t < na && s_t + w < e_t) {
            jt[t] = b_idx[s_t + w];
            vt[t] = b_val[s_t + w];
        }
    }
    __syncwarp(gmask);                                     // C's columns visible to the group
    int pos[SG_A];
#pragma unroll
    for (int t = 0; t < SG_A; ++t) pos[t] = jt[t] >= 0 ? lower_bound_i32(cols, nc, jt[t]) : 0;
#pragma unroll
    for (int t = 0; t < SG_A; ++t) {
        if (t < na) {                                      // group-uniform
            const float a_t = __shfl_sync(gmask, av, t, GRP);
            const int s_t = __shfl_sync(gmask, bs, t, GRP), e_t = __shfl_sync(gmask, be, t, GRP);
            if (jt[t] >= 0) acc[pos[t]] = fmaf(a_t, vt[t], acc[pos[t]]);
            __syncwarp(gmask);
            for (int f0 = s_t + GRP; f0 < e_t; f0 += GRP) {    // the rest of a longer B_k
                const int f = f0 + w;
                if (f < e_t) {
                    const int p2 = lower_bound_i32(cols, nc, b_idx[f]);
                    acc[p2] = fmaf(a_t, b_val[f], acc[p2]);
                }
                __syncwarp(gmask);
            }
        }
    }
    __syncwarp(gmask);
#pragma unroll
    for (int q = 0; q < SG_C / GRP; ++q)
        if (w + q * GRP < nc) c_val[c0 + w + q * GRP] = acc[w + q * GRP];
}

// One row, one warp (rows of C wider than numeric_group_kernel takes, up to WARP_CAP products).
__device__ __forceinline__ void numeric_warp_row(
    int64_t row, int lane, int* __restrict__ cols, float* __restrict__ acc, const int32_t* __restrict__ a_ptr,
    const int32_t* __restrict__ a_idx, const float* __restrict__ a_val, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const float* __restrict__ b_val, const int32_t* __restrict__ c_ptr,
    const int32_t* __restrict__ c_idx, float* __restrict__ c_val) {
    const int c0 = c_ptr[row], nc = c_ptr[row + 1] - c0;
    const int a0 = a_ptr[row], a1 = a_ptr[row + 1];
    if (nc * NGRP <= WARP_CAP) {
        // four 8-lane groups, each with a private accumulator slice of the row: group g takes
        // the entries k = g, g+4, ... of A_i in order; the slices are added in group order
        for (int t = lane; t < nc; t += 32) cols[t] = c_idx[c0 + t];
        for (int t = lane; t < nc * NGRP; t += 32) acc[t] = 0.f;
        __syncwarp();
        const int g = lane / GRP, w = lane % GRP;
        const unsigned gmask = ((1u << GRP) - 1u) << (g * GRP);
        float* mine = acc + g * nc;
        for (int e = a0 + g; e < a1; e += NGRP) {
            const int k = a_idx[e];
            const float av = a_val[e];
            for (int f = b_ptr[k] + w; f < b_ptr[k + 1]; f += GRP) {
                const int pos = lower_bound_i32(cols, nc, b_idx[f]);
                mine[pos] = fmaf(av, b_val[f], mine[pos]);
            }
            __syncwarp(gmask);                      // the group's next k may hit the same columns
        }
        __syncwarp();
        for (int t = lane; t < nc; t += 32) {
            float sum = acc[t];
#pragma unroll
            for (int q = 1; q < NGRP; ++q) sum += acc[q * nc + t];
            c_val[c0 + t] = sum;
        }
        __syncwarp();                               // cols / acc free for the warp's next row
        return;
    }
    // wider rows: the whole warp on one k at a time, one accumulator
    for (int t = lane; t < nc; t += 32) {
        cols[t] = c_idx[c0 + t];
        acc[t] = 0.f;
    }
    __syncwarp();
    for (int e = a0; e < a1; ++e) {
        const int k = a_idx[e];
        const float av = a_val[e];
        for (int f = b_ptr[k] + lane; f < b_ptr[k + 1]; f += 32) {
            const int pos = lower_bound_i32(cols, nc, b_idx[f]);
            acc[pos] = fmaf(av, b_val[f], acc[pos]);
        }
        __syncwarp();
    }
    for (int t = lane; t < nc; t += 32) c_val[c0 + t] = acc[t];
    __syncwarp();
}

// The rows neither numeric_group_kernel (small rows) nor numeric_big_kernel (more than
// WARP_CAP products) takes: each warp checks 32 rows at once (lane r row base + r), then
// runs the ones that are its, one at a time.  Grid-strided over the rows.
__global__ void __launch_bounds__(NUM_WARPS * 32) numeric_warp_kernel(
    int32_t m, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const float* __restrict__ a_val,
    const int32_t* __restrict__ b_ptr, const int32_t* __restrict__ b_idx, const float* __restrict__ b_val,
    const int32_t* __restrict__ c_ptr, const int32_t* __restrict__ c_idx, const int32_t* __restrict__ prod,
    float* __restrict__ c_val) {
    __shared__ int cols_all[NUM_WARPS][WARP_CAP];
    __shared__ float acc_all[NUM_WARPS][WARP_CAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * NUM_WARPS;
    for (int64_t base = ((int64_t)blockIdx.x * NUM_WARPS + warp) * 32; base < m; base += nw * 32) {
        const int64_t r = base + lane;
        bool mine = false;
        if (r < m) {
            const int p = prod[r];
            mine = p <= WARP_CAP && !small_row(a_ptr[r + 1] - a_ptr[r], c_ptr[r + 1] - c_ptr[r], p);
        }
        unsigned todo = __ballot_sync(FULL, mine);
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            numeric_warp_row(base + b, lane, cols_all[warp], acc_all[warp], a_ptr, a_idx, a_val, b_ptr, b_idx, b_val,
                             c_ptr, c_idx, c_val);
        }
    }
}

__global__ void __launch_bounds__(BIG_THREADS) numeric_big_kernel(
    const int32_t* __restrict__ big_rows, const int32_t* __restrict__ n_big_dev, const int32_t* __restrict__ a_ptr,
    const int32_t* __restrict__ a_idx, const float* __restrict__ a_val, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const float* __restrict__ b_val, const int32_t* __restrict__ c_ptr,
    const int32_t* __restrict__ c_idx, float* __restrict__ c_val) {
    const int n_big = *n_big_dev;
    for (int q = blockIdx.x; q < n_big; q += gridDim.x) {
        const int row = big_rows[q];
        const int c0 = c_ptr[row], nc = c_ptr[row + 1] - c0;
        for (int t = threadIdx.x; t < nc; t += BIG_THREADS) c_val[c0 + t] = 0.f;
        __syncthreads();
        for (int e = a_ptr[row]; e < a_ptr[row + 1]; ++e) {
            const int k = a_idx[e];
            const float av = a_val[e];
            for (int f = b_ptr[k] + threadIdx.x; f < b_ptr[k + 1]; f += BIG_THREADS) {
                const int pos = c0 + lower_bound_i32(c_idx + c0, nc, b_idx[f]);
                c_val[pos] = fmaf(av, b_val[f], c_val[pos]);
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------ backward
// sum over the GRP lanes of a group, a fixed xor tree (the same order on every run)
__device__ __forceinline__ float group_sum(float v, unsigned gmask) {
#pragma unroll
    for (int o = GRP / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(gmask, v, o, GRP);
    return v;
}

// gA on small rows (at most SG_A entries of A and SG_C columns of C): one 8-lane group per row
// i, C_i's columns and V's values staged in shared memory (padded per group as in
// numeric_group_kernel); lane w owns A's entry w, loads the first 8 entries of its B_k at
// once, places each column in C_i by a binary search in shared memory (all searches before
// the sum) and adds V[i, j] B[k, j] in B_k's order.  grad_a_kernel skips these rows.
__global__ void __launch_bounds__(SG_THREADS, 5) grad_a_group_kernel(
    int32_t m, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const float* __restrict__ b_val, const int32_t* __restrict__ c_ptr,
    const int32_t* __restrict__ c_idx, const float* __restrict__ gc, float* __restrict__ ga) {
    __shared__ int scol[SG_THREADS / GRP][SG_C + 8];
    __shared__ float sv[SG_THREADS / GRP][SG_C + 8];
    const int lane = threadIdx.x & 31;
    const int gid = threadIdx.x / GRP;
    const int w = lane % GRP;
    const unsigned gmask = ((1u << GRP) - 1u) << ((lane / GRP) * GRP);
    const int64_t row = (int64_t)blockIdx.x * (SG_THREADS / GRP) + gid;
    if (row >= m) return;                                  // the whole group leaves
    const int a0 = a_ptr[row], na = a_ptr[row + 1] - a0;
    const int c0 = c_ptr[row], nc = c_ptr[row + 1] - c0;
    if (na > SG_A || nc > SG_C) return;
    int* cols = scol[gid];
    float* v = sv[gid];
    {
        int cv[SG_C / GRP];
        float vv[SG_C / GRP];
#pragma unroll
        for (int q = 0; q < SG_C / GRP; ++q) {
            const bool in = w + q * GRP < nc;
            cv[q] = in ? c_idx[c0 + w + q * GRP] : 0;
            vv[q] = in ? gc[c0 + w + q * GRP] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < SG_C / GRP; ++q)
            if (w + q * GRP < nc) {
                cols[w + q * GRP] = cv[q];
                v[w + q * GRP] = vv[q];
            }
    }
    int bs = 0, be = 0;
    if (w < na) {
        const int k = a_idx[a0 + w];
        bs = b_ptr[k];
        be = b_ptr[k + 1];
    }
    int jt[GRP];
    float bt[GRP];
#pragma unroll
    for (int q = 0; q < GRP; ++q) {
        jt[q] = bs + q < be ? b_idx[bs + q] : -1;
        bt[q] = bs + q < be ? b_val[bs + q] : 0.f;
    }
    __syncwarp(gmask);                                     // the staged row visible to the group
    int pos[GRP];
#pragma unroll
    for (int q = 0; q < GRP; ++q) pos[q] = jt[q] >= 0 ? lower_bound_i32(cols, nc, jt[q]) : nc;
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < GRP; ++q)
        if (pos[q] < nc && cols[pos[q]] == jt[q]) sum = fmaf(v[pos[q]], bt[q], sum);
    for (int f = bs + GRP; f < be; ++f) {                  // the rest of a longer B_k
        const int j = b_idx[f];
        const int p = lower_bound_i32(cols, nc, j);
        if (p < nc && cols[p] == j) sum = fmaf(v[p], b_val[f], sum);
    }
    if (w < na) ga[a0 + w] = sum;
}

// gA[(i,k)] = sum_{f in B_k} V[i, B_idx[f]] * B_val[f]   (V on C's pattern), the rows
// grad_a_group_kernel does not take: each warp checks 32 rows at once and runs its own, one at
// a time (grid-strided).
__global__ void __launch_bounds__(NUM_WARPS * 32) grad_a_kernel(
    int32_t m, const int32_t* __restrict__ a_ptr, const int32_t* __restrict__ a_idx, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const float* __restrict__ b_val, const int32_t* __restrict__ c_ptr,
    const int32_t* __restrict__ c_idx, const float* __restrict__ gc, float* __restrict__ ga) {
    __shared__ int cols_all[NUM_WARPS][WARP_CAP];
    __shared__ float v_all[NUM_WARPS][WARP_CAP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane / GRP, w = lane % GRP;
    const unsigned gmask = ((1u << GRP) - 1u) << (g * GRP);
    const int64_t nw = (int64_t)gridDim.x * NUM_WARPS;
    for (int64_t base = ((int64_t)blockIdx.x * NUM_WARPS + warp) * 32; base < m; base += nw * 32) {
        const int64_t r = base + lane;
        const bool mine = r < m && (a_ptr[r + 1] - a_ptr[r] > SG_A || c_ptr[r + 1] - c_ptr[r] > SG_C);
        unsigned todo = __ballot_sync(FULL, mine);
        while (todo) {
            const int bb = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t row = base + bb;
            const int c0 = c_ptr[row], nc = c_ptr[row + 1] - c0;
            const bool staged = nc <= WARP_CAP;
            const int* cols = staged ? cols_all[warp] : c_idx + c0;
            const float* v = staged ? v_all[warp] : gc + c0;
            if (staged) {
                for (int t = lane; t < nc; t += 32) {
                    cols_all[warp][t] = c_idx[c0 + t];
                    v_all[warp][t] = gc[c0 + t];
                }
            }
            __syncwarp();
            const int a0 = a_ptr[row], a1 = a_ptr[row + 1];
            // the groups take the row's entries round-robin; every lane of a group runs the same trips
            for (int e0 = a0; e0 < a1; e0 += NGRP) {
                const int e = e0 + g;
                float s = 0.f;
                if (e < a1) {
                    const int k = a_idx[e];
                    for (int f = b_ptr[k] + w; f < b_ptr[k + 1]; f += GRP) {
                        const int j = b_idx[f];
                        const int pos = lower_bound_i32(cols, nc, j);
                        if (pos < nc && cols[pos] == j) s = fmaf(v[pos], b_val[f], s);
                    }
                }
                s = group_sum(s, gmask);
                if (e < a1 && w == 0) ga[e] = s;
            }
            __syncwarp();                                  // the staged row is free again
        }
    }
}

// gB[(k,j)] = sum_{i in A^T_k} A[i,k] * V[i,j] for one row k of B, one warp: a group per stored
// (k,j), its lanes over A^T_k (binary search of j in C_i), then a fixed shuffle tree.  When
// A^T_k fits one entry per lane and B_k two rounds of the four groups (both at most 8), each
// lane loads its entry of A^T_k, A's value and C_i's bounds once and the two rounds' searches
// advance together; the sums are the same (one term per lane, the same tree).
__device__ __forceinline__ void grad_b_row(int64_t k, int g, int w, unsigned gmask, const int32_t* __restrict__ at_ptr,
                                           const int32_t* __restrict__ at_idx, const int32_t* __restrict__ a_perm,
                                           const float* __restrict__ a_val, const int32_t* __restrict__ b_ptr,
                                           const int32_t* __restrict__ b_idx, const int32_t* __restrict__ c_ptr,
                                           const int32_t* __restrict__ c_idx, const float* __restrict__ gc,
                                           float* __restrict__ gb) {
    const int ia = at_ptr[k], ib = at_ptr[k + 1];
    const int fb = b_ptr[k], f1 = b_ptr[k + 1];
    if (ib - ia <= GRP && f1 - fb <= 2 * NGRP) {
        const int t = ia + w;
        int c0 = 0, nc = 0;
        float aik = 0.f;
        if (t < ib) {
            const int i = at_idx[t];
            aik = a_val[a_perm[t]];
            c0 = c_ptr[i];
            nc = c_ptr[i + 1] - c0;
        }
        const int fa = fb + g, fz = fb + g + NGRP;
        const int ja = fa < f1 ? b_idx[fa] : -1, jz = fz < f1 ? b_idx[fz] : -1;
        int la = 0, lz = 0;
        for (int n = nc; n > 1;) {                         // both lower bounds, one level per step
            const int half = n >> 1;
            if (ja >= 0 && c_idx[c0 + la + half - 1] < ja) la += half;
            if (jz >= 0 && c_idx[c0 + lz + half - 1] < jz) lz += half;
            n -= half;
        }
        float sa = 0.f, sz = 0.f;
        if (nc > 0) {
            if (ja >= 0) {
                const int p = la + (c_idx[c0 + la] < ja ? 1 : 0);
                if (p < nc && c_idx[c0 + p] == ja) sa = fmaf(aik, gc[c0 + p], 0.f);
            }
            if (jz >= 0) {
                const int p = lz + (c_idx[c0 + lz] < jz ? 1 : 0);
                if (p < nc && c_idx[c0 + p] == jz) sz = fmaf(aik, gc[c0 + p], 0.f);
            }
        }
        sa = group_sum(sa, gmask);
        sz = group_sum(sz, gmask);
        if (w == 0) {
            if (fa < f1) gb[fa] = sa;
            if (fz < f1) gb[fz] = sz;
        }
        return;
    }
    for (int f0 = fb; f0 < f1; f0 += NGRP) {
        const int f = f0 + g;
        float s = 0.f;
        if (f < f1) {
            const int j = b_idx[f];
            for (int t = ia + w; t < ib; t += GRP) {
                const int i = at_idx[t];
                const float aik = a_val[a_perm[t]];
                const int c0 = c_ptr[i], nc = c_ptr[i + 1] - c0;
                const int pos = lower_bound_i32(c_idx + c0, nc, j);
                if (pos < nc && c_idx[c0 + pos] == j) s = fmaf(aik, gc[c0 + pos], s);
            }
        }
        s = group_sum(s, gmask);
        if (f < f1 && w == 0) gb[f] = s;
    }
}

// gB on every row of B, one warp per row.
__global__ void __launch_bounds__(256) grad_b_kernel(
    int32_t kb, const int32_t* __restrict__ at_ptr, const int32_t* __restrict__ at_idx,
    const int32_t* __restrict__ a_perm, const float* __restrict__ a_val, const int32_t* __restrict__ b_ptr,
    const int32_t* __restrict__ b_idx, const int32_t* __restrict__ c_ptr, const int32_t* __restrict__ c_idx,
    const float* __restrict__ gc, float* __restrict__ gb) {
    const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int g = lane / GRP, w = lane % GRP;
    const unsigned gmask = ((1u << GRP) - 1u) << (g * GRP);
    if (k >= kb) return;
    grad_b_row(k, g, w, gmask, at_ptr, at_idx, a_perm, a_val, b_ptr, b_idx, c_ptr, c_idx, gc, gb);
}

int big_grid() { return num_sms() * 2; }

spx_status check_pair(const spx_csr* A, const spx_csr* B, bool vals, const char* who) {
    SPX_TRY(check_csr(A, vals, who));
    SPX_TRY(check_csr(B, vals, who));
    if (A->n != B->m) return set_error(SPX_INVALID_ARG, "%s: inner dimensions differ (%d vs %d)", who, A->n, B->m);
    return SPX_OK;
}

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_spgemm_workspace_size(int32_t m, size_t* bytes) {
    if (!bytes || m < 0) return set_error(SPX_INVALID_ARG, "spx_spgemm_workspace_size: bad arguments");
    *bytes = gemm_layout(m).total;
    return SPX_OK;
}

extern "C" spx_status spx_spgemm_analyse(const spx_csr* A, const spx_csr* B, int64_t* products_host, void* ws,
                                         size_t ws_bytes, void* stream) {
    SPX_TRY(check_pair(A, B, false, "spx_spgemm_analyse"));
    const GemmLayout L = gemm_layout(A->m);
    if (!ws || ws_bytes < L.total)
        return set_error(SPX_OOM_WORKSPACE, "spx_spgemm_analyse: workspace %zu < %zu", ws_bytes, L.total);
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    int32_t* prod = (int32_t*)(w + L.prod);
    int64_t* pptr = (int64_t*)(w + L.pptr);
    int32_t* n_big = (int32_t*)(w + L.big_pos) + A->m;     // the count the big-row kernels read
    int32_t* brows = (int32_t*)(w + L.big_rows);
    SPX_CUDA(cudaMemsetAsync(n_big, 0, sizeof(int32_t), st), "spx_spgemm_analyse clear");
    if (A->m > 0) {
        int64_t threads = (int64_t)A->m * 8;
        products_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A->m, A->indptr, A->indices, B->indptr,
                                                                           prod, brows, n_big);
        SPX_CHECK_LAUNCH("spgemm products");
    }
    SPX_TRY((scan_counts<int32_t, int64_t>(prod, pptr, A->m, (int64_t*)(w + L.scan64), st)));
    if (products_host) {
        SPX_CUDA(cudaMemcpyAsync(products_host, pptr + A->m, sizeof(int64_t), cudaMemcpyDeviceToHost, st),
                 "spx_spgemm_analyse copy");
        SPX_CUDA(cudaStreamSynchronize(st), "spx_spgemm_analyse sync");
    }
    return SPX_OK;
}

extern "C" spx_status spx_spgemm_symbolic(const spx_csr* A, const spx_csr* B, int64_t products, int32_t* c_indptr,
                                          int64_t* nnz_c_host, void* ws, size_t ws_bytes, void* tmp, size_t tmp_bytes,
                                          void* stream) {
    SPX_TRY(check_pair(A, B, false, "spx_spgemm_symbolic"));
    if (!c_indptr || products < 0) return set_error(SPX_INVALID_ARG, "spx_spgemm_symbolic: bad arguments");
    const GemmLayout L = gemm_layout(A->m);
    if (!ws || ws_bytes < L.total)
        return set_error(SPX_OOM_WORKSPACE, "spx_spgemm_symbolic: workspace %zu < %zu", ws_bytes, L.total);
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    const int64_t* pptr = (const int64_t*)(w + L.pptr);
    if (tmp_bytes < (size_t)products * 4 || (products > 0 && !tmp))
        return set_error(SPX_OOM_WORKSPACE, "spx_spgemm_symbolic: scratch %zu < %lld", tmp_bytes,
                         (long long)products * 4);
    int32_t* row_nnz = (int32_t*)(w + L.row_nnz);
    if (A->m > 0) {
        symbolic_group_kernel<<<(unsigned)((A->m + SYG_THREADS / GRP - 1) / (SYG_THREADS / GRP)), SYG_THREADS, 0,
                                st>>>(A->m, A->indptr, A->indices, B->indptr, B->indices,
                                      (const int32_t*)(w + L.prod), pptr, (int32_t*)tmp, row_nnz);
        SPX_CHECK_LAUNCH("spgemm symbolic small rows");
        const int64_t wblocks = ((int64_t)A->m + 32 * SYM_WARPS - 1) / (32 * SYM_WARPS);
        const int64_t wcap = (int64_t)num_sms() * 8;
        symbolic_warp_kernel<<<(unsigned)(wblocks < wcap ? wblocks : wcap), SYM_WARPS * 32, 0, st>>>(
            A->m, A->indptr, A->indices, B->indptr, B->indices, (const int32_t*)(w + L.prod), pptr, (int32_t*)tmp,
            row_nnz);
        SPX_CHECK_LAUNCH("spgemm symbolic");
        symbolic_big_kernel<<<big_grid(), BIG_THREADS, 0, st>>>(
            (const int32_t*)(w + L.big_rows), (const int32_t*)(w + L.big_pos) + A->m, B->n, A->indptr, A->indices,
            B->indptr, B->indices, pptr, (int32_t*)tmp, row_nnz);
        SPX_CHECK_LAUNCH("spgemm symbolic big");
    }
    SPX_TRY((scan_counts<int32_t, int32_t>(row_nnz, c_indptr, A->m, (int32_t*)(w + L.scan32), st)));
    if (nnz_c_host) {
        int32_t nnz = 0;
        SPX_CUDA(cudaMemcpyAsync(&nnz, c_indptr + A->m, sizeof(int32_t), cudaMemcpyDeviceToHost, st),
                 "spx_spgemm_symbolic copy");
        SPX_CUDA(cudaStreamSynchronize(st), "spx_spgemm_symbolic sync");
        *nnz_c_host = nnz;
    }
    return SPX_OK;
}

extern "C" spx_status spx_spgemm_fill(const spx_csr* A, const int32_t* c_indptr, int32_t* c_indices, const void* ws,
                                      size_t ws_bytes, const void* tmp, void* stream) {
    SPX_TRY(check_csr(A, false, "spx_spgemm_fill"));
    const GemmLayout L = gemm_layout(A->m);
    if (!ws || ws_bytes < L.total) return set_error(SPX_OOM_WORKSPACE, "spx_spgemm_fill: workspace too small");
    if (!c_indptr || !c_indices) return set_error(SPX_INVALID_ARG, "spx_spgemm_fill: NULL output");
    if (A->m == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    const char* w = static_cast<const char*>(ws);
    int64_t threads = (int64_t)A->m * FILL_LANES;
    fill_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(A->m, (const int64_t*)(w + L.pptr),
                                                                     (const int32_t*)tmp, c_indptr, c_indices);
    SPX_CHECK_LAUNCH("spgemm fill");
    return SPX_OK;
}

extern "C" spx_status spx_spgemm_numeric(const spx_csr* A, const spx_csr* B, const spx_csr* C, float* c_values,
                                         const void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_pair(A, B, true, "spx_spgemm_numeric"));
    SPX_TRY(check_csr(C, false, "spx_spgemm_numeric"));
    if (C->m != A->m || C->n != B->n) return set_error(SPX_INVALID_ARG, "spx_spgemm_numeric: C shape");
    const GemmLayout L = gemm_layout(A->m);
    if (!ws || ws_bytes < L.total) return set_error(SPX_OOM_WORKSPACE, "spx_spgemm_numeric: workspace too small");
    if (C->nnz > 0 && !c_values) return set_error(SPX_INVALID_ARG, "spx_spgemm_numeric: NULL output");
    if (A->m == 0) return SPX_OK;
    cudaStream_t st = as_stream(stream);
    const char* w = static_cast<const char*>(ws);
    numeric_group_kernel<<<(unsigned)((A->m + SG_THREADS / GRP - 1) / (SG_THREADS / GRP)), SG_THREADS, 0, st>>>(
        A->m, A->indptr, A->indices, A->values, B->indptr, B->indices, B->values, C->indptr, C->indices,
        (const int32_t*)(w + L.prod), c_values);
    SPX_CHECK_LAUNCH("spgemm numeric small rows");
    const int64_t wblocks = ((int64_t)A->m + 32 * NUM_WARPS - 1) / (32 * NUM_WARPS);
    const int64_t wcap = (int64_t)num_sms() * 16;
    numeric_warp_kernel<<<(unsigned)(wblocks < wcap ? wblocks : wcap), NUM_WARPS * 32, 0, st>>>(
        A->m, A->indptr, A->indices, A->values, B->indptr, B->indices, B->values, C->indptr, C->indices,
        (const int32_t*)(w + L.prod), c_values);
    SPX_CHECK_LAUNCH("spgemm numeric");
    numeric_big_kernel<<<big_grid(), BIG_THREADS, 0, st>>>(
        (const int32_t*)(w + L.big_rows), (const int32_t*)(w + L.big_pos) + A->m, A->indptr, A->indices, A->values,
        B->indptr, B->indices, B->values, C->indptr, C->indices, c_values);
    SPX_CHECK_LAUNCH("spgemm numeric big");
    return SPX_OK;
}

extern "C" spx_status spx_spgemm_backward(const spx_csr* A, const spx_csr* B, const spx_csr* C, const float* gc,
                                          float* ga, float* gb, const int32_t* at_indptr, const int32_t* at_indices,
                                          const int32_t* a_perm, void* stream) {
    SPX_TRY(check_pair(A, B, false, "spx_spgemm_backward"));
    SPX_TRY(check_csr(C, false, "spx_spgemm_backward"));
    if (C->m != A->m || C->n != B->n) return set_error(SPX_INVALID_ARG, "spx_spgemm_backward: C shape");
    if (C->nnz > 0 && !gc) return set_error(SPX_INVALID_ARG, "spx_spgemm_backward: NULL V");
    cudaStream_t st = as_stream(stream);
    if (ga && A->m > 0) {
        if (B->nnz > 0 && !B->values) return set_error(SPX_INVALID_ARG, "spx_spgemm_backward: B values needed");
        grad_a_group_kernel<<<(unsigned)((A->m + SG_THREADS / GRP - 1) / (SG_THREADS / GRP)), SG_THREADS, 0, st>>>(
            A->m, A->indptr, A->indices, B->indptr, B->indices, B->values, C->indptr, C->indices, gc, ga);
        SPX_CHECK_LAUNCH("spgemm grad_a small rows");
        const int64_t wb = ((int64_t)A->m + 32 * NUM_WARPS - 1) / (32 * NUM_WARPS);
        const int64_t cap = (int64_t)num_sms() * 16;
        grad_a_kernel<<<(unsigned)(wb < cap ? wb : cap), NUM_WARPS * 32, 0, st>>>(
            A->m, A->indptr, A->indices, B->indptr, B->indices, B->values, C->indptr, C->indices, gc, ga);
        SPX_CHECK_LAUNCH("spgemm grad_a");
    }
    if (gb && B->m > 0) {
        if (!at_indptr || (A->nnz > 0 && (!at_indices || !a_perm || !A->values)))
            return set_error(SPX_INVALID_ARG, "spx_spgemm_backward: grad B needs A's transpose and values");
        const int64_t threads = (int64_t)B->m * 32;
        grad_b_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
            B->m, at_indptr, at_indices, a_perm, A->values, B->indptr, B->indices, C->indptr, C->indices, gc, gb);
        SPX_CHECK_LAUNCH("spgemm grad_b");
    }
    return SPX_OK;
}
