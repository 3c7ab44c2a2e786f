// Zero-fill incomplete Cholesky IC(0) of a block-diagonal SPD batch -- the baseline
// preconditioner M = (L L^T)^-1 whose application is two sparse triangular solves
// (Section 3.1.5) -- and the level schedule those solves need.
//
// Levels: level(i) = 0 if row i of L has no off-diagonal entry, else 1 + max level(j)
// over its entries j < i.  Rows of one level are independent in the forward solve (and,
// in reverse level order, in the transposed solve).  The schedule is built per system by
// one thread (a sequential pass over the rows, O(nnz)), then rows are bucketed by level.
//
// Factorisation (Saad, Sec. 10.3): level by level, one thread per row:
//   L_ik = (a_ik - sum_{j<k} L_ij L_kj) / L_kk  (k < i, in column order),
//   L_ii = sqrt(a_ii - sum_{j<i} L_ij^2),
// with the sums over the columns stored in both rows; one thread block per system.
// A non-positive pivot sets the system's status to SPX_BREAKDOWN.
#include <math.h>

#include "common.cuh"
#include "scan.cuh"

namespace spx {
namespace {

__global__ void ic0_levels_kernel(int32_t nsys, const int32_t* __restrict__ sys_ptr, const int32_t* __restrict__ lptr,
                                  const int32_t* __restrict__ lidx, int32_t* __restrict__ level,
                                  int32_t* __restrict__ nlev) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    int mx = -1;
    for (int i = sys_ptr[s]; i < sys_ptr[s + 1]; ++i) {
        int lv = 0;
        for (int e = lptr[i]; e < lptr[i + 1]; ++e) {
            const int j = lidx[e];
            if (j < i) lv = max(lv, level[j] + 1);
        }
        level[i] = lv;
        mx = max(mx, lv);
    }
    nlev[s] = mx + 2;                    // levels + 1 pointer slots
}

// rows bucketed by level: lev_ptr[off_s + l] .. lev_ptr[off_s + l + 1] index lev_rows
__global__ void ic0_buckets_kernel(int32_t nsys, const int32_t* __restrict__ sys_ptr,
                                   const int32_t* __restrict__ level, const int32_t* __restrict__ off,
                                   int32_t* __restrict__ lev_ptr, int32_t* __restrict__ lev_rows) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const int R0 = sys_ptr[s], R1 = sys_ptr[s + 1];
    int32_t* lp = lev_ptr + off[s];
    const int nl = off[s + 1] - off[s] - 1;
    for (int l = 0; l <= nl; ++l) lp[l] = 0;
    for (int i = R0; i < R1; ++i) lp[level[i] + 1] += 1;
    lp[0] = R0;
    for (int l = 1; l <= nl; ++l) lp[l] += lp[l - 1];
    // fill (stable: rows increasing within a level); lp[l] is used as a cursor, then restored
    for (int i = R0; i < R1; ++i) lev_rows[lp[level[i]]++] = i;
    for (int l = nl; l >= 1; --l) lp[l] = lp[l - 1];
    lp[0] = R0;
}

__device__ __forceinline__ int find_col(const int32_t* __restrict__ idx, int beg, int end, int j) {
    int lo = beg, hi = end;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (idx[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && idx[lo] == j) ? lo : -1;
}

__global__ void __launch_bounds__(512) ic0_factor_kernel(
    int32_t nsys, const int32_t* __restrict__ off, const int32_t* __restrict__ lev_ptr,
    const int32_t* __restrict__ lev_rows, const int32_t* __restrict__ lptr, const int32_t* __restrict__ lidx,
    const int32_t* __restrict__ lsrc, const float* __restrict__ a_val, float* __restrict__ lval,
    int32_t* __restrict__ status) {
    const int s = blockIdx.x;
    if (s >= nsys) return;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    const int32_t* lp = lev_ptr + off[s];
    const int nl = off[s + 1] - off[s] - 1;
    for (int l = 0; l < nl; ++l) {
        for (int q = lp[l] + threadIdx.x; q < lp[l + 1]; q += blockDim.x) {
            const int i = lev_rows[q];
            const int b0 = lptr[i], b1 = lptr[i + 1];
            for (int e = b0; e < b1; ++e) {
                const int k = lidx[e];
                float v = a_val[lsrc[e]];
                for (int f = b0; f < e; ++f) {
                    const int g = find_col(lidx, lptr[k], lptr[k + 1], lidx[f]);
                    if (g >= 0) v = fmaf(-lval[f], lval[g], v);
                }
                if (k < i) {
                    lval[e] = v / lval[lptr[k + 1] - 1];       // diagonal last in row k
                } else {
                    if (!(v > 0.f)) {
                        bad = 1;
                        v = 1.f;
                    }
                    lval[e] = sqrtf(v);
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) status[s] = bad ? SPX_BREAKDOWN : SPX_OK;
}

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace spx

using namespace spx;

extern "C" spx_status spx_ic0_workspace_size(int32_t n, int32_t nsys, size_t* bytes) {
    if (!bytes || n < 0 || nsys < 0) return set_error(SPX_INVALID_ARG, "spx_ic0_workspace_size");
    *bytes = al(4 * (size_t)n) + al(4 * (size_t)nsys + 4) + scan_workspace_bytes<int32_t>(nsys) + 256;
    return SPX_OK;
}

extern "C" spx_status spx_ic0_analyse(const spx_csr* Lpat, const int32_t* sys_ptr, int32_t nsys, int32_t* sys_lev_off,
                                      int32_t* lev_ptr, int32_t* lev_rows, void* ws, size_t ws_bytes, void* stream) {
    SPX_TRY(check_csr(Lpat, false, "spx_ic0_analyse"));
    size_t need = 0;
    spx_ic0_workspace_size(Lpat->m, nsys, &need);
    if (!ws || ws_bytes < need) return set_error(SPX_OOM_WORKSPACE, "spx_ic0_analyse: workspace too small");
    if (nsys == 0) return SPX_OK;
    if (!sys_ptr || !sys_lev_off || !lev_ptr || !lev_rows) return set_error(SPX_INVALID_ARG, "spx_ic0_analyse: NULL");
    cudaStream_t st = as_stream(stream);
    char* w = static_cast<char*>(ws);
    int32_t* level = (int32_t*)w;
    int32_t* nlev = (int32_t*)(w + al(4 * (size_t)Lpat->m));
    int32_t* sws = (int32_t*)(w + al(4 * (size_t)Lpat->m) + al(4 * (size_t)nsys + 4));
    const unsigned g = (unsigned)((nsys + 63) / 64);
    ic0_levels_kernel<<<g, 64, 0, st>>>(nsys, sys_ptr, Lpat->indptr, Lpat->indices, level, nlev);
    SPX_CHECK_LAUNCH("ic0 levels");
    SPX_TRY((scan_counts<int32_t, int32_t>(nlev, sys_lev_off, nsys, sws, st)));
    ic0_buckets_kernel<<<g, 64, 0, st>>>(nsys, sys_ptr, level, sys_lev_off, lev_ptr, lev_rows);
    SPX_CHECK_LAUNCH("ic0 buckets");
    return SPX_OK;
}

extern "C" spx_status spx_ic0_factor(const spx_csr* Lpat, const int32_t* l_src, const float* a_values, int32_t nsys,
                                     const int32_t* sys_lev_off, const int32_t* lev_ptr, const int32_t* lev_rows,
                                     float* l_values, int32_t* status, void* stream) {
    SPX_TRY(check_csr(Lpat, false, "spx_ic0_factor"));
    if (nsys == 0) return SPX_OK;
    if (!l_src || !a_values || !sys_lev_off || !lev_ptr || !lev_rows || !l_values || !status)
        return set_error(SPX_INVALID_ARG, "spx_ic0_factor: NULL argument");
    ic0_factor_kernel<<<nsys, 512, 0, as_stream(stream)>>>(nsys, sys_lev_off, lev_ptr, lev_rows, Lpat->indptr,
                                                           Lpat->indices, l_src, a_values, l_values, status);
    SPX_CHECK_LAUNCH("spx_ic0_factor");
    return SPX_OK;
}
