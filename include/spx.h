/*
 * spx.h -- C ABI of the GB300 (sm_103a) sparse forward / reverse-mode kernels.
 *
 * The operations follow "Optimized Sparse Matrix Operations for Reverse Mode
 * Automatic Differentiation" (arXiv 2212.05159): CSR matrices (Section 3), the
 * vector-Jacobian products of Table 1, with gradients of sparse inputs kept on the
 * input's own sparsity pattern (Section 3.1, "Sparse Methods").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an spx_status; SPX_OK is 0.  Nothing throws or aborts
 *   across the ABI.  spx_last_error() returns a thread-local message describing the
 *   most recent failure on the calling thread.
 * - The caller owns all memory.  Pointers marked "device" must be device memory of
 *   the current CUDA device; pointers marked "host" are host memory.  No entry point
 *   allocates device memory except where its comment says so; scratch space is a
 *   caller-provided workspace whose size a *_workspace_size() query returns.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *   are asynchronous on that stream unless their comment says they synchronize it.
 * - Integers: int32 row/column indices and indptr entries (nnz < 2^31); values are
 *   IEEE float32 on the device.  Dense operands are row-major with a leading
 *   dimension (ld*, in elements, >= the number of columns).
 * - CSR patterns must have sorted, unique column indices per row.  spx_csr_validate()
 *   checks a pattern on the device; the compute entry points do not re-check it.
 * - mask(A) is the *structural* pattern of A: every stored entry, including stored
 *   zeros, belongs to it (reading of the mask definition in Section 3).
 */
#ifndef SPX_H
#define SPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum spx_status {
    SPX_OK = 0,
    SPX_INVALID_ARG = 1,     /* a pointer, size or leading dimension is unusable */
    SPX_BAD_PATTERN = 2,     /* indptr not monotone, or an index out of range */
    SPX_UNSORTED = 3,        /* column indices not strictly increasing in a row */
    SPX_OOM_WORKSPACE = 4,   /* the workspace passed is smaller than required */
    SPX_MAXITER = 5,         /* an iterative solve hit its iteration limit */
    SPX_BREAKDOWN = 6,       /* CG breakdown: p^T A p <= 0 or r^T z <= 0 */
    SPX_NONFINITE = 7,       /* a NaN / Inf appeared */
    SPX_DEVICE_TIMEOUT = 8,  /* a bounded device-side wait ran out */
    SPX_CUDA_ERROR = 9,      /* a CUDA runtime call failed (see spx_last_error) */
    SPX_NOT_SUPPORTED = 10   /* the combination of arguments is not implemented */
} spx_status;

/* A CSR matrix view (Section 3): m x n, nnz stored entries.
 * indptr: device int32[m+1], indptr[0] = 0, indptr[m] = nnz, non-decreasing.
 * indices: device int32[nnz], column of each entry, sorted and unique per row.
 * values: device float32[nnz] (may be NULL where only the pattern is read). */
typedef struct spx_csr {
    int32_t m;
    int32_t n;
    int64_t nnz;
    const int32_t* indptr;
    const int32_t* indices;
    const float* values;
} spx_csr;

/* Load-balancing plan of a CSR pattern for the row-wise products (spx_spmm,
 * spx_spmm_t): the rows longer than `threshold` entries, processed by a whole thread
 * block each instead of one warp.  Built once per pattern by spx_rowplan_build(). */
typedef struct spx_rowplan {
    const int32_t* long_rows; /* device int32[n_long], increasing row ids */
    int32_t n_long;           /* host-known count */
    int32_t threshold;        /* rows with more than this many entries are "long" */
    int32_t col_block;        /* dense columns per pass (0 = all k in one pass); narrower
                                 blocks gather from column-block slabs of the dense
                                 operand repacked into the workspace, one pass per block */
    int32_t rows_per_group;   /* rows walked by one lane group (0 = default) */
    int32_t engine;           /* gathers of the dense rows: 0 = loads into registers,
                                 1 = TMA-engine bulk copies into shared memory (needs k and
                                 the leading dimensions multiples of 4 and 16-byte aligned
                                 operands; otherwise 0 is used), 2 = loads into registers
                                 with no batch prefetched ahead, for more resident warps
                                 (one pass over all k, same conditions as 1; otherwise 0) */
    const int32_t* medium_rows; /* device int32[n_medium]: rows with medium_threshold < length
                                   <= threshold, one warp each (NULL / 0 = none) */
    int32_t n_medium;
    int32_t medium_threshold;
    const int32_t* part_ptr;  /* device int32[(n_parts - 1) * m] or NULL: column-range split of
                                 every row, written by spx_rowplan_build_parts.  With
                                 n_parts > 1 the products run one pass per range of the dense
                                 operand's rows (A's columns [p * ceil(n / n_parts), ...)), so
                                 the part gathered in a pass can stay resident in L2; the
                                 passes add into the output in range order. */
    int32_t n_parts;          /* 0 or 1 = one pass over all columns */
    const int32_t* short_rows; /* device int32[n_short] or NULL: the order in which the short-row
                                  path (rows of at most medium_threshold entries, or threshold
                                  without a medium list) walks its rows, from
                                  spx_rowplan_build_short: grouped by length so that the lane
                                  groups of a warp walk rows of about the same length; NULL =
                                  every row in natural order.  Results do not depend on it. */
    int32_t n_short;
} spx_rowplan;

/* ------------------------------------------------------------------ library */

/* Waits for `stream`, then reads and clears the library's device-side error word:
 * SPX_DEVICE_TIMEOUT if a kernel's bounded wait (e.g. on a TMA copy) ran out since the
 * last check, else SPX_OK. */
spx_status spx_check_device(void* stream);

/* Message of the most recent failure on the calling thread ("" if none). */
const char* spx_last_error(void);

/* Static name of a status code ("SPX_OK", ...). */
const char* spx_status_name(int status);

/* ABI version: major * 10000 + minor * 100 + patch. */
int32_t spx_version(void);

/* Validates a CSR pattern on the device: indptr[0] == 0, indptr[m] == nnz,
 * indptr non-decreasing, 0 <= indices < n, strictly increasing within each row.
 * Synchronizes `stream`; returns SPX_OK, SPX_BAD_PATTERN or SPX_UNSORTED.
 * workspace: device, >= 16 bytes. */
spx_status spx_csr_validate(const spx_csr* A, void* workspace, size_t workspace_bytes,
                            void* stream);

/* ------------------------------------------------ SpMV / SpMM (Section 3.1.1, 3.1.3) */

/* Workspace bytes needed by spx_rowplan_build for an m-row pattern. */
spx_status spx_rowplan_workspace_size(int32_t m, size_t* bytes);

/* Builds the row plan of A's pattern: writes the ids of rows with more than
 * `threshold` entries, in increasing order, to long_rows (device int32[m]) and their
 * count to *n_long_host.  Synchronizes `stream` (the count is returned to the host). */
spx_status spx_rowplan_build(const spx_csr* A, int32_t threshold, int32_t* long_rows,
                             int32_t* n_long_host, void* workspace, size_t workspace_bytes,
                             void* stream);

/* Column-range split of A's rows for plans with n_parts > 1 (no counterpart in the paper;
 * a layout choice for operands larger than L2).  With w = ceil(n / n_parts), writes
 * part_ptr[(p - 1) * m + i] = the offset of the first entry of row i whose column is
 * >= p * w, for p = 1 .. n_parts - 1 (rows sorted, so these offsets split each row into
 * n_parts consecutive segments).  part_ptr: device int32[(n_parts - 1) * m], caller-owned.
 * Asynchronous on `stream`.  Returns SPX_INVALID_ARG for n_parts < 2 or n_parts > n. */
spx_status spx_rowplan_build_parts(const spx_csr* A, int32_t n_parts, int32_t* part_ptr, void* stream);

/* Workspace bytes with which spx_spmm repacks X into column-block slabs (0 when the
 * gathered operand fits the L2 budget, or k is not a multiple of 4). */
spx_status spx_spmm_workspace_size(const spx_csr* A, int32_t k, const spx_rowplan* plan,
                                   size_t* bytes);

/* Scheduling of the row-wise products of Sections 3.1.1 / 3.1.3 (SpMM, A^T G) and of the
 * SDDMM VJP.  Builds a plan's short-row order: the ids of the rows with at most `threshold` entries,
 * grouped by their number of 8-entry batches (more than 8 batches share one group),
 * groups in decreasing length, ids increasing within a group (stable), into short_rows
 * (device int32[m]); count to *n_short_host, number of non-empty groups to *n_groups_host
 * (may be NULL; with one group the order is the natural one and gains nothing -- measured
 * 5 % slower on the 3D Poisson stencil, 16 % faster SpMM on the power-law matrix at k = 32).
 * Same workspace as spx_rowplan_build.  Synchronizes `stream`. */
spx_status spx_rowplan_build_short(const spx_csr* A, int32_t threshold, int32_t* short_rows,
                                   int32_t* n_short_host, int32_t* n_groups_host, void* workspace,
                                   size_t workspace_bytes, void* stream);

/* Builds the medium-row list of a plan: ids of rows with medium_threshold < length <=
 * long_threshold, increasing, into medium_rows (device int32[m]), count to
 * *n_medium_host.  Same workspace as spx_rowplan_build.  Synchronizes `stream`. */
spx_status spx_rowplan_build_medium(const spx_csr* A, int32_t medium_threshold,
                                    int32_t long_threshold, int32_t* medium_rows,
                                    int32_t* n_medium_host, void* workspace,
                                    size_t workspace_bytes, void* stream);

/* Sparse x dense product (Section 3.1.3; SpMV of Section 3.1.1 when k = 1):
 *   Y = alpha * A X + beta * Y.
 * A: m x n CSR with values.  X: device float32, n rows x k columns, leading dim ldx.
 * Y: device float32, m x k, leading dim ldy; not read when beta == 0.
 * plan: optional row plan (NULL = no long-row blocks, default column blocks).
 * workspace: device scratch of spx_spmm_workspace_size() bytes, or NULL.  With it, X is
 * first repacked into contiguous column-block slabs so that each pass's gathered slab
 * fits in L2; without it the passes gather the strided X directly (same results).
 * A non-NULL workspace smaller than required is an error (SPX_OOM_WORKSPACE).
 * Each output element is reduced in a fixed order: results are run-to-run
 * deterministic. */
spx_status spx_spmm(const spx_csr* A, const float* X, int64_t ldx, int32_t k, float* Y,
                    int64_t ldy, float alpha, float beta, const spx_rowplan* plan,
                    void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------- reverse mode of SpMV / SpMM (Table 1) */

/* Workspace bytes with which spx_sddmm repacks X into column-block slabs. */
spx_status spx_sddmm_workspace_size(const spx_csr* A, int32_t k, int32_t col_block,
                                    size_t* bytes);

/* Gradient w.r.t. the sparse matrix of Y = A X (Table 1, SpMV/SpDMM row "A"):
 *   out[e] = scale * sum_c G[i,c] * X[j,c]   for every stored entry e = (i, j) of A,
 * i.e. (G X^T) masked to mask(A) -- an SDDMM.  A.values is not read.
 * G: device float32 m x k (ldg); X: device float32 n x k (ldx); out: device float32[nnz].
 * col_block: dense columns per pass (0 = all k in one pass); with several passes
 * the partial dot products are added into out in column order.
 * plan: optional row plan of A (spx_rowplan_build[_medium]); with it rows are binned as in
 * spx_spmm and each lane group keeps G's row in registers, without it every warp takes an
 * equal slice of the entries; its rows_per_group and n_parts fields apply, its col_block
 * and engine fields are not used (col_block is the argument).
 * workspace: device scratch of spx_sddmm_workspace_size() bytes, or NULL (as spx_spmm). */
spx_status spx_sddmm(const spx_csr* A, const float* G, int64_t ldg, const float* X,
                     int64_t ldx, int32_t k, float scale, float* out, int32_t col_block,
                     const spx_rowplan* plan, void* workspace, size_t workspace_bytes,
                     void* stream);

/* The k = 1 case: out[e] = scale * u[i] * v[j] on mask(A) (Table 1, SpMV row "A";
 * with scale = -1 and u = lambda, v = x it is the SpSolve gradient w.r.t. A).
 * u: device float32[m]; v: device float32[n]. */
spx_status spx_masked_outer(const spx_csr* A, const float* u, const float* v, float scale,
                            float* out, void* stream);

/* Workspace bytes needed by spx_csr_transpose. */
spx_status spx_transpose_workspace_size(int32_t m, int32_t n, int64_t nnz, size_t* bytes);

/* Sparse transpose of A's pattern (Section 3.1.3 forms A^T to compute A^T V):
 * t_indptr: device int32[n+1]; t_indices: device int32[nnz] (row ids of A, sorted
 * within each row of A^T); perm: device int32[nnz] with
 *   A^T.values[e'] = A.values[perm[e']].
 * Stable and deterministic.  A.values is not read. */
spx_status spx_csr_transpose(const spx_csr* A, int32_t* t_indptr, int32_t* t_indices,
                             int32_t* perm, void* workspace, size_t workspace_bytes,
                             void* stream);

/* Workspace bytes for spx_spmm_t: A^T's gathered values (4 * nnz) plus the column-block
 * slabs of G (as spx_spmm).  AT is the transposed pattern (see below). */
spx_status spx_spmm_t_workspace_size(const spx_csr* AT, int32_t k, const spx_rowplan* plan,
                                     size_t* bytes);

/* Gradient w.r.t. the dense operand of Y = A X (Table 1, SpMV/SpDMM row "x"/"B"):
 *   gX = alpha * A^T G + beta * gX,
 * computed as a row-wise product over the transposed pattern (no atomics;
 * deterministic).  A's values reach A^T's order through perm: with a workspace they
 * are gathered once into it (one streaming pass) and G is repacked into slabs;
 * with workspace == NULL every pass gathers the values through perm.
 * AT: the pattern of A^T from spx_csr_transpose (m = A.n rows, n = A.m columns) with
 *     AT.values = A.values (in A's order).  perm: device int32[nnz].
 * G: device float32 A.m x k (ldg).  gX: device float32 A.n x k (ldgx).
 * plan: optional row plan of the transposed pattern.
 * workspace: device scratch of spx_spmm_t_workspace_size() bytes or NULL; a non-NULL
 * workspace that is too small is an error. */
spx_status spx_spmm_t(const spx_csr* AT, const int32_t* perm, const float* G, int64_t ldg,
                      int32_t k, float* gX, int64_t ldgx, float alpha, float beta,
                      const spx_rowplan* plan, void* workspace, size_t workspace_bytes,
                      void* stream);

/* Both gradients of Y = A X in one pass over A^T (Table 1, SpDMM rows, w.r.t. A and X):
 *   gX = alpha * A^T G + beta * gX,
 *   gA[p] = scale * <G_i, X_j> for the entry a_ij stored at position p of A (SDDMM),
 * exactly the products of spx_spmm_t and spx_sddmm, computed together: row j of A^T
 * gathers the rows G_i of its entries once and uses each for both (X_j is read once per
 * row), so the pass has one random gather stream instead of two.  A's values are read
 * through perm, which also places each gA entry.  Deterministic (fixed-order sums).
 * AT: the pattern of A^T from spx_csr_transpose (m = A.n rows, n = A.m columns; values
 * unused); perm: device int32[nnz]; a_values: A's values in A's order (float32[nnz]).
 * G: device float32 A.m x k (ldg); X: device float32 A.n x k (ldx), the forward's
 * operand; gX: device float32 A.n x k (ldgx); gA: device float32[nnz] in A's order.
 * k a multiple of 4 in 4..128; dense operands 16-byte aligned with ld % 4 == 0.
 * plan: optional row plan of the transposed pattern (its row lists and order are used;
 * column blocks and parts are not).  variant: 0..5, launch shapes with the same result (1
 * requests every gathered row of a batch before using any; 2 and 3 keep more blocks
 * resident with fewer registers; 4 and 5 also hold no batch ahead; the faster one depends
 * on k and the pattern, chosen by timing).  Other k: SPX_NOT_SUPPORTED (use the two
 * calls). */
spx_status spx_spmm_t_sddmm(const spx_csr* AT, const int32_t* perm, const float* a_values,
                            const float* G, int64_t ldg, const float* X, int64_t ldx, int32_t k,
                            float* gX, int64_t ldgx, float alpha, float beta, float* gA,
                            float scale, const spx_rowplan* plan, int32_t variant, void* stream);

/* ------------------------------------- SpSpMM / SpGEMM (Section 3.1.2, Table 1) */

/* Workspace bytes of the SpGEMM calls for an m-row A (per-row counts, offsets and the
 * list of rows too large for one warp).  The same workspace must be passed to
 * analyse, symbolic, fill and numeric of one product, in that order. */
spx_status spx_spgemm_workspace_size(int32_t m, size_t* bytes);

/* C = A B, step 1 (expand): per-row product counts P_i = sum_{k in A_i} |B_k| and their
 * prefix sums.  Writes the total number of products to *products_host; the symbolic
 * step needs 4 * products bytes of scratch.  A, B patterns only.  Synchronizes to return
 * the count; with products_host NULL (a caller that knows the count, e.g. from an earlier
 * analysis of the same patterns) it is asynchronous. */
spx_status spx_spgemm_analyse(const spx_csr* A, const spx_csr* B, int64_t* products_host,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Step 2 (sort / compress): the pattern of C is the structural product -- every (i, j)
 * reached by some A_ik B_kj, with no dropping of numerical zeros.  Writes C_indptr
 * (device int32[m+1]) and nnz(C) to *nnz_c_host, and keeps each row's sorted unique
 * columns in `scratch` (device, >= 4 * products bytes) for spx_spgemm_fill.  products: the
 * count spx_spgemm_analyse returned (sizes the scratch check without a read-back).
 * Rows of at most 64 products are sorted in registers (bitonic network over shuffles),
 * longer ones in shared memory or, above 512, with a block bitmap.  Synchronizes once to
 * return nnz(C); with nnz_c_host NULL it is asynchronous (nnz(C) = C_indptr[m] on the
 * device). */
spx_status spx_spgemm_symbolic(const spx_csr* A, const spx_csr* B, int64_t products,
                               int32_t* c_indptr, int64_t* nnz_c_host, void* workspace,
                               size_t workspace_bytes, void* scratch, size_t scratch_bytes,
                               void* stream);

/* Step 3: C_indices (device int32[nnz(C)], sorted within rows) from the scratch. */
spx_status spx_spgemm_fill(const spx_csr* A, const int32_t* c_indptr, int32_t* c_indices,
                           const void* workspace, size_t workspace_bytes, const void* scratch,
                           void* stream);

/* Step 4: C values on C's pattern, C_ij = sum_{k in A_i, in A's order} A_ik B_kj
 * (deterministic).  C: the pattern from steps 2-3 (C.values ignored); c_values: device
 * float32[nnz(C)].  Needs the workspace of step 1 (row classes).  May be repeated for
 * new values of A and B with the same patterns. */
spx_status spx_spgemm_numeric(const spx_csr* A, const spx_csr* B, const spx_csr* C,
                              float* c_values, const void* workspace, size_t workspace_bytes,
                              void* stream);

/* Reverse mode of C = A B with V = dL/dC given on C's pattern (Table 1, SpSpMM):
 *   ga[(i,k)] = sum_{j in B_k} V_ij B_kj          ((V B^T) masked to A; needs B.values)
 *   gb[(k,j)] = sum_{i : A_ik stored} A_ik V_ij   ((A^T V) masked to B; needs A.values and
 *                                                   A's transpose from spx_csr_transpose)
 * Either output may be NULL.  gc: device float32[nnz(C)]; ga: float32[nnz(A)];
 * gb: float32[nnz(B)].  Deterministic. */
spx_status spx_spgemm_backward(const spx_csr* A, const spx_csr* B, const spx_csr* C,
                               const float* gc, float* ga, float* gb,
                               const int32_t* at_indptr, const int32_t* at_indices,
                               const int32_t* a_perm, void* stream);

/* ------------------------------------------------------- solver conveniences */

/* z = M r for the preconditioners of spx_cg_batched, applied outside the solver (e.g. to
 * use a learned M elsewhere): pc_kind 0 z = r; 1 z = pc_diag_inv .* r; 2 z = L (LT r) with
 * LT the CSR of L^T with values (tmp: device float32[n]); 3 z = L r for an explicit M passed
 * as L; 4 (IC(0)) z = L^-T (L^-1 r) by two spx_sptrsv solves with the level schedule
 * ic0_levels of nsys systems (tmp: device float32[n]).  r, z: device float32[n], distinct.
 * Asynchronous. */
spx_status spx_precond_apply(int32_t pc_kind, int64_t n, const float* r, float* z,
                             const float* pc_diag_inv, const spx_csr* L, const spx_csr* LT,
                             int32_t nsys, const int32_t* const* ic0_levels, float* tmp, void* stream);

/* The SpSolve VJP of Table 1 in one call, for a batch solved with spx_cg_batched: lambda =
 * A^-T g (A symmetric, so the same PCG with right-hand side g; lambda: device float64[n],
 * = grad_b), then grad_A = -(lambda x^T) on mask(A) (device float32[nnz], or NULL to skip;
 * x: the forward solution, device float64[n]).  The remaining arguments are those of
 * spx_cg_batched and have the same meaning; iters / status / relres describe the adjoint
 * solve.  Asynchronous. */
spx_status spx_cg_adjoint(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys,
                          const int32_t* order, const double* x, const float* g, double* lambda,
                          float* grad_A, int32_t pc_kind, const float* pc_diag_inv,
                          const spx_csr* L, const spx_csr* LT, const int32_t* const* ic0_levels,
                          double tol, int32_t maxit, double delta, int32_t* iters, int32_t* status,
                          double* relres, void* workspace, size_t workspace_bytes, void* stream);

/* Chooses the launch parameters of spx_spmm for A and width k by timing on `stream`: rows
 * per lane group 1, 2, 4, 8 and both gather engines (when the operands allow the TMA
 * engine), one pass over all k columns; keeps the plan's row lists and column parts.  X, Y:
 * the operands to time with (Y is overwritten).  Writes the fastest into *plan and its time
 * (ms per call) into *best_ms.  Synchronizes `stream`. */
spx_status spx_spmm_autotune(const spx_csr* A, const float* X, int64_t ldx, int32_t k, float* Y,
                             int64_t ldy, spx_rowplan* plan, float* best_ms, void* stream);

/* Copies n status words (e.g. the per-system status of spx_cg_batched) from the device to
 * status_host after the work queued on `stream`, checks the device error word like
 * spx_check_device, and returns SPX_OK if every word is SPX_OK, else the first one that is
 * not (with its index in spx_last_error()).  Synchronizes `stream`. */
spx_status spx_sync_status(const int32_t* status_dev, int32_t n, int32_t* status_host, void* stream);

/* ------------------------------------------ sparse triangular solve (Section 3.1.5) */

/* Solves T x = b for every system of a block-diagonal batch of triangular systems.
 * upper = 0: T is lower triangular with the diagonal stored as the last entry of each row
 * (sorted columns); upper = 1: T is the CSR of L^T for such an L (upper triangular, the
 * diagonal first in each row), which gives the transposed solve L^T x = b of the VJP
 * (grad_b = L^-T v; grad_L = -(L^-T v) x^T on mask(L), i.e. spx_masked_outer with scale -1).
 * {sys_lev_off, lev_ptr, lev_rows}: the level schedule of L's pattern from spx_ic0_analyse
 * (used in reverse order for upper = 1).  b, x: device float32[n]; status: device
 * int32[nsys] (SPX_OK, or SPX_BREAKDOWN for a zero, missing or non-finite pivot) or NULL.
 * One thread block per system, one block barrier per level.  Asynchronous. */
spx_status spx_sptrsv(const spx_csr* T, int32_t upper, int32_t nsys, const int32_t* sys_lev_off,
                      const int32_t* lev_ptr, const int32_t* lev_rows, const float* b, float* x,
                      int32_t* status, void* stream);

/* ------------------------------------------------- sparse + sparse (Section 3.1.4) */

/* Workspace bytes of spx_spadd_symbolic for m rows. */
spx_status spx_spadd_workspace_size(int32_t m, size_t* bytes);

/* Row offsets of C = alpha A + beta B, whose pattern is the union of A's and B's stored
 * patterns row by row (structural: entries that cancel stay).  A, B: device CSR patterns of
 * the same shape (sorted, unique columns).  c_indptr: device int32[m + 1] (written);
 * *nnz_c: host, nnz of C.  Synchronizes `stream` (the count returns to the host);
 * SPX_INVALID_ARG when nnz(C) does not fit int32. */
spx_status spx_spadd_symbolic(const spx_csr* A, const spx_csr* B, int32_t* c_indptr, int64_t* nnz_c,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Columns of C and the maps between the patterns: src_a[e] / src_b[e] = the entry of A / B
 * that entry e of C takes its value from (-1 if none); pos_a[e] / pos_b[e] = the position in
 * C of entry e of A / B.  c_indices, src_a, src_b: device int32[nnz_c]; pos_a: int32[nnz(A)];
 * pos_b: int32[nnz(B)].  Asynchronous. */
spx_status spx_spadd_fill(const spx_csr* A, const spx_csr* B, const int32_t* c_indptr,
                          int32_t* c_indices, int32_t* src_a, int32_t* src_b, int32_t* pos_a,
                          int32_t* pos_b, void* stream);

/* c_vals[e] = alpha a_vals[src_a[e]] + beta b_vals[src_b[e]] (absent terms skipped), each
 * value written once.  Device float32 arrays.  Asynchronous. */
spx_status spx_spadd_numeric(int64_t nnz_c, float alpha, const float* a_vals, const int32_t* src_a,
                             float beta, const float* b_vals, const int32_t* src_b, float* c_vals,
                             void* stream);

/* Gradients of C = alpha A + beta B (Table 1, Sp + Sp): ga[e] = alpha gc[pos_a[e]] on
 * mask(A), gb[e] = beta gc[pos_b[e]] on mask(B), gc given on mask(C).  ga or gb may be NULL
 * (not computed).  Asynchronous. */
spx_status spx_spadd_backward(int64_t nnz_a, int64_t nnz_b, float alpha, float beta, const float* gc,
                              const int32_t* pos_a, const int32_t* pos_b, float* ga, float* gb,
                              void* stream);

/* ------------------------------ sparse approximate inverse by descent (Section 4.6) */

/* The residual of the SPAI loss ||I - M A||_F^2 on the pattern of C = M A (formed by the
 * SpGEMM entry points): out[e] = scale * ([i == j] - C.values[e]) for every stored entry
 * e = (i, j) of C; scale = -2 gives the gradient of the loss w.r.t. C's values, to be passed
 * to spx_spgemm_backward for the gradient w.r.t. M.  diag_count (device int32, may be NULL)
 * receives the number of diagonal entries stored in C (each missing one adds 1 to the
 * loss).  C: device CSR with values; out: device float32[C.nnz].  Asynchronous. */
spx_status spx_spai_residual(const spx_csr* C, float scale, float* out, int32_t* diag_count,
                             void* stream);

/* Workspace bytes of spx_dot for vectors of n entries. */
spx_status spx_dot_workspace_size(int64_t n, size_t* bytes);

/* *out = sum_i x[i] y[i] (device float32 inputs, device double output), accumulated in
 * double-float per thread and FP64 across threads and blocks in a fixed order, so the
 * result is reproducible bit for bit.  workspace: device, spx_dot_workspace_size bytes.
 * Asynchronous; the result stays on the device. */
spx_status spx_dot(int64_t n, const float* x, const float* y, double* out, void* workspace,
                   size_t workspace_bytes, void* stream);

/* The exact line-search step of the SPAI descent: m[e] -= eta * g[e] with
 * eta = (1/2) *gg / *dada, where gg = <g, g> and dada = <g A, g A> are device doubles (from
 * spx_dot).  The loss is quadratic in M, so eta minimises it along -g.  No step is taken
 * when dada is not positive and finite.  m, g: device float32[nnz].  Asynchronous. */
spx_status spx_spai_update(int64_t nnz, float* m, const float* g, const double* gg,
                           const double* dada, void* stream);

/* spx_spmm_t for callers that cannot allocate device memory when they call it -- e.g. a
 * host framework that owns all device memory through its own pool and forbids other
 * allocations, or code that must not let an allocation synchronise the device.  The paper
 * has no counterpart: this is a deployment variant of spx_spmm_t.
 * Same operation, arguments and results as spx_spmm_t with no workspace and no G slabs,
 * except that A^T's gathered values are staged in a scratch array built into the library
 * (16 MiB of device memory per device that loads the library, held until exit), so:
 *  - AT->nnz must be <= 4,194,304 (2^22); larger sizes return SPX_INVALID_ARG with a
 *    message, before any device work;
 *  - it calls no cudaMalloc / cudaFree and allocates nothing;
 *  - the first call on a device looks the array's device address up once for that
 *    device (cudaGetSymbolAddress, with that device current), and looks it up again only
 *    when that device's context is a new one (after cudaDeviceReset, say); make that
 *    first call before any stream capture;
 *  - every call shares the one array and leaves its contents behind; each call writes
 *    all the entries it reads, so nothing needs clearing, but calls whose work overlaps
 *    on the GPU (other streams, other host threads) race on the array: serialise them. */
spx_status spx_spmm_t_noalloc(const spx_csr* AT, const int32_t* perm, const float* G,
                              int64_t ldg, int32_t k, float* gX, int64_t ldgx, float alpha,
                              float beta, const spx_rowplan* plan, void* stream);

/* ------------------------------------------- merge-path products (load balancing)
 *
 * The m row ends and the nnz entries of A merged into one sequence (entry e of row i
 * before the end of row i) and cut into segments of `items` consecutive items, one per
 * lane group: every group gets the same share of rows plus entries whatever the row
 * lengths (power-law rows, empty rows, hub rows).  Row-plan products (spx_spmm,
 * spx_sddmm) split the rows instead; both compute the same operations. */
typedef struct spx_mergeplan {
    const int32_t* seg_row;   /* device int32[n_segments + 1]: the row each segment starts in */
    int32_t n_segments;       /* ceil((m + nnz) / items), at least 1 */
    int64_t items;            /* merged items (row ends + entries) per segment */
} spx_mergeplan;

/* Number of segments of a merge plan with `items` per segment (host only). */
spx_status spx_merge_plan_segments(const spx_csr* A, int64_t items, int32_t* n_segments);

/* Fills seg_row (device int32[n_segments + 1]) for A's pattern: seg_row[s] = the number of
 * row ends among the first s * items merged items (a binary search along each cut).  Once
 * per pattern and segment size; asynchronous. */
spx_status spx_merge_plan_build(const spx_csr* A, int64_t items, int32_t* seg_row,
                                int32_t n_segments, void* stream);

/* Workspace bytes of spx_spmm_merge: one carry row id and one k-wide partial sum per
 * segment. */
spx_status spx_spmm_merge_workspace_size(const spx_csr* A, int32_t k, const spx_mergeplan* plan,
                                         size_t* bytes);

/* Y = alpha * A X + beta * Y (Section 3.1.1 SpMV, 3.1.3 SpDMM) over the merge plan's
 * segments; with perm non-NULL, entry e takes the value A->values[perm[e]] (the transpose
 * product A^T G on spx_csr_transpose's pattern, Table 1).  X: n x k, Y: m x k row-major
 * float32, 16-byte aligned, leading dimensions >= k and multiples of 4; k in {4, 8, 16,
 * 32, 64, 128}.  A row cut by segment boundaries is finished by the segment holding its
 * end; the earlier segments' partial sums go to the workspace and a second kernel adds
 * them in segment order (deterministic).  variant: 0 = 8-entry batches with 4 resident
 * blocks per SM, 1 = 8-entry batches with 5, 2 = 4-entry batches with 6 (launch shapes
 * for the autotuner; same results).  m + nnz < 2^31.  Asynchronous. */
spx_status spx_spmm_merge(const spx_csr* A, const int32_t* perm, const float* X, int64_t ldx,
                          int32_t k, float* Y, int64_t ldy, float alpha, float beta,
                          const spx_mergeplan* plan, int32_t variant, void* workspace,
                          size_t workspace_bytes, void* stream);

/* out[e] = scale * sum_c G[i,c] X[j,c] for every stored e = (i, j) (the SDDMM of Table 1:
 * the SpDMM gradient w.r.t. A) over the merge plan's segments.  G: m x k, X: n x k with
 * the same layout rules as spx_spmm_merge; variant 0 = 8 row gathers in flight per lane
 * with 4 resident blocks per SM, 1 = 4 with 5, 2 = 8 with 3 (same results).  Every output
 * written once; m + nnz < 2^31; asynchronous. */
spx_status spx_sddmm_merge(const spx_csr* A, const float* G, int64_t ldg, const float* X,
                           int64_t ldx, int32_t k, float scale, float* out,
                           const spx_mergeplan* plan, int32_t variant, void* stream);

/* Measurement instrument, not an operation of the paper: the gather bound of the products
 * that read dense rows through a column stream (spx_spmm, spx_sddmm, spx_spmm_t).  For every
 * e < nnz it reads row indices[e] of X (k float32 columns, row-major, leading dimension
 * ldx) as the SpMM kernel gathers it -- k / 4 lanes per row with 16-byte loads, indices
 * evict-first and X evict-last in L2 -- and adds it to a per-lane sum: no values, no row
 * boundaries, no output rows.  Its time is the floor for any kernel that gathers the same
 * rows in the same order.  unroll (1, 2 or 4): batches of 8 entries in flight per lane
 * group; blocks_per_sm (1..16): resident 256-thread blocks per SM (the grid).  Entries with
 * an index outside [0, n) are skipped.  out: device float32[out_len], out_len >=
 * blocks_per_sm * SMs * 256 (per-thread sums).  k in {4, 8, 16, 32, 64, 128}; X 16-byte
 * aligned, ldx % 4 == 0.  Device pointers; asynchronous. */
spx_status spx_gather_probe(const int32_t* indices, int64_t nnz, int32_t n, const float* X,
                            int64_t ldx, int32_t k, int32_t unroll, int32_t blocks_per_sm,
                            float* out, int64_t out_len, void* stream);

/* Diagonal of A (the paper's A.diagonal(), Section 4.1): for i < min(m, n),
 * diag[i] = a_ii, or 0 where row i stores no diagonal entry, and pos[i] = the index of
 * entry (i, i) in A's indices / values, or -1.  Either output may be NULL (diag needs
 * A's values).  Binary search per row (columns sorted).  Device pointers; asynchronous. */
spx_status spx_csr_diagonal(const spx_csr* A, float* diag, int32_t* pos, void* stream);

/* VJP of spx_csr_diagonal w.r.t. A's values (a gradient on A's pattern):
 * g_values[pos[i]] += g_diag[i] for i < nd with pos[i] >= 0 (positions are distinct, so
 * no two threads touch one entry).  g_values: device float32[nnz], typically zeroed. */
spx_status spx_diagonal_backward(int32_t nd, const int32_t* pos, const float* g_diag,
                                 float* g_values, void* stream);

/* dst[e] = src[perm[e]] for e < nnz -- e.g. A^T's values from A's through the
 * permutation of spx_csr_transpose.  Device pointers. */
spx_status spx_gather_values(int64_t nnz, const int32_t* perm, const float* src, float* dst,
                             void* stream);

/* ------------------------------ differentiable sparse solve (Section 4.3, Table 1) */

/* Workspace bytes of spx_cg_batched for an n-row batch (six float vectors). */
spx_status spx_cg_workspace_size(int32_t n, size_t* bytes);

/* Batched PCG: solves A_s x_s = b_s for every diagonal block s of the block-diagonal
 * SPD matrix A (row offsets sys_ptr, device int32[nsys+1]; A's column indices are global
 * and stay inside their block), from x0 = 0, until the TRUE relative residual
 * ||b_s - A_s x_s|| / ||b_s||, computed in FP64, is <= tol, or maxit iterations.
 * The iteration runs in FP32 with reliable updates into the FP64 solution whenever the
 * recurrence residual drops by the factor `delta` (0 < delta < 1, e.g. 0.1); inner
 * products accumulate in double-float and are combined in FP64.
 * order: optional device int32[nsys], the order in which systems are taken (largest
 *        first balances the load); NULL = natural order.
 * b: device float32[n]; x: device float64[n] (output).
 * pc_kind: 0 none, 1 Jacobi (pc_diag_inv = device float32[n] holding 1 / a_ii),
 *          2 M = L L^T (Section 4.3): L lower-triangular CSR with values on the
 *          diagonal blocks and LT its transpose with values (spx_csr_transpose +
 *          spx_gather_values), applied as two sparse products,
 *          3 an explicit SPD sparse M passed as L (LT unused), applied as one
 *          sparse product -- e.g. L L^T formed once with the SpGEMM calls,
 *          4 IC(0): L the factor from spx_ic0_factor, LT its transpose with values,
 *          ic0_levels = {sys_lev_off, lev_ptr, lev_rows} from spx_ic0_analyse (a host
 *          array of three device pointers); the two triangular solves run level by level
 *          on the first block of each cluster.  Ignored (may be NULL) for kinds 0-3.
 * iters, status (spx_status per system: OK, MAXITER, BREAKDOWN, NONFINITE): device
 * int32[nsys]; relres: device float64[nsys], the true relative residual of the
 * returned x.  One launch of thread-block clusters (one cluster per system at a time,
 * shape set by spx_cg_set_launch; for kinds 0, 1 and 3 each block takes 192 bytes of
 * dynamic shared memory per thread for its private vectors, see
 * spx_cg_set_vector_residency); capturable in a CUDA graph.  The call's own status reports argument / launch errors only. */
spx_status spx_cg_batched(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys,
                          const int32_t* order, const float* b, double* x, int32_t pc_kind,
                          const float* pc_diag_inv, const spx_csr* L, const spx_csr* LT,
                          const int32_t* const* ic0_levels, double tol, int32_t maxit,
                          double delta, int32_t* iters, int32_t* status, double* relres,
                          void* workspace, size_t workspace_bytes, void* stream);

/* The factored approximate inverse M = L L^T of Section 4.3 with L lower-triangular in
 * diagonal form, per system: L_{i, i + off_d} for at most 3 offsets off_d <= 0 (e.g. the
 * 0, -1, -N of tril(A) for a 5-point grid of side N).  spx_dia_analyse finds each system's
 * offsets from L's pattern (offsets: device int32[nsys * 3], ascending |off|; nd: device
 * int32[nsys], -1 for a system with more than 3 offsets or an entry above the diagonal)
 * and writes 1 to *supported_host when every system has at most 3 (synchronizes: reads nd
 * back).  Once per pattern. */
spx_status spx_dia_analyse(const spx_csr* L, const int32_t* sys_ptr, int32_t nsys,
                           int32_t* offsets, int32_t* nd, int32_t* supported_host, void* stream);

/* values_bf16 (device BF16[3 * n], n = L->m): values[d * n + i] = L_{i, i + off_d} rounded
 * to BF16 (round to nearest even), 0 where row i has no such entry.  Per value set of L;
 * asynchronous. */
spx_status spx_dia_fill(const spx_csr* L, const int32_t* sys_ptr, int32_t nsys,
                        const int32_t* offsets, const int32_t* nd, void* values_bf16, void* stream);

/* M = L L^T from L's diagonal form (the offsets, counts and BF16 values above) by its lower
 * diagonals: with s_d = -off_d, M_{i, i - o} = sum over pairs (d, e) with s_d - s_e = o of
 * L_{i, i - s_d} L_{i - o, i - o - s_e}, summed in FP32 in (d, e) order (the products of BF16
 * values are exact) and rounded to BF16.  m_offsets: device int32[nsys * 4], the distances
 * o >= 0 ascending (0, then every positive s_d - s_e: at most 4 for 3 diagonals of L; for a
 * 5-point grid of side N: 0, 1, N - 1, N); m_nd: device int32[nsys] (-1 where L's nd is -1);
 * m_values_bf16: device BF16[4 * n], m_values[q * n + i] = M_{i, i - o_q}, 0 where row i - o_q
 * lies outside the system.  n = rows of the batch.  Per value set of L; asynchronous. */
spx_status spx_dia_square(const int32_t* sys_ptr, int32_t nsys, int32_t n, const int32_t* l_offsets,
                          const int32_t* l_nd, const void* l_values_bf16, int32_t* m_offsets,
                          int32_t* m_nd, void* m_values_bf16, void* stream);

/* spx_cg_batched with a symmetric M given by its lower diagonals (spx_dia_square's output:
 * dia_offsets int32[nsys * 4] distances, dia_nd int32[nsys], dia_values BF16[4 * n]), e.g.
 * M = L L^T of Section 4.3.  Each block keeps its rows of M's diagonals (BF16) and of q = A p,
 * z, r and p in shared memory for the whole solve (192 KB per 1024-thread block: 8 rows per
 * thread, every system's rows must fit 8 per thread per block of the cluster) and applies M in
 * one pass, (M x)_i = M_0[i] x_i + sum_{d>=1} (M_d[i] x_{i - o_d} + M_d[i + o_d] x_{i + o_d}),
 * reading x (and M's rows) of the neighbouring blocks from their shared memory (the
 * cluster's distributed shared memory).  It carries z = M r by z <- z - alpha M q: q is
 * complete over the cluster after the reduction that gives alpha, so M q needs no cluster
 * barrier; at the start and after every reliable update z = M r is formed directly from the
 * recomputed r.  A system whose diagonals are unsupported, or whose halo max o_d exceeds a
 * block's rows, gets status SPX_NOT_SUPPORTED and relres -1.  Other arguments and results as
 * in spx_cg_batched (threads per block and cluster from spx_cg_set_launch). */
spx_status spx_cg_batched_dia(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys,
                              const int32_t* order, const float* b, double* x,
                              const int32_t* dia_offsets, const int32_t* dia_nd,
                              const void* dia_values_bf16, double tol, int32_t maxit,
                              double delta, int32_t* iters, int32_t* status, double* relres,
                              void* workspace, size_t workspace_bytes, void* stream);

/* Launch shape of spx_cg_batched for this process: threads per block (256, 512 or 1024),
 * blocks per cluster (1, 2, 4, 8, or 16 -- a non-portable cluster size the call opts into)
 * and the most clusters resident at once (fewer systems in flight keep their vectors in
 * L2); 0 keeps the default (512 threads, 8 blocks, as many clusters as fit).  A tuning
 * knob: results do not depend on it beyond floating-point rounding of the reductions. */
spx_status spx_cg_set_launch(int32_t threads_per_block, int32_t cluster_size, int32_t max_clusters);

/* Where spx_cg_batched keeps the vectors a block reads only on its own rows (x's FP32
 * partial, A p, z, D^-1, r when the preconditioner does not gather it, and a copy of p):
 * 1 (default) in shared memory whenever a system's rows per block are at most 8 x the
 * threads per block (preconditioner kinds 0, 1 and 3); 0 always in the global workspace.
 * p (gathered by the sparse product) always lives in the workspace.  The arithmetic and
 * its order are the same either way: results are bitwise identical. */
spx_status spx_cg_set_vector_residency(int32_t shared_memory);

/* dinv[i] = 1 / a_ii (0 where the diagonal is absent or zero); device float32[m]. */
spx_status spx_diag_inverse(const spx_csr* A, float* dinv, void* stream);

/* out[e] = (float)(scale * u[i] * v[j]) on mask(A) with FP64 u, v: the SpSolve
 * gradient w.r.t. A, -(A^{-T} g) x^T masked to A (Table 1), with scale = -1,
 * u = lambda = A^{-T} g and v = x. */
spx_status spx_masked_outer_f64(const spx_csr* A, const double* u, const double* v,
                                double scale, float* out, void* stream);

/* ----------------------- learned preconditioner (Section 4.3) and its network */

/* Workspace bytes of spx_pcg_train for an n-row batch, n_it iterations and a checkpoint
 * interval (0: keep every iterate).  With interval s < n_it: 5 (s + 1) + 6 + 2 ceil(n_it / s)
 * float vectors (one segment of iterates, the adjoint vectors, r and p at every segment
 * start); otherwise 5 (n_it + 1) + 6. */
spx_status spx_pcg_train_workspace_size(int32_t n, int32_t n_it, int32_t ckpt_interval,
                                        size_t* bytes);

/* Loss of n_it unrolled PCG iterations with M = L L^T from x0 = 0 (Section 4.3):
 *   loss_s = sum_{i=1..n_it} weights[i-1] ||r_i|| / ||b_s||   for every system s,
 * and grad_L = d(mean_s loss_s) / d L.values on L's pattern (reverse mode through the
 * iterations; A itself is not differentiated and is assumed symmetric).
 * A, sys_ptr: the block-diagonal batch as in spx_cg_batched; L: lower-triangular CSR
 * with values on the diagonal blocks; LT: its transpose with values.  weights: device
 * float32[n_it] (e.g. gamma^(n_it-i) normalised); b: device float32[n].
 * ckpt_interval: 0 (or >= n_it) keeps every forward iterate for the reverse pass; s in
 * 1..n_it-1 keeps r and p every s iterations and recomputes the iterates in between
 * during the reverse pass (one more forward pass of work, workspace O(s + n_it / s)
 * vectors instead of O(n_it)); the results are bitwise the same either way.
 * loss: device float32[nsys]; grad_L: device float32[nnz(L)] (overwritten).
 * 1 <= n_it <= 64.  One thread block per system; deterministic. */
spx_status spx_pcg_train(const spx_csr* A, const int32_t* sys_ptr, int32_t nsys,
                         const spx_csr* L, const spx_csr* LT, const float* b, int32_t n_it,
                         int32_t ckpt_interval, const float* weights, float* loss,
                         float* grad_L, void* workspace, size_t workspace_bytes, void* stream);

/* Scale-free inputs of the network: d[i] = a_ii^(-1/2), e_vals[k] = d_i a_ij d_j on A's
 * pattern, feats[i, 0..3] = [1, sum_{j != i} e_ij, min_{j != i} e_ij, max_{j != i} e_ij]
 * (the last three 0 for a row without off-diagonal entries).  Device float32. */
spx_status spx_mpnn_features(const spx_csr* A, float* d, float* e_vals, float* feats,
                             void* stream);

/* Dense layer Y = [X1 X2] W + b on n rows (X1: n x K1, X2: n x K2 or NULL with K2 = 0,
 * W: (K1+K2) x N row-major BF16, b: float32[N] or NULL; K1 + K2 <= 128, N <= 128).
 * mode 0: Y = pre-activation; 1: Y = relu(pre); 2: U = pre and Y = Hin + relu(pre)
 * (residual layer; Hin, Y, U: n x N).  FP32 accumulation.  Device pointers. */
spx_status spx_dense_forward(int64_t n, const float* X1, int32_t K1, const float* X2, int32_t K2,
                             const void* W_bf16, const float* bias, int32_t N, int32_t mode,
                             const float* Hin, float* Y, float* U, void* stream);

/* spx_dense_forward on the tensor cores (tcgen05, accumulator in tensor memory): the
 * activations are rounded to BF16 (round to nearest even) while they are staged, so the
 * result equals spx_dense_forward applied to BF16-rounded X1, X2 up to the order of the
 * FP32 accumulation.  N must be a multiple of 16 (16..128), K1 + K2 <= 128.  Besides modes
 * 0-2, two epilogues for inference: mode 3 = the residual layer without U (Y = Hin +
 * relu(pre), the pre-activation kept nowhere), mode 4 = the product's column halves to two
 * outputs, Y = pre[:, :N/2] and U = pre[:, N/2:] (each n x N/2), e.g. both heads of the
 * network from one pass over the activations.  Shapes with K1 (and K2) multiples of 32,
 * N a multiple of 32 (mode 4: N / 2) run on the pipelined kernel (one persistent CTA per
 * SM: TMA tensor loads into a ring of stages, converter warps, one MMA-issuing thread, two
 * accumulators in tensor memory, epilogue warps storing through TMA); other shapes on
 * persistent CTAs that stage, multiply and store in turn.  Both give bitwise the same
 * result.  Device pointers; asynchronous on `stream`. */
spx_status spx_dense_forward_tc(int64_t n, const float* X1, int32_t K1, const float* X2,
                                int32_t K2, const void* W_bf16, const float* bias, int32_t N,
                                int32_t mode, const float* Hin, float* Y, float* U, void* stream);

/* spx_dense_backward_data on the tensor cores (tcgen05, accumulator in tensor memory): G is
 * rounded to BF16 while staged, so the result equals spx_dense_backward_data applied to a
 * BF16-rounded G up to the order of the FP32 accumulation.  N, K1, K2 multiples of 4,
 * N <= 128, K1 + K2 <= 128; G, dX1, dX2 16-byte aligned.  With N, K1 (and K2) multiples
 * of 32 it runs on the pipelined kernel of spx_dense_forward_tc, accumulating by TMA
 * reduce-add stores (old + new, the same single rounding as a load-add-store).
 * Asynchronous. */
spx_status spx_dense_backward_data_tc(int64_t n, const float* G, int32_t N, const void* W_bf16,
                                      int32_t K1, int32_t K2, float* dX1, float* dX2,
                                      int32_t accumulate, void* stream);

/* Enables (1, the default) or disables (0) the pipelined kernel of spx_dense_forward_tc and
 * spx_dense_backward_data_tc for the calls that follow (process-wide), e.g. to time or
 * compare the two kernels; results are bitwise equal either way.  Never fails. */
spx_status spx_tc_set_pipeline(int32_t enabled);

/* Data gradient [dX1 dX2] = G W^T (or += with accumulate != 0); dX2 may be NULL. */
spx_status spx_dense_backward_data(int64_t n, const float* G, int32_t N, const void* W_bf16,
                                   int32_t K1, int32_t K2, float* dX1, float* dX2,
                                   int32_t accumulate, void* stream);

/* Workspace bytes of spx_dense_backward_weight_tc: one (K + 1) x N float32 partial per CTA
 * (at most two CTAs per SM of the current device).  K = K1 + K2 <= 128, K % 4 == 0;
 * N in {16, 32, 64, 128}. */
spx_status spx_dense_backward_weight_tc_workspace_size(int64_t n, int32_t K, int32_t N,
                                                       size_t* bytes);

/* spx_dense_backward_weight on the tensor cores (tcgen05): dW = [X1 X2]^T G with X and G
 * rounded to BF16 while staged and the products summed in FP32 in tensor memory; db = the
 * column sums of G in FP32 (or NULL).  Overwrites dW (K x N row-major) and db.  K1 >= 4,
 * K1, K2 multiples of 4, K1 + K2 <= 128, N in {16, 32, 64, 128}; X1, X2, G, workspace
 * 16-byte aligned.  Deterministic: per-CTA partials (fixed row tiles per CTA) added in CTA
 * order.  A tensor-core completion wait that exceeds 2 s records a device error
 * (spx_check_device).  Asynchronous. */
spx_status spx_dense_backward_weight_tc(int64_t n, const float* X1, int32_t K1, const float* X2,
                                        int32_t K2, const float* G, int32_t N, float* dW,
                                        float* db, void* workspace, size_t workspace_bytes,
                                        void* stream);

/* Workspace bytes of spx_dense_backward_weight ((K + 1) * N <= 8448). */
spx_status spx_dense_backward_weight_workspace_size(int64_t n, int32_t K, int32_t N,
                                                    size_t* bytes);

/* Weight gradient dW = [X1 X2]^T G (K x N, float32) and db = column sums of G (or NULL);
 * per-block partial sums added in a fixed order (deterministic). */
spx_status spx_dense_backward_weight(int64_t n, const float* X1, int32_t K1, const float* X2,
                                     int32_t K2, const float* G, int32_t N, float* dW,
                                     float* db, void* workspace, size_t workspace_bytes,
                                     void* stream);

/* gu[t] = gh[t] if u[t] > 0 else 0 (the derivative of relu at the pre-activation u). */
spx_status spx_relu_backward(int64_t count, const float* gh, const float* u, float* gu,
                             void* stream);

/* Workspace bytes of spx_tril_pattern. */
spx_status spx_tril_workspace_size(int32_t n, size_t* bytes);

/* The pattern of tril(A) (entries with j <= i): l_indptr (device int32[m+1]) and its
 * nnz to *nnz_host (synchronizes); when l_indices and l_src are non-NULL (device
 * int32[nnz]) also the columns and, for each entry, its position in A. */
spx_status spx_tril_pattern(const spx_csr* A, int32_t* l_indptr, int32_t* l_indices,
                            int32_t* l_src, int64_t* nnz_host, void* workspace,
                            size_t workspace_bytes, void* stream);

/* Edge head on tril(A) (hidden width 64): for each stored (i, j) of Lpat,
 *   o = relu(P_i + Q_j + e_ij u + c) . v + (bd if i == j else bo),
 *   L = d_i * (softplus(o) if i == j else o).
 * e_low: e values on Lpat; P, Q: n x 64; u, c, v: float32[64]; bd, bo: float32[1]. */
spx_status spx_edge_forward(const spx_csr* Lpat, const float* e_low, const float* d,
                            const float* P, const float* Q, const float* u, const float* c,
                            const float* v, const float* bd, const float* bo, float* L_values,
                            void* stream);

/* Workspace bytes of spx_edge_backward. */
spx_status spx_edge_backward_workspace_size(int32_t n, size_t* bytes);

/* Reverse of spx_edge_forward for the upstream gradient gL (on Lpat): gP, gQ (n x 64,
 * overwritten) and gparams = [gv (64), gc (64), gu (64), gbd, gbo] (float32[194]).
 * lt_*: the transpose of Lpat (spx_csr_transpose).  Deterministic. */
spx_status spx_edge_backward(const spx_csr* Lpat, const int32_t* lt_indptr,
                             const int32_t* lt_indices, const int32_t* lt_perm,
                             const float* e_low, const float* d, const float* P, const float* Q,
                             const float* u, const float* c, const float* v, const float* bd,
                             const float* bo, const float* gL, float* gP, float* gQ,
                             float* gparams, void* workspace, size_t workspace_bytes,
                             void* stream);

/* One step of Adam (Kingma and Ba, ICLR 2015, Algorithm 1), the optimiser the paper trains
 * its examples with (Section 4.1's Jacobi weights, Section 4.5's GCN), on `count` float32
 * parameters.  For every t in [0, count), with c1 = 1 - beta1^step and c2 = 1 - beta2^step
 * (formed in double on the host, then rounded to float):
 *   m[t] = beta1 m[t] + (1 - beta1) g[t],   v[t] = beta2 v[t] + (1 - beta2) g[t]^2,
 *   params[t] -= lr (m[t] / c1) / (sqrt(v[t] / c2) + eps)
 * in float32 arithmetic.  params, m, v (device float32[count], updated in place; m and v
 * zero before step 1) and grads (device float32[count]) belong to the caller; step >= 1 is
 * the step number.  When params_bf16 (device bf16[count]) is non-NULL the updated
 * parameters are also written there, rounded to nearest even.  SPX_INVALID_ARG for
 * count < 0, step < 1 or a NULL array with count > 0.  Asynchronous on `stream`. */
spx_status spx_adam_step(int64_t count, float* params, const float* grads, float* m, float* v,
                         int32_t step, float lr, float beta1, float beta2, float eps,
                         void* params_bf16, void* stream);

/* dst[t] = src[t] rounded to BF16 (nearest, ties to even); device arrays of count. */
spx_status spx_to_bf16(int64_t count, const float* src, void* dst, void* stream);

/* ---------------------------------------- IC(0) baseline (Section 3.1.5 solves) */

/* Workspace bytes of spx_ic0_analyse. */
spx_status spx_ic0_workspace_size(int32_t n, int32_t nsys, size_t* bytes);

/* Level schedule of the lower-triangular pattern Lpat (e.g. tril(A) from
 * spx_tril_pattern) per system of a block-diagonal batch: level(i) = 0 without
 * off-diagonal entries, else 1 + the largest level among its columns j < i.
 * Outputs (device int32): sys_lev_off[nsys+1] (offsets into lev_ptr), lev_ptr[n + nsys]
 * (per system: start of each level in lev_rows, then the end), lev_rows[n] (rows
 * grouped by level, increasing within a level).  One thread per system. */
spx_status spx_ic0_analyse(const spx_csr* Lpat, const int32_t* sys_ptr, int32_t nsys,
                           int32_t* sys_lev_off, int32_t* lev_ptr, int32_t* lev_rows,
                           void* workspace, size_t workspace_bytes, void* stream);

/* Zero-fill incomplete Cholesky on tril(A)'s pattern (Saad Sec. 10.3): L L^T agrees with
 * A on the pattern.  l_src[e]: the position in A of tril entry e (spx_tril_pattern);
 * a_values: A's values; l_values: output float32[nnz(Lpat)]; status: per system SPX_OK or
 * SPX_BREAKDOWN (a non-positive pivot).  One thread block per system, level by level. */
spx_status spx_ic0_factor(const spx_csr* Lpat, const int32_t* l_src, const float* a_values,
                          int32_t nsys, const int32_t* sys_lev_off, const int32_t* lev_ptr,
                          const int32_t* lev_rows, float* l_values, int32_t* status,
                          void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPX_H */
