/*
 * FP64 CPU oracle for the sparse forward and reverse-mode kernels.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this file:
 * it exists so that tests, the smoke check and the CPU baseline of the benchmark can
 * compare the CUDA kernels against plain, serial, obviously-correct loops.  It shares
 * no code, header or table with the CUDA sources.
 *
 * Every routine below writes out the definition of the operation it follows, in
 * double precision, one output at a time, in the order the definition states:
 *
 *   CSR layout (Section 3): indptr[m+1], indices[nnz] (sorted, unique per row),
 *   values[nnz].  mask(A) is read structurally: every stored entry is in the mask,
 *   including explicit zeros (reading of the sparsity-mask definition, Section 3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int32_t i32;
typedef int64_t i64;

/* Section 3.1.1 (SpMV) and 3.1.3 (SpDMM): Y[i,:] = sum over the stored entries e of
 * row i of A_e * X[col_e,:].  X is n x k row-major, Y is m x k row-major. */
void orc_spmm(i64 m, const i32 *indptr, const i32 *indices, const double *vals,
              const double *X, i64 k, double *Y)
{
    for (i64 i = 0; i < m; ++i) {
        for (i64 c = 0; c < k; ++c) {
            double s = 0.0;
            for (i64 e = indptr[i]; e < indptr[i + 1]; ++e)
                s += vals[e] * X[(i64)indices[e] * k + c];
            Y[i * k + c] = s;
        }
    }
}

/* Table 1, SpMV / SpDMM gradient w.r.t. A: (V X^T) masked to A's pattern.
 * out[e] for the entry e = (i, j) is sum_c G[i,c] * X[j,c]. */
void orc_sddmm(i64 m, const i32 *indptr, const i32 *indices, const double *G,
               const double *X, i64 k, double *out)
{
    for (i64 i = 0; i < m; ++i) {
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e) {
            i64 j = indices[e];
            double s = 0.0;
            for (i64 c = 0; c < k; ++c)
                s += G[i * k + c] * X[j * k + c];
            out[e] = s;
        }
    }
}

/* Sparse transpose (Section 3.1.3 takes the transpose of A to form A^T V).
 * Counting sort over columns; scanning rows in increasing order keeps the row
 * indices of every column sorted.  perm[e'] is the position in A of the entry that
 * lands at position e' of A^T, so A^T.values[e'] = A.values[perm[e']]. */
void orc_transpose(i64 m, i64 n, const i32 *indptr, const i32 *indices,
                   i32 *t_indptr, i32 *t_indices, i32 *perm)
{
    i64 nnz = indptr[m];
    i64 *count = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    for (i64 e = 0; e < nnz; ++e)
        count[indices[e] + 1] += 1;
    for (i64 j = 0; j < n; ++j)
        count[j + 1] += count[j];
    for (i64 j = 0; j <= n; ++j)
        t_indptr[j] = (i32)count[j];
    for (i64 i = 0; i < m; ++i) {
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e) {
            i64 j = indices[e];
            i64 pos = count[j]++;
            t_indices[pos] = (i32)i;
            perm[pos] = (i32)e;
        }
    }
    free(count);
}

/* Table 1, SpMV / SpDMM gradient w.r.t. the dense operand: gX = A^T G, written as
 * the scatter gX[col_e,:] += A_e * G[i,:] over the stored entries in row order. */
void orc_spmm_t(i64 m, i64 n, const i32 *indptr, const i32 *indices, const double *vals,
                const double *G, i64 k, double *gX)
{
    memset(gX, 0, sizeof(double) * (size_t)(n * k));
    for (i64 i = 0; i < m; ++i)
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e) {
            i64 j = indices[e];
            for (i64 c = 0; c < k; ++c)
                gX[j * k + c] += vals[e] * G[i * k + c];
        }
}

/* Section 3.1.2 (SpSpMM) forward, symbolic part.  The pattern of C = A B is every
 * (i, j) reached by a structural product A_ik B_kj (no dropping of numerical zeros).
 * For each row i a dense marker over the p columns of B records the distinct j.
 * row_nnz[i] = |pattern of C_i|, row_products[i] = number of products A_ik B_kj.
 * Returns nnz(C). */
i64 orc_spgemm_count(i64 m, i64 p, const i32 *a_indptr, const i32 *a_indices,
                     const i32 *b_indptr, const i32 *b_indices, i64 *row_nnz,
                     i64 *row_products)
{
    i64 *mark = (i64 *)malloc(sizeof(i64) * (size_t)(p > 0 ? p : 1));
    for (i64 j = 0; j < p; ++j)
        mark[j] = -1;
    i64 total = 0;
    for (i64 i = 0; i < m; ++i) {
        i64 cnt = 0, prods = 0;
        for (i64 e = a_indptr[i]; e < a_indptr[i + 1]; ++e) {
            i64 kk = a_indices[e];
            for (i64 f = b_indptr[kk]; f < b_indptr[kk + 1]; ++f) {
                i64 j = b_indices[f];
                prods += 1;
                if (mark[j] != i) {
                    mark[j] = i;
                    cnt += 1;
                }
            }
        }
        row_nnz[i] = cnt;
        row_products[i] = prods;
        total += cnt;
    }
    free(mark);
    return total;
}

static int cmp_i32(const void *a, const void *b)
{
    i32 x = *(const i32 *)a, y = *(const i32 *)b;
    return (x > y) - (x < y);
}

/* Section 3.1.2 (SpSpMM) forward, pattern and values.  c_indptr must already hold
 * the prefix sums of row_nnz.  Per row: gather the distinct columns with a dense
 * marker, sort them, then C_ij = sum over k (in row order of A) of A_ik B_kj. */
void orc_spgemm_fill(i64 m, i64 p, const i32 *a_indptr, const i32 *a_indices,
                     const double *a_vals, const i32 *b_indptr, const i32 *b_indices,
                     const double *b_vals, const i32 *c_indptr, i32 *c_indices,
                     double *c_vals)
{
    i64 *mark = (i64 *)malloc(sizeof(i64) * (size_t)(p > 0 ? p : 1));
    double *acc = (double *)calloc((size_t)(p > 0 ? p : 1), sizeof(double));
    for (i64 j = 0; j < p; ++j)
        mark[j] = -1;
    for (i64 i = 0; i < m; ++i) {
        i64 pos = c_indptr[i];
        for (i64 e = a_indptr[i]; e < a_indptr[i + 1]; ++e) {
            i64 kk = a_indices[e];
            for (i64 f = b_indptr[kk]; f < b_indptr[kk + 1]; ++f) {
                i64 j = b_indices[f];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    c_indices[pos++] = (i32)j;
                }
                acc[j] += a_vals[e] * b_vals[f];
            }
        }
        i64 beg = c_indptr[i];
        qsort(c_indices + beg, (size_t)(pos - beg), sizeof(i32), cmp_i32);
        for (i64 q = beg; q < pos; ++q)
            c_vals[q] = acc[c_indices[q]];
    }
    free(mark);
    free(acc);
}

/* Position of column j in the sorted row [beg, end) of a CSR pattern, or -1. */
static i64 find_col(const i32 *indices, i64 beg, i64 end, i64 j)
{
    i64 lo = beg, hi = end;
    while (lo < hi) {
        i64 mid = lo + (hi - lo) / 2;
        if (indices[mid] < j)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < end && indices[lo] == j) ? lo : -1;
}

/* Table 1, SpSpMM gradient w.r.t. A: (V B^T) masked to A's pattern.  V lives on
 * C's pattern.  gA[(i,k)] = sum over the entries (k, j) of row k of B of
 * V[i,j] * B[k,j], where V[i,j] is zero when (i, j) is not stored in C. */
void orc_spgemm_grad_a(i64 m, const i32 *a_indptr, const i32 *a_indices,
                       const i32 *b_indptr, const i32 *b_indices, const double *b_vals,
                       const i32 *c_indptr, const i32 *c_indices, const double *gc_vals,
                       double *ga)
{
    for (i64 i = 0; i < m; ++i) {
        for (i64 e = a_indptr[i]; e < a_indptr[i + 1]; ++e) {
            i64 kk = a_indices[e];
            double s = 0.0;
            for (i64 f = b_indptr[kk]; f < b_indptr[kk + 1]; ++f) {
                i64 q = find_col(c_indices, c_indptr[i], c_indptr[i + 1], b_indices[f]);
                if (q >= 0)
                    s += gc_vals[q] * b_vals[f];
            }
            ga[e] = s;
        }
    }
}

/* Table 1, SpSpMM gradient w.r.t. B: (A^T V) masked to B's pattern.
 * gB[(k,j)] = sum over rows i with A_ik stored of A_ik * V[i,j]; written as the
 * scatter over every stored A_ik and every stored B_kj. */
void orc_spgemm_grad_b(i64 m, i64 nnz_b, const i32 *a_indptr, const i32 *a_indices,
                       const double *a_vals, const i32 *b_indptr, const i32 *b_indices,
                       const i32 *c_indptr, const i32 *c_indices, const double *gc_vals,
                       double *gb)
{
    memset(gb, 0, sizeof(double) * (size_t)nnz_b);
    for (i64 i = 0; i < m; ++i) {
        for (i64 e = a_indptr[i]; e < a_indptr[i + 1]; ++e) {
            i64 kk = a_indices[e];
            for (i64 f = b_indptr[kk]; f < b_indptr[kk + 1]; ++f) {
                i64 q = find_col(c_indices, c_indptr[i], c_indptr[i + 1], b_indices[f]);
                if (q >= 0)
                    gb[f] += a_vals[e] * gc_vals[q];
            }
        }
    }
}

/* ---------------------------------------------------------------------------------
 * Preconditioned conjugate gradient (Section 4.3; the textbook PCG of Saad,
 * "Iterative Methods for Sparse Linear Systems", Algorithm 9.1), all in FP64.
 * ------------------------------------------------------------------------------- */

enum { ORC_PC_NONE = 0, ORC_PC_JACOBI = 1, ORC_PC_LLT = 2, ORC_PC_IC0 = 3 };

static void spmv(i64 n, const i32 *indptr, const i32 *indices, const double *vals,
                 const double *x, double *y)
{
    for (i64 i = 0; i < n; ++i) {
        double s = 0.0;
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e)
            s += vals[e] * x[indices[e]];
        y[i] = s;
    }
}

/* y = L^T x for a CSR L, as a scatter over the stored entries. */
static void spmv_t(i64 n, const i32 *indptr, const i32 *indices, const double *vals,
                   const double *x, double *y)
{
    memset(y, 0, sizeof(double) * (size_t)n);
    for (i64 i = 0; i < n; ++i)
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e)
            y[indices[e]] += vals[e] * x[i];
}

static double dot(i64 n, const double *a, const double *b)
{
    double s = 0.0;
    for (i64 i = 0; i < n; ++i)
        s += a[i] * b[i];
    return s;
}

/* Forward substitution L y = r for lower-triangular CSR L (diagonal stored last in
 * each row because columns are sorted) -- Section 3.1.5. */
void orc_trsv_lower(i64 n, const i32 *indptr, const i32 *indices, const double *vals,
                    const double *r, double *y)
{
    for (i64 i = 0; i < n; ++i) {
        double s = r[i], d = 0.0;
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e) {
            i64 j = indices[e];
            if (j < i)
                s -= vals[e] * y[j];
            else if (j == i)
                d = vals[e];
        }
        y[i] = s / d;
    }
}

/* Back substitution L^T z = y for the same lower-triangular CSR L, column-oriented:
 * once z_i is known its contribution is removed from every earlier row. */
void orc_trsv_lower_t(i64 n, const i32 *indptr, const i32 *indices, const double *vals,
                      const double *y, double *z)
{
    for (i64 i = 0; i < n; ++i)
        z[i] = y[i];
    for (i64 i = n - 1; i >= 0; --i) {
        double d = 0.0;
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e)
            if (indices[e] == i)
                d = vals[e];
        z[i] /= d;
        for (i64 e = indptr[i]; e < indptr[i + 1]; ++e) {
            i64 j = indices[e];
            if (j < i)
                z[j] -= vals[e] * z[i];
        }
    }
}

/* Zero-fill incomplete Cholesky IC(0) (Saad Section 10.3): L has the pattern of
 * tril(A) and L L^T agrees with A on that pattern.  Row i, in column order:
 *   L_ik = (a_ik - sum_{j<k} L_ij L_kj) / L_kk   for k < i,
 *   L_ii = sqrt(a_ii - sum_{j<i} L_ij^2),
 * where the sums run over columns j stored in both rows.  l_indptr/l_indices give
 * the pattern of tril(A); l_vals is the output.  Returns 0, or 1 when a pivot is
 * not positive. */
int orc_ic0(i64 n, const i32 *a_indptr, const i32 *a_indices, const double *a_vals,
            const i32 *l_indptr, const i32 *l_indices, double *l_vals)
{
    for (i64 i = 0; i < n; ++i) {
        for (i64 e = l_indptr[i]; e < l_indptr[i + 1]; ++e) {
            i64 k = l_indices[e];
            i64 ae = find_col(a_indices, a_indptr[i], a_indptr[i + 1], k);
            double s = a_vals[ae];
            /* sum over j < k stored in both row i and row k of L */
            for (i64 f = l_indptr[i]; f < e; ++f) {
                i64 j = l_indices[f];
                i64 g = find_col(l_indices, l_indptr[k], l_indptr[k + 1], j);
                if (g >= 0)
                    s -= l_vals[f] * l_vals[g];
            }
            if (k < i) {
                i64 dk = l_indptr[k + 1] - 1; /* diagonal is last in row k */
                l_vals[e] = s / l_vals[dk];
            } else {
                if (!(s > 0.0))
                    return 1;
                l_vals[e] = sqrt(s);
            }
        }
    }
    return 0;
}

/* z = M r for the preconditioner kinds of the batched solver. */
static void apply_pc(int kind, i64 n, const double *diag, const i32 *l_indptr,
                     const i32 *l_indices, const double *l_vals, const double *r,
                     double *z, double *tmp)
{
    switch (kind) {
    case ORC_PC_JACOBI:
        for (i64 i = 0; i < n; ++i)
            z[i] = r[i] / diag[i];
        break;
    case ORC_PC_LLT: /* M = L L^T, an approximate inverse (Section 4.3) */
        spmv_t(n, l_indptr, l_indices, l_vals, r, tmp);
        spmv(n, l_indptr, l_indices, l_vals, tmp, z);
        break;
    case ORC_PC_IC0: /* M = (L L^T)^{-1} with the IC(0) factor */
        orc_trsv_lower(n, l_indptr, l_indices, l_vals, r, tmp);
        orc_trsv_lower_t(n, l_indptr, l_indices, l_vals, tmp, z);
        break;
    default:
        for (i64 i = 0; i < n; ++i)
            z[i] = r[i];
    }
}

/* PCG from x0 = 0 until the TRUE relative residual ||b - A x|| / ||b|| <= tol (the
 * recurrence residual only triggers the check).  Returns 0 converged, 1 max
 * iterations, 2 breakdown (p^T A p <= 0 or r^T z <= 0), 3 non-finite.
 * iters_out receives the iteration count; hist (may be NULL, size maxit+1) the
 * recurrence residual norms ||r_i|| / ||b||. */
int orc_pcg(i64 n, const i32 *indptr, const i32 *indices, const double *vals,
            const double *b, double *x, int pc_kind, const double *diag,
            const i32 *l_indptr, const i32 *l_indices, const double *l_vals, double tol,
            i64 maxit, i64 *iters_out, double *hist)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    double *t = (double *)malloc(sizeof(double) * (size_t)n);
    int status = 1;
    i64 it = 0;
    for (i64 i = 0; i < n; ++i) {
        x[i] = 0.0;
        r[i] = b[i];
    }
    double bnorm = sqrt(dot(n, b, b));
    if (bnorm == 0.0) {
        *iters_out = 0;
        if (hist)
            hist[0] = 0.0;
        free(r); free(z); free(p); free(q); free(t);
        return 0;
    }
    if (hist)
        hist[0] = 1.0;
    apply_pc(pc_kind, n, diag, l_indptr, l_indices, l_vals, r, z, t);
    for (i64 i = 0; i < n; ++i)
        p[i] = z[i];
    double rz = dot(n, r, z);
    if (!isfinite(rz)) { status = 3; goto done; }
    if (!(rz > 0.0)) { status = 2; goto done; }
    while (it < maxit) {
        spmv(n, indptr, indices, vals, p, q);
        double pq = dot(n, p, q);
        if (!isfinite(pq)) { status = 3; break; }
        if (!(pq > 0.0)) { status = 2; break; }
        double alpha = rz / pq;
        for (i64 i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        ++it;
        double rnorm = sqrt(dot(n, r, r));
        if (hist)
            hist[it] = rnorm / bnorm;
        if (!isfinite(rnorm)) { status = 3; break; }
        if (rnorm <= tol * bnorm) {
            spmv(n, indptr, indices, vals, x, t);
            double s = 0.0;
            for (i64 i = 0; i < n; ++i)
                s += (b[i] - t[i]) * (b[i] - t[i]);
            if (sqrt(s) <= tol * bnorm) { status = 0; break; }
        }
        apply_pc(pc_kind, n, diag, l_indptr, l_indices, l_vals, r, z, t);
        double rz_new = dot(n, r, z);
        if (!isfinite(rz_new)) { status = 3; break; }
        if (!(rz_new > 0.0)) { status = 2; break; }
        double beta = rz_new / rz;
        rz = rz_new;
        for (i64 i = 0; i < n; ++i)
            p[i] = z[i] + beta * p[i];
    }
done:
    *iters_out = it;
    free(r); free(z); free(p); free(q); free(t);
    return status;
}

/* ---------------------------------------------------------------------------------------
 * Row-parallel variants, for timing the oracle on every host core (the CPU baseline).
 * Each thread takes a contiguous block of output rows holding about the same number of
 * stored entries and runs the serial loops above on it, so every output is the same
 * sum in the same order as in the serial routine: the results are equal bit for bit.
 * A^T G runs as rows of the transpose (orc_transpose's pattern and permutation):
 * gX[j,:] = sum over the entries of column j of A, in increasing row order, of
 * A_e G[i,:] -- the terms and order of orc_spmm_t's scatter, started from zero. */
#include <pthread.h>

typedef struct {
    int op;                         /* 0 spmm, 1 sddmm, 2 spmm on the transpose */
    i64 r0, r1;
    const i32 *indptr, *indices, *perm;
    const double *vals, *A, *B;     /* spmm: X; sddmm: G, X; transpose: G */
    i64 k;
    double *out;
} orc_job;

static void *orc_run_job(void *arg)
{
    orc_job *j = (orc_job *)arg;
    const i64 k = j->k;
    for (i64 i = j->r0; i < j->r1; ++i) {
        if (j->op == 0) {
            for (i64 c = 0; c < k; ++c) {
                double s = 0.0;
                for (i64 e = j->indptr[i]; e < j->indptr[i + 1]; ++e)
                    s += j->vals[e] * j->A[(i64)j->indices[e] * k + c];
                j->out[i * k + c] = s;
            }
        } else if (j->op == 1) {
            for (i64 e = j->indptr[i]; e < j->indptr[i + 1]; ++e) {
                i64 col = j->indices[e];
                double s = 0.0;
                for (i64 c = 0; c < k; ++c)
                    s += j->A[i * k + c] * j->B[col * k + c];
                j->out[e] = s;
            }
        } else {
            for (i64 c = 0; c < k; ++c) {
                double s = 0.0;
                for (i64 e = j->indptr[i]; e < j->indptr[i + 1]; ++e)
                    s += j->vals[j->perm[e]] * j->A[(i64)j->indices[e] * k + c];
                j->out[i * k + c] = s;
            }
        }
    }
    return NULL;
}

/* Splits rows [0, m) into `threads` blocks of about nnz / threads entries each and runs
 * them in parallel; returns the number of threads that ran. */
static int orc_parallel(orc_job base, i64 m, int threads)
{
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    orc_job jobs[256];
    pthread_t tid[256];
    const i64 nnz = base.indptr[m];
    i64 r = 0;
    int used = 0;
    for (int t = 0; t < threads && r < m; ++t) {
        i64 target = (t == threads - 1) ? nnz : (nnz * (t + 1)) / threads;
        i64 r1 = r;
        while (r1 < m && (base.indptr[r1 + 1] <= target || r1 == r))
            ++r1;
        if (t == threads - 1)
            r1 = m;
        jobs[used] = base;
        jobs[used].r0 = r;
        jobs[used].r1 = r1;
        r = r1;
        ++used;
    }
    int started = 0;
    for (int t = 0; t < used; ++t)
        if (pthread_create(&tid[t], NULL, orc_run_job, &jobs[t]) == 0)
            ++started;
        else
            orc_run_job(&jobs[t]);           /* no thread available: run it here */
    for (int t = 0, s = 0; t < used && s < started; ++t, ++s)
        pthread_join(tid[t], NULL);
    return used;
}

int orc_spmm_mt(i64 m, const i32 *indptr, const i32 *indices, const double *vals,
                const double *X, i64 k, double *Y, int threads)
{
    orc_job b = {0, 0, 0, indptr, indices, NULL, vals, X, NULL, k, Y};
    return orc_parallel(b, m, threads);
}

int orc_sddmm_mt(i64 m, const i32 *indptr, const i32 *indices, const double *G,
                 const double *X, i64 k, double *out, int threads)
{
    orc_job b = {1, 0, 0, indptr, indices, NULL, NULL, G, X, k, out};
    return orc_parallel(b, m, threads);
}

int orc_spmm_t_mt(i64 n, const i32 *t_indptr, const i32 *t_indices, const i32 *perm,
                  const double *vals, const double *G, i64 k, double *gX, int threads)
{
    orc_job b = {2, 0, 0, t_indptr, t_indices, perm, vals, G, NULL, k, gX};
    return orc_parallel(b, n, threads);
}
