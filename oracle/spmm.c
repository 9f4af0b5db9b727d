/*
 * CPU FP64 oracle: symmetric SpMM from one stored triangle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code with the CUDA path.
 *
 * The stored matrix is the lower triangle L of a symmetric H, diagonal
 * included, in CSR with sorted columns (Section 3.1: only half of H is
 * stored).  H = L + L^T - diag(L), so for every stored (i, j, h) with j <= i:
 *     y_i += h * x_j          (the triangle, Algorithm 2)
 *     y_j += h * x_i, j < i   (its transpose, Section 3.3: the same loop with
 *                              the roles of row and column swapped)
 * X and Y are n x k row-major (Section 3.3: the k entries of one row are
 * contiguous).  Values may be stored as float64 or float32; arithmetic is
 * float64 either way.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline double vload(const void *val, int64_t e, int val_fp32) {
    return val_fp32 ? (double)((const float *)val)[e] : ((const double *)val)[e];
}

/*
 * Form (i): Algorithm 2 over the triangle, followed by a separate transposed
 * loop (Section 3.2 keeps the SpMM and the transpose SpMM as two loops).  The
 * row loop is split over threads by rows; the transposed loop is split over
 * threads by the output rows each thread owns, so neither needs atomics.
 */
void oracle_spmm_tri(int64_t n, const int64_t *row_ptr, const int32_t *col,
                     const void *val, int val_fp32, const double *X, int32_t k,
                     double *Y) {
    memset(Y, 0, sizeof(double) * (size_t)n * (size_t)k);
    /* Triangle: Y = L X */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        double *yi = Y + (size_t)i * k;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            const double h = vload(val, e, val_fp32);
            const double *xj = X + (size_t)col[e] * k;
            for (int32_t q = 0; q < k; q++) yi[q] += h * xj[q];
        }
    }
    /* Transpose without the diagonal: Y += (L - D)^T X.  Thread t owns the
     * output rows [a, b) and visits every stored row i > a, using the sorted
     * columns to find the entries of row i that land in [a, b). */
#pragma omp parallel
    {
        int nt = 1, t = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        t = omp_get_thread_num();
#endif
        int64_t a = n * t / nt, b = n * (t + 1) / nt;
        for (int64_t i = a + 1; i < n; i++) {
            int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
            while (lo < hi) {                       /* first entry with col >= a */
                int64_t mid = lo + (hi - lo) / 2;
                if (col[mid] < a) lo = mid + 1; else hi = mid;
            }
            const double *xi = X + (size_t)i * k;
            for (int64_t e = lo; e < row_ptr[i + 1]; e++) {
                int64_t j = col[e];
                if (j >= b || j >= i) break;
                const double h = vload(val, e, val_fp32);
                double *yj = Y + (size_t)j * k;
                for (int32_t q = 0; q < k; q++) yj[q] += h * xi[q];
            }
        }
    }
}

/*
 * Form (ii): expand the triangle to full symmetric CSR, then one plain row
 * loop.  Independent of form (i): it never runs a transposed loop.
 * Returns 0, or -1 if memory could not be allocated.
 */
int oracle_spmm_full(int64_t n, const int64_t *row_ptr, const int32_t *col,
                     const void *val, int val_fp32, const double *X, int32_t k,
                     double *Y) {
    int64_t *cnt = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            cnt[i + 1]++;
            if (col[e] != i) cnt[col[e] + 1]++;
        }
    for (int64_t i = 0; i < n; i++) cnt[i + 1] += cnt[i];
    int64_t nnz_full = cnt[n];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *fcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz_full ? nnz_full : 1));
    double *fval = (double *)malloc(sizeof(double) * (size_t)(nnz_full ? nnz_full : 1));
    if (!fill || !fcol || !fval) { free(cnt); free(fill); free(fcol); free(fval); return -1; }
    memcpy(fill, cnt, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            int64_t j = col[e];
            double h = vload(val, e, val_fp32);
            fcol[fill[i]] = (int32_t)j; fval[fill[i]++] = h;
            if (j != i) { fcol[fill[j]] = (int32_t)i; fval[fill[j]++] = h; }
        }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; i++) {
        double *yi = Y + (size_t)i * k;
        for (int32_t q = 0; q < k; q++) yi[q] = 0.0;
        for (int64_t e = cnt[i]; e < cnt[i + 1]; e++) {
            const double *xj = X + (size_t)fcol[e] * k;
            for (int32_t q = 0; q < k; q++) yi[q] += fval[e] * xj[q];
        }
    }
    free(cnt); free(fill); free(fcol); free(fval);
    return 0;
}

/*
 * Selected output rows of Y = H X, each computed on its own from the
 * definition (row i of L, plus column i of L below the diagonal found by
 * scanning the later rows).  Used to check large products at sampled rows.
 * Cost O(nnz) per sampled row; rows are independent (parallel over rows).
 */
void oracle_spmm_rows(int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const void *val, int val_fp32, const double *X, int32_t k,
                      int64_t nrows, const int64_t *rows, double *Yrows) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < nrows; s++) {
        int64_t i = rows[s];
        double *y = Yrows + (size_t)s * k;
        for (int32_t q = 0; q < k; q++) y[q] = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            const double h = vload(val, e, val_fp32);
            const double *xj = X + (size_t)col[e] * k;
            for (int32_t q = 0; q < k; q++) y[q] += h * xj[q];
        }
        for (int64_t r = i + 1; r < n; r++) {
            int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (col[mid] < i) lo = mid + 1; else hi = mid;
            }
            if (lo < row_ptr[r + 1] && col[lo] == i) {
                const double h = vload(val, lo, val_fp32);
                const double *xr = X + (size_t)r * k;
                for (int32_t q = 0; q < k; q++) y[q] += h * xr[q];
            }
        }
    }
}

/* Gershgorin bound ||H||_G = max_i sum_j |h_ij| over full rows of H. */
double oracle_gershgorin(int64_t n, const int64_t *row_ptr, const int32_t *col,
                         const void *val, int val_fp32) {
    double *s = (double *)calloc((size_t)n, sizeof(double));
    if (!s) return -1.0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            double a = vload(val, e, val_fp32);
            a = a < 0 ? -a : a;
            s[i] += a;
            if (col[e] != i) s[col[e]] += a;
        }
    double m = 0.0;
    for (int64_t i = 0; i < n; i++) if (s[i] > m) m = s[i];
    free(s);
    return m;
}

/* Diagonal of H (d_i = h_ii; 0 where no diagonal entry is stored). */
void oracle_diag(int64_t n, const int64_t *row_ptr, const int32_t *col,
                 const void *val, int val_fp32, double *d) {
    for (int64_t i = 0; i < n; i++) {
        d[i] = 0.0;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++)
            if (col[e] == i) d[i] = vload(val, e, val_fp32);
    }
}

/* Dense symmetric block H[r0:r0+m, r0:r0+m] (row-major m x m) from the triangle. */
void oracle_dense_block(int64_t n, const int64_t *row_ptr, const int32_t *col,
                        const void *val, int val_fp32, int64_t r0, int32_t m,
                        double *B) {
    memset(B, 0, sizeof(double) * (size_t)m * (size_t)m);
    for (int64_t i = r0; i < r0 + m && i < n; i++)
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) {
            int64_t j = col[e];
            if (j < r0) continue;
            double h = vload(val, e, val_fp32);
            B[(size_t)(i - r0) * m + (j - r0)] = h;
            B[(size_t)(j - r0) * m + (i - r0)] = h;
        }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
