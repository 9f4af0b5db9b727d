/*
 * CPU FP64 oracle: small dense symmetric eigensolver, Cholesky and LU.
 *
 * TEST INFRASTRUCTURE ONLY (see spmm.c).  Shares no code with the CUDA path.
 *
 * The eigensolver is the cyclic Jacobi method (Golub & Van Loan, Matrix
 * Computations, Section 8.5: a sweep over all (p, q) pairs, each applying the
 * 2x2 symmetric Schur rotation that zeroes a_pq).  It stands in for LAPACK's
 * dsygv used for the projected problem of eq. (rreig) (Section 3.4).
 * All matrices are row-major, FP64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/*
 * Eigen-decomposition A = V diag(w) V^T of the symmetric m x m matrix A
 * (overwritten).  w ascending, V row-major with eigenvectors in columns.
 * Returns the number of sweeps used, or -1 if it did not converge.
 */
int oracle_jacobi_eig(int32_t m, double *A, double *w, double *V, int32_t max_sweeps) {
    for (int32_t i = 0; i < m; i++)
        for (int32_t j = 0; j < m; j++) V[(size_t)i * m + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (size_t e = 0; e < (size_t)m * m; e++) fro += A[e] * A[e];
    fro = sqrt(fro);
    int sweeps = 0, done = (m <= 1);
    while (!done && sweeps < max_sweeps) {
        double off = 0.0;
        for (int32_t p = 0; p < m; p++)
            for (int32_t q = p + 1; q < m; q++) off += 2.0 * A[(size_t)p * m + q] * A[(size_t)p * m + q];
        if (sqrt(off) <= 1e-15 * fro || off == 0.0) { done = 1; break; }
        for (int32_t p = 0; p < m - 1; p++) {
            for (int32_t q = p + 1; q < m; q++) {
                double apq = A[(size_t)p * m + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
                /* symmetric Schur rotation: (c, s) with [c s; -s c]^T A_pq [c s; -s c] diagonal */
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                        : -1.0 / (-tau + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- A J (columns p, q) */
                for (int32_t i = 0; i < m; i++) {
                    double aip = A[(size_t)i * m + p], aiq = A[(size_t)i * m + q];
                    A[(size_t)i * m + p] = c * aip - s * aiq;
                    A[(size_t)i * m + q] = s * aip + c * aiq;
                }
                /* A <- J^T A (rows p, q) */
                for (int32_t j = 0; j < m; j++) {
                    double apj = A[(size_t)p * m + j], aqj = A[(size_t)q * m + j];
                    A[(size_t)p * m + j] = c * apj - s * aqj;
                    A[(size_t)q * m + j] = s * apj + c * aqj;
                }
                A[(size_t)p * m + q] = 0.0;
                A[(size_t)q * m + p] = 0.0;
                /* V <- V J */
                for (int32_t i = 0; i < m; i++) {
                    double vip = V[(size_t)i * m + p], viq = V[(size_t)i * m + q];
                    V[(size_t)i * m + p] = c * vip - s * viq;
                    V[(size_t)i * m + q] = s * vip + c * viq;
                }
            }
        }
        sweeps++;
    }
    if (!done) {
        double off = 0.0;
        for (int32_t p = 0; p < m; p++)
            for (int32_t q = p + 1; q < m; q++) off += 2.0 * A[(size_t)p * m + q] * A[(size_t)p * m + q];
        if (!(sqrt(off) <= 1e-15 * fro || off == 0.0)) return -1;
    }
    for (int32_t i = 0; i < m; i++) w[i] = A[(size_t)i * m + i];
    /* selection sort, ascending, permuting the columns of V alongside */
    for (int32_t i = 0; i < m; i++) {
        int32_t b = i;
        for (int32_t j = i + 1; j < m; j++) if (w[j] < w[b]) b = j;
        if (b != i) {
            double tw = w[i]; w[i] = w[b]; w[b] = tw;
            for (int32_t r = 0; r < m; r++) {
                double tv = V[(size_t)r * m + i];
                V[(size_t)r * m + i] = V[(size_t)r * m + b];
                V[(size_t)r * m + b] = tv;
            }
        }
    }
    return sweeps;
}

/*
 * Cholesky factorisation A = L L^T of the symmetric m x m matrix A (row-major,
 * lower triangle read).  L written to Lout (upper part zeroed).  Returns 0, or
 * the 1-based index of the first pivot that is not > 0.
 */
int oracle_cholesky(int32_t m, const double *A, double *Lout) {
    memset(Lout, 0, sizeof(double) * (size_t)m * m);
    for (int32_t j = 0; j < m; j++) {
        double s = A[(size_t)j * m + j];
        for (int32_t p = 0; p < j; p++) s -= Lout[(size_t)j * m + p] * Lout[(size_t)j * m + p];
        if (!(s > 0.0)) return j + 1;
        double ljj = sqrt(s);
        Lout[(size_t)j * m + j] = ljj;
        for (int32_t i = j + 1; i < m; i++) {
            double t = A[(size_t)i * m + j];
            for (int32_t p = 0; p < j; p++) t -= Lout[(size_t)i * m + p] * Lout[(size_t)j * m + p];
            Lout[(size_t)i * m + j] = t / ljj;
        }
    }
    return 0;
}

/*
 * Solve A Y = B for the m x m matrix A and m x r right-hand sides B (both
 * row-major; A and B overwritten, the solution left in B) by Gaussian
 * elimination with partial pivoting.  Returns 0, or -1 for an exactly
 * singular pivot.
 */
int oracle_lu_solve(int32_t m, double *A, int32_t r, double *B) {
    for (int32_t c = 0; c < m; c++) {
        int32_t piv = c;
        double best = fabs(A[(size_t)c * m + c]);
        for (int32_t i = c + 1; i < m; i++)
            if (fabs(A[(size_t)i * m + c]) > best) { best = fabs(A[(size_t)i * m + c]); piv = i; }
        if (best == 0.0) return -1;
        if (piv != c) {
            for (int32_t j = 0; j < m; j++) {
                double t = A[(size_t)c * m + j]; A[(size_t)c * m + j] = A[(size_t)piv * m + j]; A[(size_t)piv * m + j] = t;
            }
            for (int32_t j = 0; j < r; j++) {
                double t = B[(size_t)c * r + j]; B[(size_t)c * r + j] = B[(size_t)piv * r + j]; B[(size_t)piv * r + j] = t;
            }
        }
        for (int32_t i = c + 1; i < m; i++) {
            double f = A[(size_t)i * m + c] / A[(size_t)c * m + c];
            if (f == 0.0) continue;
            for (int32_t j = c; j < m; j++) A[(size_t)i * m + j] -= f * A[(size_t)c * m + j];
            for (int32_t j = 0; j < r; j++) B[(size_t)i * r + j] -= f * B[(size_t)c * r + j];
        }
    }
    for (int32_t c = m - 1; c >= 0; c--) {
        for (int32_t j = 0; j < r; j++) {
            double s = B[(size_t)c * r + j];
            for (int32_t p = c + 1; p < m; p++) s -= A[(size_t)c * m + p] * B[(size_t)p * r + j];
            B[(size_t)c * r + j] = s / A[(size_t)c * m + c];
        }
    }
    return 0;
}
