// One-CTA FP64 kernels on the small matrices of block LOBPCG (Algorithm 1):
//
//   k_rayleigh_ritz  the k leftmost pairs of the pencil (G, O) of eq. rreig
//                    (m = 2k or 3k; up to 96 for the block Davidson basis)
//   k_orth_factor    the Cholesky-QR factor of W (Section 3.4), SVQB on
//                    breakdown
//
// All arithmetic is FP64.  GB300 issues one FP64 warp instruction per 64
// cycles per warp (about one per 19 cycles per SM), whatever the number of
// active lanes, so these kernels count warp instructions on their critical
// paths: work that can share an instruction goes into its lanes.
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"

namespace lobpcg {

// ---------------------------------------------------------------- small FP64 (one CTA)



__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// GB300 issues one FP64 warp instruction per 64 cycles on each SM
// sub-partition (one warp's dependent FP64 operations are 64 cycles apart,
// and four warps on four sub-partitions reach the SM's FP64 rate), while an
// FP64 division or square root is a sequence of several FP64 instructions.
// The one-CTA kernels below therefore count FP64 warp instructions: lanes
// are filled before warps are added, reciprocals and reciprocal square
// roots start from a float32 estimate refined by Newton steps, and the
// float32 estimate is taken from the bit pattern (integer operations only).

// float32 value of x with its mantissa truncated (|x| within 2^+-100).
__device__ __forceinline__ float f32_trunc(double x) {
    const int hi = __double2hiint(x);
    const unsigned lo = static_cast<unsigned>(__double2loint(x));
    const unsigned e = static_cast<unsigned>(((hi >> 20) & 0x7ff) - 1023 + 127);
    const unsigned mant = (static_cast<unsigned>(hi & 0xfffff) << 3) | (lo >> 29);
    return __uint_as_float((static_cast<unsigned>(hi) & 0x80000000u) | (e << 23) | mant);
}
// Exact float64 value of a normal float32 f.
__device__ __forceinline__ double f64_exact(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = ((u >> 23) & 0xffu) - 127u + 1023u;
    const unsigned hi = (u & 0x80000000u) | (e << 20) | ((u & 0x7fffffu) >> 3);
    return __hiloint2double(static_cast<int>(hi), static_cast<int>((u & 7u) << 29));
}
__device__ __forceinline__ bool in_seed_range(double x) {   // |x| within [2^-100, 2^100]
    const int e = (__double2hiint(x) >> 20) & 0x7ff;
    return e >= 1023 - 100 && e <= 1023 + 100;
}
// 1/q: float32 estimate (relative error ~2^-22), two Newton steps
// r <- r + r (1 - q r); IEEE division outside the seed range.
__device__ __forceinline__ double rcp64(double q) {
    if (!in_seed_range(q)) return 1.0 / q;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f32_trunc(q)));
    double r = f64_exact(rf);
    double e = fma(-q, r, 1.0);
    r = fma(r, e, r);
    e = fma(-q, r, 1.0);
    return fma(r, e, r);
}
// 1/sqrt(s) for s > 0: float32 estimate, two Newton steps r <- r (3/2 - s r^2 / 2).
__device__ __forceinline__ double rsqrt64(double s) {
    if (!in_seed_range(s)) return 1.0 / sqrt(s);
    float rf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f32_trunc(s)));
    double r = f64_exact(rf);
    const double hs = 0.5 * s;
    r = r * fma(-hs, r * r, 1.5);
    return r * fma(-hs, r * r, 1.5);
}
// |a| >= |b| on the bit patterns (integer compare, no FP64 instruction).
__device__ __forceinline__ bool abs_ge(double a, double b) {
    return (static_cast<unsigned long long>(__double_as_longlong(a)) & 0x7fffffffffffffffull) >=
           (static_cast<unsigned long long>(__double_as_longlong(b)) & 0x7fffffffffffffffull);
}

// Row r and column c of the e-th entry of a strictly lower triangle listed
// row by row ((1,0), (2,0), (2,1), ...): r(r-1)/2 <= e < r(r+1)/2.
__device__ __forceinline__ void tri_rc(int e, int &r, int &c) {
    int q = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) + 1.f) * 0.5f);
    while (q * (q - 1) / 2 > e) --q;
    while ((q + 1) * q / 2 <= e) ++q;
    r = q;
    c = e - q * (q - 1) / 2;
}

// In-place Cholesky of the m x m matrix A (lower triangle used), row-major in
// shared memory: A = L L^T, L in the lower triangle, upper triangle zeroed.
// Right-looking; the pivot reciprocal 1/L_jj goes to rd[j].  Returns false if
// a pivot is not > 0 or the pivots span more than `span` (max L_jj / min L_jj).
__device__ bool cta_cholesky(double *A, int m, double span, double *rd) {
    __shared__ int ok;
    __shared__ double dmin, dmax, rl;
    if (threadIdx.x == 0) { ok = 1; dmin = 1e300; dmax = 0.0; }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (threadIdx.x == 0) {
            const double sj = A[j * m + j];
            if (!(sj > 0.0)) {
                ok = 0;
            } else {
                const double r = rsqrt64(sj);
                const double l = sj * r;
                A[j * m + j] = l;
                rl = r;
                rd[j] = r;
                dmin = fmin(dmin, l);
                dmax = fmax(dmax, l);
            }
        }
        __syncthreads();
        if (!ok) return false;
        const double r = rl;
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i * m + j] *= r;
        __syncthreads();
        // trailing lower triangle including its diagonal: pairs (i, l), j < l <= i
        const int nt = m - j - 1;
        const int cnt = nt * (nt + 1) / 2;
        for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
            int r1, c1;
            tri_rc(e, r1, c1);            // strictly lower pairs of an (nt + 1) triangle
            const int i = j + r1, l = j + 1 + c1;
            A[i * m + l] -= A[i * m + j] * A[l * m + j];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, jj = e % m;
        if (jj > i) A[e] = 0.0;
    }
    __syncthreads();
    return dmax <= span * dmin;
}

// Li = L^{-1} for lower-triangular L (m x m, shared memory), rd[i] = 1/L_ii:
// column j by forward substitution, one thread per column.
__device__ void cta_tri_inverse(const double *L, const double *rd, double *Li, int m) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        for (int i = 0; i < m; ++i) {
            if (i < j) { Li[i * m + j] = 0.0; continue; }
            double s = (i == j) ? 1.0 : 0.0;
            for (int p = j; p < i; ++p) s -= L[i * m + p] * Li[p * m + j];
            Li[i * m + j] = s * rd[i];
        }
    }
    __syncthreads();
}

// B <- L^{-1} B for lower-triangular L (m x m) with rd[i] = 1 / L_ii; B is
// m x nc, row stride nc (nc <= blockDim).  Right-looking: at step i row i
// holds L_ii z_i (z = L^{-1} B), and rows below subtract L[r][i] z_i.  Rows
// are scaled by rd at the end.  One barrier per step.
__device__ void cta_trsm_rows(const double *L, const double *rd, double *B, int m, int nc) {
    const int per = blockDim.x / nc;                 // rows per pass
    const int c = threadIdx.x % nc, r0 = threadIdx.x / nc;
    for (int i = 0; i + 1 < m; ++i) {
        if (r0 < per) {
            const double zi = B[i * nc + c] * rd[i];
            for (int r = i + 1 + r0; r < m; r += per) B[r * nc + c] = fma(-L[r * m + i], zi, B[r * nc + c]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) B[e] *= rd[e / nc];
    __syncthreads();
}

// Y <- L^{-T} Y (Y m x nc, row stride nc): back substitution, right-looking
// from the last row, same conventions as cta_trsm_rows.
__device__ void cta_trsm_rows_t(const double *L, const double *rd, double *Y, int m, int nc) {
    const int per = blockDim.x / nc;
    const int c = threadIdx.x % nc, r0 = threadIdx.x / nc;
    for (int i = m - 1; i > 0; --i) {
        if (r0 < per) {
            const double ci = Y[i * nc + c] * rd[i];
            for (int r = r0; r < i; r += per) Y[r * nc + c] = fma(-L[i * m + r], ci, Y[r * nc + c]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) Y[e] *= rd[e / nc];
    __syncthreads();
}

// C = A B (m x m, shared), optionally with A or B transposed.
__device__ void cta_matmul(const double *A, bool ta, const double *B, bool tb, double *Cm, int m) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, j = e % m;
        double s = 0.0;
        for (int p = 0; p < m; ++p) {
            const double a = ta ? A[p * m + i] : A[i * m + p];
            const double b = tb ? B[j * m + p] : B[p * m + j];
            s += a * b;
        }
        Cm[e] = s;
    }
    __syncthreads();
}

// Cyclic Jacobi (Golub & Van Loan, Section 8.5) with the round-robin
// ordering: each round rotates m/2 disjoint (p, q) pairs in parallel.
// A (m x m, symmetric) becomes diagonal; V accumulates the rotations.
// Returns the number of sweeps, or -1 if not converged.
__device__ int cta_jacobi(double *A, double *V, int m, double *cs, int *pairs, int max_sweeps) {
    __shared__ double off, fro;
    const int mm = (m % 2) ? m + 1 : m;   // pad odd m with a dummy index
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) V[e] = (e / m == e % m) ? 1.0 : 0.0;
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int e = 0; e < m * m; ++e) f += A[e] * A[e];
        fro = sqrt(f);
    }
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) {
            double o = 0.0;
            for (int p = 0; p < m; ++p)
                for (int q = p + 1; q < m; ++q) o += 2.0 * A[p * m + q] * A[p * m + q];
            off = sqrt(o);
        }
        __syncthreads();
        if (off <= 1e-14 * fro || off == 0.0) return sweep;
        for (int round = 0; round < mm - 1; ++round) {
            // round-robin: position 0 fixed, the others rotate
            for (int t = threadIdx.x; t < mm / 2; t += blockDim.x) {
                int a = (t == 0) ? 0 : 1 + (t - 1 + round) % (mm - 1);
                int b = 1 + (mm - 2 - t + round) % (mm - 1);
                int p = min(a, b), q = max(a, b);
                if (q >= m) { pairs[2 * t] = -1; continue; }
                pairs[2 * t] = p;
                pairs[2 * t + 1] = q;
                const double apq = A[p * m + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                    const double tt = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                                   : -1.0 / (-tau + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    s = tt * c;
                }
                cs[2 * t] = c;
                cs[2 * t + 1] = s;
            }
            __syncthreads();
            // A <- A J (columns p, q of every row), V <- V J
            for (int e = threadIdx.x; e < (mm / 2) * m; e += blockDim.x) {
                const int t = e / m, i = e % m;
                const int p = pairs[2 * t];
                if (p < 0) continue;
                const int q = pairs[2 * t + 1];
                const double c = cs[2 * t], s = cs[2 * t + 1];
                const double aip = A[i * m + p], aiq = A[i * m + q];
                A[i * m + p] = c * aip - s * aiq;
                A[i * m + q] = s * aip + c * aiq;
                const double vip = V[i * m + p], viq = V[i * m + q];
                V[i * m + p] = c * vip - s * viq;
                V[i * m + q] = s * vip + c * viq;
            }
            __syncthreads();
            // A <- J^T A (rows p, q)
            for (int e = threadIdx.x; e < (mm / 2) * m; e += blockDim.x) {
                const int t = e / m, j = e % m;
                const int p = pairs[2 * t];
                if (p < 0) continue;
                const int q = pairs[2 * t + 1];
                const double c = cs[2 * t], s = cs[2 * t + 1];
                const double apj = A[p * m + j], aqj = A[q * m + j];
                A[p * m + j] = c * apj - s * aqj;
                A[q * m + j] = s * apj + c * aqj;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < mm / 2; t += blockDim.x) {
                const int p = pairs[2 * t];
                if (p < 0) continue;
                const int q = pairs[2 * t + 1];
                A[p * m + q] = 0.0;
                A[q * m + p] = 0.0;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        double o = 0.0;
        for (int p = 0; p < m; ++p)
            for (int q = p + 1; q < m; ++q) o += 2.0 * A[p * m + q] * A[p * m + q];
        off = sqrt(o);
    }
    __syncthreads();
    return (off <= 1e-13 * fro || off == 0.0) ? max_sweeps : -1;
}

// The k smallest eigenpairs of the symmetric m x m matrix A (shared memory,
// lower triangle used, destroyed), FP64, one CTA of at least 128 threads
// (m <= 96, k <= 32):
//   1. Householder tridiagonalisation A = Q T Q^T (Golub & Van Loan,
//      Section 8.3.1), updating the lower triangle only; the reflectors stay
//      in A's lower triangle.
//   2. Eigenvalue brackets of T / ||T|| by float32 multisection on the Sturm
//      count (the number of negative pivots of T - x I): one warp per
//      eigenvalue, 32 points per step.
//   3. float64 bisection of the brackets to 1e-10 ||T||: four warps (one per
//      sub-partition), 128 / k points per eigenvalue, with the Sturm count as
//      the sign changes of the leading principal minors p_r of T - x I
//      (p_{r+1} = (d_r - x) p_r - e_{r-1}^2 p_{r-1}: no division).
//   4. Eigenvector by two steps of inverse iteration with T - w_i I
//      (tridiagonal LU with partial pivoting), one lane per pair, the pairs
//      spread over four warps; the eigenvalue is then the Rayleigh quotient.
//      Vectors of eigenvalues closer than 1e-10 ||T|| are re-orthogonalised.
//   5. Back-transformation by the reflectors, V = Q Y, one warp per group of
//      columns (no barrier between reflectors).
// Outputs: w[0..k) ascending, V (m x k, row-major, shared memory).
constexpr int EIG_MAXM = 96;

// Step 5 of cta_eigh_smallest for one warp: columns c = warp + 4 cl of V,
// rows r = rg + RG t (t < NR), lane = cl RG + rg.
template <int NR>
__device__ __forceinline__ void back_transform(const double *A, const double *tau, double *V, int m, int k, int warp,
                                               int lane, int RG, int ncol) {
    const int cl = lane / RG, rg = lane % RG;
    const int c = warp + 4 * cl;
    const bool colok = cl < ncol;
    double vc[NR];
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        const int r = rg + RG * t;
        vc[t] = (colok && r < m) ? V[r * k + c] : 0.0;
    }
    for (int j = m - 3; j >= 0; --j) {
        const double tj = tau[j];
        if (tj == 0.0) continue;
        double dot = 0.0;
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            const int r = rg + RG * t;
            if (r > j && r < m) dot = fma(A[r * m + j], vc[t], dot);
        }
        for (int o = 1; o < RG; o <<= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        dot *= tj;
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            const int r = rg + RG * t;
            if (r > j && r < m) vc[t] = fma(-dot, A[r * m + j], vc[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        const int r = rg + RG * t;
        if (colok && r < m) V[r * k + c] = vc[t];
    }
}

__device__ void cta_eigh_smallest(double *A, int m, int k, double *w, double *V, double *d, double *e,
                                  double *tau, double *pv) {
    __shared__ double red_s, tnorm, tau_s;
    __shared__ double blo[32], bhi[32], e2[EIG_MAXM], sv[EIG_MAXM], sw[EIG_MAXM];
    __shared__ float df[EIG_MAXM], e2f[EIG_MAXM];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // 1. tridiagonalisation
    for (int j = 0; j + 2 < m; ++j) {
        if (warp == 0) {
            double sg = 0.0;
            for (int i = j + 2 + lane; i < m; i += 32) sg = fma(A[i * m + j], A[i * m + j], sg);
            sg = warp_sum_d(sg);
            if (lane == 0) {
                const double x0 = A[(j + 1) * m + j];
                d[j] = A[j * m + j];
                if (sg == 0.0) {
                    tau_s = 0.0;
                    e[j] = x0;
                } else {
                    // alpha = -sign(x0) mu, v = x - alpha e_1 scaled to v_0 = 1,
                    // tau = 2 / (v^T v) = 1 + |x0| / mu, 1 / v_0 by Newton steps
                    const double s2 = fma(x0, x0, sg);
                    const double r = rsqrt64(s2);
                    const double mu = s2 * r;
                    const double alpha = (x0 <= 0.0) ? mu : -mu;
                    tau_s = fma(fabs(x0), r, 1.0);
                    red_s = rcp64(x0 - alpha);
                    e[j] = alpha;
                }
            }
        }
        __syncthreads();
        const double tj = tau_s;
        tau[j] = tj;   // every thread writes the same value
        if (tj == 0.0) {
            if (threadIdx.x == 0) A[(j + 1) * m + j] = 1.0;
            __syncthreads();
            continue;
        }
        const double rs = red_s;
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
            const double v = (i == j + 1) ? 1.0 : A[i * m + j] * rs;
            A[i * m + j] = v;
            sv[i] = v;
        }
        __syncthreads();
        // p = tau A22 v, four threads per row (A22 read through its lower triangle)
        const int nt = m - j - 1;
        const int qend = (4 * nt + 31) & ~31;   // whole warps, so the shuffles see every lane
        for (int q = threadIdx.x; q < qend; q += blockDim.x) {
            const bool act = q < 4 * nt;
            const int i = j + 1 + (q >> 2), part = q & 3;
            double a0 = 0.0, a1 = 0.0;
            if (act) {
                int l = j + 1 + part;
                for (; l + 4 < m; l += 8) {
                    const double m0 = (l <= i) ? A[i * m + l] : A[l * m + i];
                    const double m1 = (l + 4 <= i) ? A[i * m + l + 4] : A[(l + 4) * m + i];
                    a0 = fma(m0, sv[l], a0);
                    a1 = fma(m1, sv[l + 4], a1);
                }
                if (l < m) a0 = fma((l <= i) ? A[i * m + l] : A[l * m + i], sv[l], a0);
            }
            double acc = a0 + a1;
            acc += __shfl_xor_sync(0xffffffffu, acc, 1);
            acc += __shfl_xor_sync(0xffffffffu, acc, 2);
            if (act && part == 0) pv[i] = tj * acc;
        }
        __syncthreads();
        // K = tau v^T p / 2, w = p - K v
        if (warp == 0) {
            double kk = 0.0;
            for (int l = j + 1 + lane; l < m; l += 32) kk = fma(sv[l], pv[l], kk);
            kk = warp_sum_d(kk);
            const double K = 0.5 * tj * kk;
            for (int l = j + 1 + lane; l < m; l += 32) sw[l] = fma(-K, sv[l], pv[l]);
        }
        __syncthreads();
        // A22 -= v w^T + w v^T (lower triangle including the diagonal)
        const int cnt = nt * (nt + 1) / 2;
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
            int r1, c1;
            tri_rc(q, r1, c1);
            const int i = j + r1, l = j + 1 + c1;
            A[i * m + l] -= fma(sv[i], sw[l], sw[i] * sv[l]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (m >= 2) {
            d[m - 2] = A[(m - 2) * m + (m - 2)];
            e[m - 2] = A[(m - 1) * m + (m - 2)];
            if (m >= 3) tau[m - 2] = 0.0;
        }
        d[m - 1] = A[(m - 1) * m + (m - 1)];
        double tn = 0.0;
        for (int i = 0; i < m; ++i) {
            const double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < m ? fabs(e[i]) : 0.0);
            tn = fmax(tn, r);
        }
        tnorm = (tn > 0.0) ? tn : 1.0;
    }
    __syncthreads();
    // T / ||T||: diagonal d / ||T||, squared off-diagonal e^2 / ||T||^2
    const double sc = rcp64(tnorm);
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const double ds = d[r] * sc;
        d[r] = ds;
        df[r] = static_cast<float>(ds);
        if (r + 1 < m) {
            const double es = e[r] * sc;
            e[r] = es;
            e2[r] = es * es;
            e2f[r] = static_cast<float>(es * es);
        }
    }
    __syncthreads();
    // 2. float32 multisection: 32 points per step, each step narrows the
    //    bracket 33-fold.  The float32 count is that of a matrix within a few
    //    float32 roundings of T, so the bracket is widened by 4e-6.
    for (int i = warp; i < k; i += nwarps) {
        float flo = -1.f, fhi = 1.f;
        for (int it = 0; it < 8 && fhi - flo > 2e-7f * fmaxf(fabsf(flo), fabsf(fhi)) + 1e-30f; ++it) {
            const float x = flo + (fhi - flo) * static_cast<float>(lane + 1) / 33.f;
            int cnt = 0;
            float q = df[0] - x;
            cnt += q < 0.f;
            for (int r = 1; r < m; ++r) {
                if (fabsf(q) < 1e-30f) q = (q < 0.f) ? -1e-30f : 1e-30f;
                q = (df[r] - x) - __fdividef(e2f[r - 1], q);
                cnt += q < 0.f;
            }
            const unsigned above = __ballot_sync(0xffffffffu, cnt > i);
            const int first = above ? (__ffs(above) - 1) : 32;    // first point with cnt > i
            const float nlo = (first == 0) ? flo : flo + (fhi - flo) * static_cast<float>(first) / 33.f;
            const float nhi = (first == 32) ? fhi : flo + (fhi - flo) * static_cast<float>(first + 1) / 33.f;
            flo = nlo;
            fhi = nhi;
        }
        if (lane == 0) {
            blo[i] = fmax(-1.0 - 1e-5, static_cast<double>(flo) - 4e-6);
            bhi[i] = fmin(1.0 + 1e-5, static_cast<double>(fhi) + 4e-6);
        }
    }
    __syncthreads();
    // 3. float64 bisection, warps 0..3: eigenvalue i on lanes [i npts, (i+1) npts)
    //    of the 128, npts a power of two (so a group lies within one warp)
    if (warp < 4) {
        int npts = 32;
        while (npts > 1 && npts * k > 128) npts >>= 1;
        const int gl = warp * 32 + lane;
        const int i = gl / npts, jp = gl % npts;
        const bool act = i < k;
        const double frac = static_cast<double>(jp + 1) / static_cast<double>(npts + 1);
        const double step = 1.0 / static_cast<double>(npts + 1);
        double lo = act ? blo[i] : 0.0, hi = act ? bhi[i] : 0.0;
        for (int it = 0; it < 40; ++it) {
            const bool done = !act || !(hi - lo > 1e-10);
            if (__all_sync(0xffffffffu, done)) break;
            const double x = fma(hi - lo, frac, lo);
            int cnt = 0;
            if (act) {
                // a zero minor takes the sign opposite to the previous one (it
                // counts as a sign change, as a zero pivot counts as negative)
                double pp = 1.0, p = d[0] - x;
                if ((__double_as_longlong(p) << 1) == 0) p = -0x1p-80;
                cnt += __double2hiint(p) < 0;
                for (int r = 1; r < m; ++r) {
                    const double t = e2[r - 1] * pp;
                    double pn = fma(d[r] - x, p, -t);
                    if ((__double_as_longlong(pn) << 1) == 0) pn = -p * 0x1p-80;
                    cnt += (__double2hiint(pn) ^ __double2hiint(p)) < 0;
                    pp = p;
                    p = pn;
                    if (((__double2hiint(p) >> 20) & 0x7ff) < 400) {   // |p| < 2^-623: rescale both (rare)
                        p *= 0x1p+600;
                        pp *= 0x1p+600;
                    }
                }
            }
            const unsigned above = __ballot_sync(0xffffffffu, act && cnt > i);
            if (act && !done) {
                const int sh = (i * npts) & 31;
                const unsigned grp = (above >> sh) & ((npts == 32) ? 0xffffffffu : ((1u << npts) - 1u));
                const int first = grp ? (__ffs(grp) - 1) : npts;   // first point with cnt > i
                const double w0 = hi - lo;
                const double nlo = (first == 0) ? lo : fma(w0, step * first, lo);
                const double nhi = (first == npts) ? hi : fma(w0, step * (first + 1), lo);
                lo = nlo;
                hi = nhi;
            }
        }
        if (act && jp == 0) w[i] = 0.5 * (lo + hi);
    }
    __syncthreads();
    // 4. inverse iteration (T scaled by 1 / ||T||): pair i on warp i % 4, lane i / 4
    if (warp < 4 && lane < (k + 3) / 4 && lane * 4 + warp < k) {
        const int i = lane * 4 + warp;
        const double lam = w[i];
        double D[EIG_MAXM], DL[EIG_MAXM], DU[EIG_MAXM], DU2[EIG_MAXM], rD[EIG_MAXM], y[EIG_MAXM];
        bool piv[EIG_MAXM];
        const double pert = 0x1p-52;   // replaces an exactly zero pivot (T scaled to norm 1)
        for (int r = 0; r < m; ++r) {
            D[r] = d[r] - lam;
            DL[r] = (r + 1 < m) ? e[r] : 0.0;
            DU[r] = DL[r];
            DU2[r] = 0.0;
        }
        for (int r = 0; r + 1 < m; ++r) {
            const bool sw_ = !abs_ge(D[r], DL[r]);
            piv[r] = sw_;
            const double pvt = sw_ ? DL[r] : D[r];
            const double rp = rcp64(pvt == 0.0 ? pert : pvt);
            rD[r] = rp;
            if (!sw_) {
                const double f = DL[r] * rp;
                DL[r] = f;
                D[r + 1] = fma(-f, DU[r], D[r + 1]);
            } else {
                const double f = D[r] * rp;
                D[r] = pvt;
                DL[r] = f;
                const double t = DU[r];
                DU[r] = D[r + 1];
                D[r + 1] = fma(-f, D[r + 1], t);
                if (r + 2 < m) {
                    DU2[r] = DU[r + 1];
                    DU[r + 1] = -f * DU[r + 1];
                }
            }
        }
        rD[m - 1] = rcp64(D[m - 1] == 0.0 ? pert : D[m - 1]);
        // start vector 1 + (small multiples of 1/44), exact in float32
        for (int r = 0; r < m; ++r) y[r] = f64_exact(1.f + 0.25f * static_cast<float>((r * 7 + i * 13) % 11) / 11.f);
        for (int sweep = 0; sweep < 2; ++sweep) {
            for (int r = 0; r + 1 < m; ++r) {
                if (!piv[r]) {
                    y[r + 1] = fma(-DL[r], y[r], y[r + 1]);
                } else {
                    const double t = y[r];
                    y[r] = y[r + 1];
                    y[r + 1] = fma(-DL[r], y[r], t);
                }
            }
            y[m - 1] *= rD[m - 1];
            if (m >= 2) y[m - 2] = fma(-DU[m - 2], y[m - 1], y[m - 2]) * rD[m - 2];
            for (int r = m - 3; r >= 0; --r) y[r] = fma(-DU2[r], y[r + 2], fma(-DU[r], y[r + 1], y[r])) * rD[r];
            // no normalisation between the two solves: each grows y by at
            // most 1 / (smallest pivot) <= 2^52, far inside the float64 range
        }
        double n0 = 0.0, n1 = 0.0, q0 = 0.0, q1 = 0.0;
        for (int r = 0; r < m; ++r) {
            double ty = d[r] * y[r];
            if (r > 0) ty = fma(e[r - 1], y[r - 1], ty);
            if (r + 1 < m) ty = fma(e[r], y[r + 1], ty);
            if (r & 1) { n1 = fma(y[r], y[r], n1); q1 = fma(y[r], ty, q1); }
            else { n0 = fma(y[r], y[r], n0); q0 = fma(y[r], ty, q0); }
        }
        const double rn = rsqrt64(n0 + n1);
        w[i] = (q0 + q1) * (rn * rn) * tnorm;   // Rayleigh quotient y^T T y / y^T y
        for (int r = 0; r < m; ++r) V[r * k + i] = y[r] * rn;
    }
    __syncthreads();
    // re-orthogonalise vectors of (nearly) equal eigenvalues, in order
    int close = 0;
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
        const int i = q / k, j2 = q % k;
        if (j2 < i) close |= fabs(w[i] - w[j2]) <= 1e-10 * tnorm;
    }
    if (__syncthreads_or(close)) {
        for (int i = 1; i < k; ++i) {
            for (int j2 = 0; j2 < i; ++j2) {
                if (fabs(w[i] - w[j2]) > 1e-10 * tnorm) continue;
                if (threadIdx.x == 0) {
                    double dot = 0.0;
                    for (int r = 0; r < m; ++r) dot += V[r * k + i] * V[r * k + j2];
                    red_s = dot;
                }
                __syncthreads();
                for (int r = threadIdx.x; r < m; r += blockDim.x) V[r * k + i] -= red_s * V[r * k + j2];
                __syncthreads();
                if (threadIdx.x == 0) {
                    double nrm = 0.0;
                    for (int r = 0; r < m; ++r) nrm += V[r * k + i] * V[r * k + i];
                    red_s = 1.0 / sqrt(nrm);
                }
                __syncthreads();
                for (int r = threadIdx.x; r < m; r += blockDim.x) V[r * k + i] *= red_s;
                __syncthreads();
            }
        }
    }
    // 5. V = Q Y: reflectors H_j = I - tau_j v_j v_j^T, last first.  Warps
    //    0..3 (one per sub-partition) own columns c = warp + 4 u; a warp's
    //    lanes are cpw column slots x RG row groups (row r in group r % RG),
    //    so one FP64 instruction serves cpw columns and the reflectors need no
    //    barrier between them.
    if (warp < 4) {
        const int ncol = (k - warp + 3) / 4;               // columns of this warp
        int cpw = 1;
        while (cpw < ncol) cpw <<= 1;                      // 1, 2, 4 or 8
        const int RG = 32 / cpw;                           // row groups (>= 4)
        const int rows = (m + RG - 1) / RG;                // rows per lane (<= 24)
        if (rows <= 4) back_transform<4>(A, tau, V, m, k, warp, lane, RG, ncol);
        else if (rows <= 8) back_transform<8>(A, tau, V, m, k, warp, lane, RG, ncol);
        else if (rows <= 12) back_transform<12>(A, tau, V, m, k, warp, lane, RG, ncol);
        else back_transform<24>(A, tau, V, m, k, warp, lane, RG, ncol);
    }
    __syncthreads();
}

// Rayleigh-Ritz on the pencil (G, O) of eq. rreig: keep the k leftmost pairs.
// G, O: m x m FP64 (global).  pscale (may be null): scale of the last m - p0
// rows/columns (the P block), applied as D G D, D O D and undone in C.
//   1. Cholesky O = L L^T (pivots within a span of 1e4, i.e. cond(O) <= ~1e8),
//      G_hat = L^-1 G L^-T,
//      Jacobi G_hat = V D V^T, C = L^-T V[:, :k]
//   2. if O is not numerically positive definite and p0 < m, drop the P
//      block (m -> p0; C's P rows zero)
//   3. if that fails too, go through O = U diag(s) U^T, dropping directions
//      with s < 1e-8 s_max: C = U_r s_r^{-1/2} V[:, :k]
// Out: C (m x k), theta (k), status: 0 ok, 1 P dropped, 3 eigen route,
// 2 breakdown (fewer than k directions left).
__global__ void k_rayleigh_ritz(int m, int k, int p0, const double *G, const double *O, int ld, const double *pscale,
                                double *Cout, double *theta, int *status) {
    extern __shared__ __align__(16) double sm[];
    double *sG = sm, *sO = sG + m * m, *sV = sO + m * m;
    __shared__ double cs[2 * 64];
    __shared__ int pairs[2 * 64];
    __shared__ double wsort[96], sig[96];
    __shared__ double tdd[EIG_MAXM], tee[EIG_MAXM], ttau[EIG_MAXM], tpv[EIG_MAXM];
    __shared__ int kept;
    __shared__ double red_big;
    __shared__ double rdv[EIG_MAXM];
    int mm = m;
    int st = 0;
    bool chol = false;
    auto load = [&](int mdim) {
        for (int e = threadIdx.x; e < mdim * mdim; e += blockDim.x) {
            const int i = e / mdim, j = e % mdim;
            double si = 1.0, sj = 1.0;
            if (pscale && i >= p0) si = pscale[i - p0];
            if (pscale && j >= p0) sj = pscale[j - p0];
            sG[e] = 0.5 * (G[i * ld + j] + G[j * ld + i]) * si * sj;
            sO[e] = 0.5 * (O[i * ld + j] + O[j * ld + i]) * si * sj;
        }
        __syncthreads();
    };
    load(mm);
    chol = cta_cholesky(sO, mm, 1e4, rdv);
    if (!chol && p0 < m) {
        mm = p0;
        st = 1;
        load(mm);
        chol = cta_cholesky(sO, mm, 1e4, rdv);
    }
    if (chol) {
        // G_hat = L^{-1} G L^{-T} = L^{-1} (L^{-1} G)^T (G symmetric): two
        // forward substitutions with a transpose between them; L stays in sO
        cta_trsm_rows(sO, rdv, sG, mm, mm);           // sG = L^{-1} G
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) sV[(e % mm) * mm + e / mm] = sG[e];
        __syncthreads();
        cta_trsm_rows(sO, rdv, sV, mm, mm);           // sV = L^{-1} G L^{-T}
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) sG[e] = sV[e];
        __syncthreads();
    } else {
        // eigen route on the full pencil
        st = 3;
        mm = m;
        load(mm);
        cta_jacobi(sO, sV, mm, cs, pairs, 30);         // O = U diag(s) U^T, U in sV
        if (threadIdx.x == 0) {
            double smax = 0.0;
            for (int i = 0; i < mm; ++i) smax = fmax(smax, sO[i * mm + i]);
            int kc = 0;
            for (int i = 0; i < mm; ++i) {
                const double si = sO[i * mm + i];
                sig[i] = (si > 1e-8 * smax) ? 1.0 / sqrt(si) : 0.0;
                kc += si > 1e-8 * smax;
            }
            kept = kc;
        }
        __syncthreads();
        cta_matmul(sG, false, sV, false, sO, mm);      // sO = G U
        cta_matmul(sV, true, sO, false, sG, mm);       // sG = U^T G U
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) sG[e] *= sig[e / mm] * sig[e % mm];
        __syncthreads();
        if (threadIdx.x == 0) {
            double mx = 0.0;
            for (int e = 0; e < mm * mm; ++e) mx = fmax(mx, fabs(sG[e]));
            red_big = 4.0 * mm * mx + 1.0;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) {   // dropped directions sort last
            const int i = e / mm, j = e % mm;
            if (sig[i] == 0.0 || sig[j] == 0.0) sG[e] = (i == j) ? red_big : 0.0;
        }
        // scaled basis U s^{-1/2} into sO (plays the role of L^{-T}'s transpose below)
        __syncthreads();
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) {
            const int i = e / mm, j = e % mm;
            sO[j * mm + i] = sV[e] * sig[j];           // sO[p][i] = U[i][p] s_p^{-1/2}
        }
        __syncthreads();
        if (kept < k) {
            if (threadIdx.x == 0) *status = 2;
            return;
        }
    }
    for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) {
        const int i = e / mm, j = e % mm;
        if (j > i) {
            const double sv = 0.5 * (sG[i * mm + j] + sG[j * mm + i]);
            sG[i * mm + j] = sv;
            sG[j * mm + i] = sv;
        }
    }
    __syncthreads();
    // k smallest eigenpairs of G_hat; eigenvectors (mm x k) into sV
    cta_eigh_smallest(sG, mm, k, wsort, sV, tdd, tee, ttau, tpv);
    // C = L^{-T} Y (Cholesky route) or U s^{-1/2} Y (sO[p][i] = U[i][p]
    // s_p^{-1/2}); rows of a dropped P block are zero; undo the P scaling
    if (chol) cta_trsm_rows_t(sO, rdv, sV, mm, k);
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        double sacc = 0.0;
        if (i < mm) {
            if (chol) {
                sacc = sV[i * k + j];
            } else {
                for (int p = 0; p < mm; ++p) sacc += sO[p * mm + i] * sV[p * k + j];
            }
            if (pscale && i >= p0) sacc *= pscale[i - p0];
        }
        Cout[i * k + j] = sacc;
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x) theta[j] = wsort[j];
    if (threadIdx.x == 0) *status = st;
}

// Orthonormalisation factor for W (Section 3.4), one CTA: B = W^T W (k x k),
// column scaling D = diag(B)^{-1/2} folded in.  Cholesky-QR: D B D = L L^T,
// T = D L^{-T}.  If that breaks down, SVQB (Stathopoulos & Wu 2002):
// D B D = V diag(s) V^T, T = D V diag(s)^{-1/2}, directions with
// s < 1e-12 s_max give zero columns.  W T has orthonormal (or zero) columns.
// status[1] = 0 (Cholesky-QR) or 1 (SVQB).
__global__ void k_orth_factor(int k, const double *B, double *Tout, int *status) {
    __shared__ double sB[32 * 32], sL[32 * 32], dsc[32], rdk[32];
    __shared__ double cs[2 * 16];
    __shared__ int pairs[2 * 16];
    __shared__ double smax;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double b = B[j * k + j];
        dsc[j] = (b > 0.0) ? rsqrt64(b) : 1.0;
    }
    __syncthreads();
    auto load = [&]() {
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int i = e / k, j = e % k;
            sB[e] = 0.5 * (B[i * k + j] + B[j * k + i]) * dsc[i] * dsc[j];
        }
        __syncthreads();
    };
    load();
    if (cta_cholesky(sB, k, 1e7, rdk)) {
        cta_tri_inverse(sB, rdk, sL, k);   // sL = L^{-1}
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int i = e / k, j = e % k;
            Tout[e] = dsc[i] * sL[j * k + i];
        }
        if (threadIdx.x == 0) status[1] = 0;
        return;
    }
    load();
    cta_jacobi(sB, sL, k, cs, pairs, 30);
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int j = 0; j < k; ++j) mx = fmax(mx, sB[j * k + j]);
        smax = mx;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        const double sj = sB[j * k + j];
        Tout[e] = (sj > 1e-12 * smax) ? dsc[i] * sL[i * k + j] / sqrt(sj) : 0.0;
    }
    if (threadIdx.x == 0) status[1] = 1;
}

cudaError_t launch_rayleigh_ritz(int m, int k, int p0, const double *G, const double *O, int ld, const double *pscale,
                                 double *C, double *theta, int *status, cudaStream_t s) {
    const size_t smem = sizeof(double) * 3 * m * m;
    cudaError_t e = cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_rayleigh_ritz<<<1, 256, smem, s>>>(m, k, p0, G, O, ld, pscale, C, theta, status);
    return cudaGetLastError();
}

cudaError_t launch_orth_factor(int k, const double *B, double *T, int *status, cudaStream_t s) {
    k_orth_factor<<<1, 128, 0, s>>>(k, B, T, status);
    return cudaGetLastError();
}

}  // namespace lobpcg
