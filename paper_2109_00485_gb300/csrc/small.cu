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
// Third-order (Householder) refinements of the same float32 estimates: one
// step takes the ~2^-22 relative error of the estimate to ~2^-64, with a
// dependent chain of 3 (reciprocal) or 4 (reciprocal square root) FP64
// operations instead of 4 or 6.
//   1/q:       e = 1 - q r,     r' = r (1 + e + e^2)
//   1/sqrt(s): e = 1 - s r^2,   r' = r (1 + e/2 + 3 e^2/8)
__device__ __forceinline__ double rcp64c(double q) {
    if (!in_seed_range(q)) return 1.0 / q;
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f32_trunc(q)));
    const double r = f64_exact(rf);
    const double e = fma(-q, r, 1.0);
    return fma(r, fma(e, e, e), r);
}
__device__ __forceinline__ double rsqrt64c(double s) {
    if (!in_seed_range(s)) return 1.0 / sqrt(s);
    float rf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(f32_trunc(s)));
    const double r = f64_exact(rf);
    const double e = fma(-s * r, r, 1.0);
    return fma(r * e, fma(e, 0.375, 0.5), r);
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
// lower triangle used, destroyed), FP64, one CTA of 256 threads (m <= 96,
// k <= 32):
//   1. Householder tridiagonalisation A = Q T Q^T (Golub & Van Loan,
//      Section 8.3.1) on the lower triangle.  Per column: warp 0 forms the
//      reflector while the other warps compute y = A22 x with the unscaled
//      column x (v = s (x - alpha e1) and p = tau A22 v = tau s (y - alpha
//      A22 e1), v^T p from x^T y, y_0 and A22[0][0]), then w = p - (tau/2)
//      (v^T p) v and the rank-2 update A22 -= v w^T + w v^T.  Reflector j is
//      kept in row j of A's (unused) upper triangle.
//   2. Eigenvalue brackets of T / ||T|| by float32 Sturm counts (the number
//      of negative pivots of T - x I): 256 points over [-1, 1], then each
//      bracket narrowed by 8-32 points per step on its own lanes.
//   3. float64 bisection of the brackets to 1e-10 ||T||: four warps (one per
//      sub-partition), 4-16 points per eigenvalue, the Sturm count being the
//      sign changes of the leading principal minors p_r of T - x I
//      (p_{r+1} = (d_r - x) p_r - e_{r-1}^2 p_{r-1}: no division).
//   4. Eigenvectors by two steps of inverse iteration with T - w_i I
//      (tridiagonal LU with partial pivoting), all pairs on the lanes of one
//      warp; norms and Rayleigh quotients (the eigenvalues returned) over
//      the rows on four warps.  Vectors of eigenvalues closer than
//      1e-10 ||T|| are re-orthogonalised.
//   5. Back-transformation by the reflectors, V = Q Y, four warps each
//      owning a group of columns (no barrier between reflectors).
// Outputs: w[0..k) ascending, V (m x k, row stride ldv, shared memory).
// wk: shared scratch of 3 * EIG_MAXM doubles; y: EIG_MAXM doubles.
constexpr int EIG_MAXM = 96;
constexpr int EIG_THREADS = 256;

// Folded enumeration of the lower triangle (diagonal included) of an n x n
// block: folded row q holds rows q and n - 1 - q (n + 1 entries), entry
// e = q (n + 1) + c.  Returns false for the repeated half of the middle row
// of an odd n.  Consecutive e are consecutive columns of one row.
__device__ __forceinline__ bool tri_fold(int e, int n, int &a, int &b) {
    const int q = e / (n + 1), c = e - q * (n + 1);
    if (c <= q) {
        a = q;
        b = c;
        return true;
    }
    a = n - 1 - q;
    b = c - q - 1;
    return a > q;
}

// Step 1 of cta_eigh_smallest.  d[0..m), e[0..m-1), tau[0..m-2) out;
// reflector j (v_{j+1} = 1) in A[j][j+1 .. m-1].
__device__ void cta_tridiag(double *A, int m, double *d, double *e, double *tau, double *sx, double *sy, double *sv,
                            double *sw) {
    __shared__ double scal[4];   // tau_j, s_j (v = s_j (x - alpha e1)), alpha_j, K_j
    __shared__ double sred[EIG_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) sx[i] = A[i * m];
    __syncthreads();
    for (int j = 0; j + 2 < m; ++j) {
        const int b0 = j + 1, nt = m - b0;
        if (warp == 0) {
            // reflector of x = A[b0.., j]: alpha = -sign(x0) mu, tau = 1 + |x0| / mu,
            // s = 1 / (x0 - alpha)
            double sg = 0.0;
            for (int i = b0 + 1 + lane; i < m; i += 32) sg = fma(sx[i], sx[i], sg);
            sg = warp_sum_d(sg);
            if (lane == 0) {
                const double x0 = sx[b0];
                d[j] = A[j * m + j];
                if (sg == 0.0) {
                    scal[0] = 0.0;
                    e[j] = x0;
                } else {
                    const double s2 = fma(x0, x0, sg);
                    const double r = rsqrt64c(s2);
                    const double mu = s2 * r;
                    const double alpha = (x0 <= 0.0) ? mu : -mu;
                    scal[0] = fma(fabs(x0), r, 1.0);
                    scal[1] = rcp64c(x0 - alpha);
                    scal[2] = alpha;
                    e[j] = alpha;
                }
            }
        } else {
            // y = A22 x: four lanes per row (columns b0 + part + 4 t), the
            // starting t rotated by the row so that the four rows of a
            // half-warp read different banks; x^T y summed per warp
            const int part = lane & 3, rq = lane >> 2;
            const int T = (nt + 3) >> 2;
            const int rot = (m & 3) ? rq : ((rq * (1 - (m >> 2))) & 3);
            double cxy = 0.0;
            for (int r0 = (warp - 1) * 8; r0 < nt; r0 += (nwarps - 1) * 8) {
                const int i = b0 + r0 + rq;
                const bool act = i < m;
                double a0 = 0.0, a1 = 0.0;
                if (act) {
                    int t = rot % T;
                    for (int u = 0; u < T; ++u) {
                        const int l = b0 + part + 4 * t;
                        if (l < m) {
                            const double a = (l <= i) ? A[i * m + l] : A[l * m + i];
                            if (u & 1) a1 = fma(a, sx[l], a1);
                            else a0 = fma(a, sx[l], a0);
                        }
                        if (++t == T) t = 0;
                    }
                }
                double acc = a0 + a1;
                acc += __shfl_xor_sync(0xffffffffu, acc, 1);
                acc += __shfl_xor_sync(0xffffffffu, acc, 2);
                if (act) {
                    if (part == 0) sy[i] = acc;
                    cxy = fma(sx[i], acc, cxy);
                }
            }
            // one copy per row (lanes of a row hold the same value)
            cxy += __shfl_xor_sync(0xffffffffu, cxy, 4);
            cxy += __shfl_xor_sync(0xffffffffu, cxy, 8);
            cxy += __shfl_xor_sync(0xffffffffu, cxy, 16);
            if (lane == 0) sred[warp] = cxy;
        }
        __syncthreads();
        const double tj = scal[0];
        if (tj == 0.0) {   // x = x0 e1 already: H_j = I
            if (threadIdx.x == 0) tau[j] = 0.0;
            for (int i = b0 + 1 + threadIdx.x; i < m; i += blockDim.x) sx[i] = A[i * m + b0];
            __syncthreads();
            continue;
        }
        const double sj = scal[1], alpha = scal[2];
        if (warp == 0) {
            // v^T p = tau s^2 (x^T y - 2 alpha y_0 + alpha^2 A22[0][0]), K = tau v^T p / 2
            double c = (lane >= 1 && lane < nwarps) ? sred[lane] : 0.0;
            c += __shfl_xor_sync(0xffffffffu, c, 1);
            c += __shfl_xor_sync(0xffffffffu, c, 2);
            c += __shfl_xor_sync(0xffffffffu, c, 4);
            if (lane == 0) {
                const double q = fma(alpha, fma(alpha, A[b0 * m + b0], -2.0 * sy[b0]), c);
                const double ts = tj * sj;
                scal[3] = 0.5 * (ts * ts) * q;
                tau[j] = tj;
            }
        } else {
            // v and p = tau s (y - alpha A22 e1); v also into row j (reflector)
            const double ts = tj * sj;
            for (int i = b0 + threadIdx.x - 32; i < m; i += blockDim.x - 32) {
                const double vi = (i == b0) ? 1.0 : sj * sx[i];
                sv[i] = vi;
                A[j * m + i] = vi;
                sw[i] = ts * fma(-alpha, A[i * m + b0], sy[i]);
            }
        }
        __syncthreads();
        {
            const double K = scal[3];
            for (int i = b0 + threadIdx.x; i < m; i += blockDim.x) sw[i] = fma(-K, sv[i], sw[i]);
        }
        __syncthreads();
        // A22 -= v w^T + w v^T on the lower triangle; column b0 below the
        // diagonal is the next x
        const int tot = ((nt + 1) >> 1) * (nt + 1);
        for (int q = threadIdx.x; q < tot; q += blockDim.x) {
            int a, b;
            if (!tri_fold(q, nt, a, b)) continue;
            const int i = b0 + a, l = b0 + b;
            const double val = fma(-sv[i], sw[l], fma(-sw[i], sv[l], A[i * m + l]));
            A[i * m + l] = val;
            if (b == 0 && a > 0) sx[i] = val;
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
    }
    __syncthreads();
}

// Keeps the minor recurrence of the float64 Sturm count in range: when
// |p| < 2^-623, p and its predecessor pp are both multiplied by 2^600 (the
// signs, and so the count, are unchanged).  Done on the exponent fields with
// integer operations, so that the FP64 pipe, the bottleneck of the
// recurrence, issues nothing for it; pp's exponent saturates below the
// infinity code (pp then dominates p by more than 2^1000, and the next minor
// takes pp's sign either way).
__device__ __forceinline__ void rescale_pair(double &p, double &pp) {
    const int hp = __double2hiint(p), hq = __double2hiint(pp);
    const int add = (((hp >> 20) & 0x7ff) < 400) ? 600 : 0;
    const int eq = min(((hq >> 20) & 0x7ff) + add, 2046);
    p = __hiloint2double(hp + (add << 20), __double2loint(p));
    pp = __hiloint2double((hq & static_cast<int>(0x800fffffu)) | (eq << 20), __double2loint(pp));
}

// Steps 2-3 of cta_eigh_smallest: w[0..k) = eigenvalues of T / ||T|| to
// 1e-10 (brackets' midpoints).  d, e: T (scaled in place to T / ||T||);
// e2 (EIG_MAXM doubles), df, e2f (EIG_MAXM floats), iwk (512 ints) scratch.
// Returns ||T||.
__device__ double cta_tri_eigvals(int m, int k, double *d, double *e, double *e2, float *df, float *e2f, int *iwk,
                                  double *w) {
    __shared__ unsigned long long tnb[EIG_THREADS / 32];
    __shared__ double blo[32], bhi[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    // ||T||_inf: non-negative doubles compare as their bit patterns
    unsigned long long tb = 0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        double t = fabs(d[r]);
        if (r > 0) t += fabs(e[r - 1]);
        if (r + 1 < m) t += fabs(e[r]);
        tb = max(tb, static_cast<unsigned long long>(__double_as_longlong(t)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tb = max(tb, __shfl_xor_sync(0xffffffffu, tb, o));
    if (lane == 0) tnb[warp] = tb;
    __syncthreads();
    tb = 0;
    for (int q = 0; q < nwarps; ++q) tb = max(tb, tnb[q]);
    double tnorm = __longlong_as_double(static_cast<long long>(tb));
    if (!(tnorm > 0.0)) tnorm = 1.0;
    const double sc = rcp64c(tnorm);
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
    // float32 Sturm count at x (number of eigenvalues of T / ||T|| below x,
    // up to float32 rounding of T)
    auto count32 = [&](float x) {
        int cnt = 0;
        float q = df[0] - x;
        cnt += q < 0.f;
        for (int r = 1; r < m; ++r) {
            if (fabsf(q) < 1e-30f) q = (q < 0.f) ? -1e-30f : 1e-30f;
            q = (df[r] - x) - __fdividef(e2f[r - 1], q);
            cnt += q < 0.f;
        }
        return cnt;
    };
    // 2a. counts at 256 points x_t = -1 + 2 (t + 1) / 257; for each i < k,
    //     nb[warp][i] = points of this warp with count > i
    int *nb = iwk;   // [nwarps][32]
    {
        const int c = count32(-1.f + 2.f * static_cast<float>(threadIdx.x + 1) / 257.f);
        for (int i = 0; i < k; ++i) {
            const unsigned above = __ballot_sync(0xffffffffu, c > i);
            if (lane == 0) nb[warp * 32 + i] = __popc(above);
        }
    }
    __syncthreads();
    // 2b. first point with count > i is 256 - (points above): bracket
    //     between it and its left neighbour; then G lanes per eigenvalue
    //     narrow it (G + 1)-fold per step to 2e-7 relative
    const int G = (k <= 8) ? 32 : (k <= 16 ? 16 : 8);
    {
        const int i = threadIdx.x / G, gl = threadIdx.x % G;
        const bool act = i < k;
        float flo = -1.f, fhi = 1.f;
        if (act) {
            int above = 0;
            for (int q = 0; q < nwarps; ++q) above += nb[q * 32 + i];
            const int first = 256 - above;   // first point with count > i (256: none)
            flo = (first == 0) ? -1.f : -1.f + 2.f * static_cast<float>(first) / 257.f;
            fhi = (first == 256) ? 1.f : -1.f + 2.f * static_cast<float>(first + 1) / 257.f;
        }
        const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
        for (int it = 0; it < 6; ++it) {
            const bool more = act && fhi - flo > 2e-7f * fmaxf(fabsf(flo), fabsf(fhi)) + 1e-30f;
            if (!__any_sync(0xffffffffu, more)) break;
            const float x = flo + (fhi - flo) * static_cast<float>(gl + 1) / static_cast<float>(G + 1);
            const int c = act ? count32(x) : 0;
            const unsigned ab = __ballot_sync(0xffffffffu, act && c > i) & gmask;
            if (more) {
                const unsigned grp = ab >> (lane & ~(G - 1));
                const int first = grp ? (__ffs(grp) - 1) : G;
                const float w0 = fhi - flo;
                const float nlo = (first == 0) ? flo : flo + w0 * static_cast<float>(first) / static_cast<float>(G + 1);
                const float nhi = (first == G) ? fhi : flo + w0 * static_cast<float>(first + 1) / static_cast<float>(G + 1);
                flo = nlo;
                fhi = nhi;
            }
        }
        // the float32 count is that of a matrix within a few float32
        // roundings of T: widen by 4e-6
        if (act && gl == 0) {
            blo[i] = fmax(-1.0 - 1e-5, static_cast<double>(flo) - 4e-6);
            bhi[i] = fmin(1.0 + 1e-5, static_cast<double>(fhi) + 4e-6);
        }
    }
    __syncthreads();
    // 3. float64 bisection on warps 0..3: gpw eigenvalues per warp, npts
    //    points each (lanes [g npts, (g + 1) npts) of the warp)
    if (warp < 4) {
        const int gpw = (k + 3) / 4;
        const int npts = 32 / gpw;
        const int g = lane / npts, jp = lane % npts;
        const int i = warp * gpw + g;
        const bool act = g < gpw && i < k;
        const double frac = static_cast<double>(jp + 1) / static_cast<double>(npts + 1);
        const double step = 1.0 / static_cast<double>(npts + 1);
        const unsigned gmask = ((npts == 32) ? 0xffffffffu : ((1u << npts) - 1u)) << (g * npts);
        double lo = act ? blo[i] : 0.0, hi = act ? bhi[i] : 0.0;
        for (int it = 0; it < 40; ++it) {
            const bool done = !act || !(hi - lo > 1e-10);
            if (__all_sync(0xffffffffu, done)) break;
            const double x = fma(hi - lo, frac, lo);
            int cnt = 0;
            {
                // a zero minor takes the sign opposite to the previous one
                // (a sign change, as a zero pivot counts as negative): the
                // bit pattern of -p 2^-80
                double pp = 1.0, p = d[0] - x;
                if ((__double_as_longlong(p) << 1) == 0) p = -0x1p-80;
                cnt += __double2hiint(p) < 0;
                rescale_pair(p, pp);
                for (int r = 1; r < m; ++r) {
                    const double t = e2[r - 1] * pp;
                    double pn = fma(d[r] - x, p, -t);
                    if ((__double_as_longlong(pn) << 1) == 0)
                        pn = __hiloint2double(static_cast<int>((static_cast<unsigned>(__double2hiint(p)) ^ 0x80000000u) -
                                                               (80u << 20)),
                                              __double2loint(p));
                    cnt += (__double2hiint(pn) ^ __double2hiint(p)) < 0;
                    pp = p;
                    p = pn;
                    rescale_pair(p, pp);
                }
            }
            const unsigned above = __ballot_sync(0xffffffffu, act && cnt > i) & gmask;
            if (act && !done) {
                const unsigned grp = above >> (g * npts);
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
    return tnorm;
}

// Row stride of the eigenvector block V (m x k) in shared memory: with
// cpw columns per warp slot in the back-transformation, ldv = cpw (mod 16)
// puts the 16 lanes of a half-warp on 16 different 8-byte banks; ldv = k if
// that does not fit in the m x m region.
__host__ __device__ inline int eig_ldv(int m, int k) {
    const int ncw = (k + 3) / 4;
    int cpw = 1;
    while (cpw < ncw) cpw <<= 1;
    int ldv = k;
    while ((ldv - cpw) % 16 != 0) ++ldv;
    return (ldv <= m) ? ldv : k;
}

__device__ void cta_eigh_smallest(double *A, int m, int k, double *w, double *V, int ldv, double *d, double *e,
                                  double *tau, double *y, double *wk) {
    __shared__ double e2[EIG_MAXM];
    __shared__ float df[EIG_MAXM], e2f[EIG_MAXM];
    __shared__ double red_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // 1. tridiagonalisation (wk: x, v, w; y: A22 x)
    cta_tridiag(A, m, d, e, tau, wk, y, wk + EIG_MAXM, wk + 2 * EIG_MAXM);
    // 2-3. eigenvalues of T / ||T|| (d, e scaled in place)
    const double tnorm = cta_tri_eigvals(m, k, d, e, e2, df, e2f, reinterpret_cast<int *>(wk), w);
    // 4. inverse iteration on T / ||T||, pair i on lane i of warp 0: LU with
    //    partial pivoting of T - w_i I carried in registers row by row (the
    //    pivot row's reciprocal, multiplier and first and second
    //    superdiagonals kept for the solves), then two solves from a fixed
    //    start vector
    if (warp == 0 && lane < k) {
        const int i = lane;
        const double lam = w[i];
        double rD[EIG_MAXM], DLf[EIG_MAXM], DUs[EIG_MAXM], DU2s[EIG_MAXM], yv[EIG_MAXM];
        unsigned pivm[(EIG_MAXM + 31) / 32] = {};
        const double pert = 0x1p-52;   // replaces an exactly zero pivot (T scaled to norm 1)
        double Dc = d[0] - lam;
        double Uc = (m > 1) ? e[0] : 0.0;
        for (int r = 0; r + 1 < m; ++r) {
            const double Lr = e[r];
            const double Dn = d[r + 1] - lam;
            const double Un = (r + 2 < m) ? e[r + 1] : 0.0;
            const bool sw = !abs_ge(Dc, Lr);
            double pvt = sw ? Lr : Dc;
            if ((__double_as_longlong(pvt) << 1) == 0) pvt = pert;
            const double rp = rcp64c(pvt);
            rD[r] = rp;
            const double f = (sw ? Dc : Lr) * rp;
            DLf[r] = f;
            const double a = sw ? Dn : Uc;   // U[r][r+1]
            const double b = sw ? Uc : Dn;
            DUs[r] = a;
            DU2s[r] = sw ? Un : 0.0;         // U[r][r+2]
            Dc = fma(-f, a, b);
            Uc = sw ? -f * Un : Un;
            if (sw) pivm[r >> 5] |= 1u << (r & 31);
        }
        if ((__double_as_longlong(Dc) << 1) == 0) Dc = pert;
        rD[m - 1] = rcp64c(Dc);
        // start vector 1 + (small multiples of 1/44), exact in float32
        for (int r = 0; r < m; ++r) yv[r] = f64_exact(1.f + 0.25f * static_cast<float>((r * 7 + i * 13) % 11) / 11.f);
        for (int sweep = 0; sweep < 2; ++sweep) {
            // L^{-1} with the row exchanges
            double cur = yv[0];
            for (int r = 0; r + 1 < m; ++r) {
                const double nx = yv[r + 1];
                const bool pv = (pivm[r >> 5] >> (r & 31)) & 1u;
                const double a = pv ? nx : cur;
                const double b = pv ? cur : nx;
                yv[r] = a;
                cur = fma(-DLf[r], a, b);
            }
            // U^{-1}, no normalisation between the two solves: each grows y
            // by at most 1 / (smallest pivot) <= 2^52, far inside the range
            double y1 = cur * rD[m - 1];
            yv[m - 1] = y1;
            if (m >= 2) {
                double y2 = y1;
                y1 = fma(-DUs[m - 2], y2, yv[m - 2]) * rD[m - 2];
                yv[m - 2] = y1;
                for (int r = m - 3; r >= 0; --r) {
                    const double yr = fma(-DU2s[r], y2, fma(-DUs[r], y1, yv[r])) * rD[r];
                    yv[r] = yr;
                    y2 = y1;
                    y1 = yr;
                }
            }
        }
        for (int r = 0; r < m; ++r) V[r * ldv + i] = yv[r];
    }
    __syncthreads();
    // norms and Rayleigh quotients y^T T y / y^T y: four pairs per warp,
    // eight lanes per pair over rows r = rl + 8 t
    {
        const int g = lane >> 3, rl = lane & 7;
        const int i = warp * 4 + g;
        if (warp * 4 < k) {   // warp-uniform
            const bool act = i < k;
            double n0 = 0.0, q0 = 0.0;
            if (act) {
                for (int r = rl; r < m; r += 8) {
                    const double yr = V[r * ldv + i];
                    double ty = d[r] * yr;
                    if (r > 0) ty = fma(e[r - 1], V[(r - 1) * ldv + i], ty);
                    if (r + 1 < m) ty = fma(e[r], V[(r + 1) * ldv + i], ty);
                    n0 = fma(yr, yr, n0);
                    q0 = fma(yr, ty, q0);
                }
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                n0 += __shfl_xor_sync(0xffffffffu, n0, o);
                q0 += __shfl_xor_sync(0xffffffffu, q0, o);
            }
            __syncwarp();   // every lane of the pair has read V before it is scaled
            if (act) {
                const double rn = rsqrt64c(n0);
                if (rl == 0) w[i] = q0 * (rn * rn) * tnorm;
                for (int r = rl; r < m; r += 8) V[r * ldv + i] *= rn;
            }
        }
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
                    for (int r = 0; r < m; ++r) dot += V[r * ldv + i] * V[r * ldv + j2];
                    red_s = dot;
                }
                __syncthreads();
                for (int r = threadIdx.x; r < m; r += blockDim.x) V[r * ldv + i] -= red_s * V[r * ldv + j2];
                __syncthreads();
                if (threadIdx.x == 0) {
                    double nrm = 0.0;
                    for (int r = 0; r < m; ++r) nrm += V[r * ldv + i] * V[r * ldv + i];
                    red_s = 1.0 / sqrt(nrm);
                }
                __syncthreads();
                for (int r = threadIdx.x; r < m; r += blockDim.x) V[r * ldv + i] *= red_s;
                __syncthreads();
            }
        }
    }
    // 5. V = Q Y: reflectors H_j = I - tau_j v_j v_j^T, last first.  Warp
    //    c4 < 4 owns columns [c4 ncw, (c4 + 1) ncw); its lanes are cpw column
    //    slots x RG row groups (lane = rg cpw + cl), reflector j touching
    //    rows j + 1 + rg + RG t; __syncwarp orders the lanes' shared updates
    if (warp < 4) {
        const int ncw = (k + 3) / 4;
        int cpw = 1;
        while (cpw < ncw) cpw <<= 1;
        const int RG = 32 / cpw;
        const int cl = lane % cpw, rg = lane / cpw;
        const int c = warp * ncw + cl;
        const bool colok = cl < ncw && c < k;
        for (int j = m - 3; j >= 0; --j) {
            const double tj = tau[j];
            if (tj == 0.0) continue;
            const double *vr = A + j * m;
            double dot = 0.0;
            if (colok)
                for (int r = j + 1 + rg; r < m; r += RG) dot = fma(vr[r], V[r * ldv + c], dot);
            for (int o = cpw; o < 32; o <<= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
            dot *= tj;
            if (colok)
                for (int r = j + 1 + rg; r < m; r += RG) V[r * ldv + c] = fma(-dot, vr[r], V[r * ldv + c]);
            __syncwarp();
        }
    }
    __syncthreads();
}

// Cholesky O = L L^T for the Rayleigh-Ritz solve (A: m x m in shared
// memory, lower triangle read).  One barrier per column: warp 0 finishes
// column j + 1 (its update by column j, pivot, scaling) while the other warps
// apply column j to the rest of the trailing triangle; L's columns are kept
// as rows of the upper triangle so that those updates read contiguous rows.
// On success: rd[j] = 1 / L_jj, A[j][j] = L_jj and, for r < i,
//   A[i][r] = L_ir / L_ii   (lower, rows scaled: the back substitution)
//   A[r][i] = L_ir / L_rr   (upper, columns scaled: the forward substitution)
// Returns false if a pivot is not > 0 or the pivots span more than `span`
// (max L_jj / min L_jj); A is then not usable.
__device__ bool cta_cholesky_rr(double *A, int m, double span, double *rd) {
    __shared__ int ok;
    __shared__ double sp_min, sp_max;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    double dmin = 1e300, dmax = 0.0;   // kept by warp 0
    // pivot of column c (its entries below the diagonal final), then L's
    // column c (unscaled) into row c of the upper triangle; warp 0
    auto pivot = [&](int c) {
        const double s = A[c * m + c];
        if (!(s > 0.0)) {
            if (lane == 0) ok = 0;
            return;
        }
        const double r = rsqrt64c(s);
        const double l = s * r;
        dmin = fmin(dmin, l);
        dmax = fmax(dmax, l);
        if (lane == 0) {
            A[c * m + c] = l;
            rd[c] = r;
        }
        for (int i = c + 1 + lane; i < m; i += 32) A[c * m + i] = A[i * m + c] * r;
    };
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    if (warp == 0) pivot(0);
    __syncthreads();
    for (int j = 0; j + 1 < m; ++j) {
        if (!ok) break;
        const double *Lj = A + j * m;   // Lj[i] = L_ij, i > j
        if (warp == 0) {
            const double ljp = Lj[j + 1];
            for (int i = j + 1 + lane; i < m; i += 32) A[i * m + j + 1] = fma(-Lj[i], ljp, A[i * m + j + 1]);
            __syncwarp();
            pivot(j + 1);
        } else {
            const int n = m - j - 2;   // rows and columns j + 2 .. m - 1
            const int tot = ((n + 1) >> 1) * (n + 1);
            for (int q = threadIdx.x - 32; q < tot; q += blockDim.x - 32) {
                int a, b;
                if (!tri_fold(q, n, a, b)) continue;
                const int i = j + 2 + a, l = j + 2 + b;
                A[i * m + l] = fma(-Lj[i], Lj[l], A[i * m + l]);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sp_min = dmin;
        sp_max = dmax;
    }
    __syncthreads();
    if (!ok) return false;
    for (int i = warp; i < m; i += nwarps)
        for (int r = lane; r < i; r += 32) {
            const double lv = A[r * m + i];
            A[i * m + r] = lv * rd[i];
            A[r * m + i] = lv * rd[r];
        }
    __syncthreads();
    return sp_max <= span * sp_min;
}

// B <- L^{-1} B (B: m x nc, row-major, shared) with L from cta_cholesky_rr
// (A's upper triangle: A[i][r] = L_ri / L_ii).  Right-looking: at step i row
// i holds L_ii z_i and rows r > i subtract A[i][r] times it; the rows are
// scaled by 1 / L_rr at the end.  One barrier per step.
__device__ void cta_trsm_fwd_rr(const double *A, const double *rd, double *B, int m, int nc) {
    const int T = blockDim.x, dq = T / nc, dc = T % nc;
    const int q0 = threadIdx.x / nc, c0 = threadIdx.x % nc;
    for (int i = 0; i + 1 < m; ++i) {
        const double *Lt = A + i * m;
        const double *Bi = B + i * nc;
        int r = i + 1 + q0, c = c0;
        while (r < m) {
            B[r * nc + c] = fma(-Lt[r], Bi[c], B[r * nc + c]);
            r += dq;
            c += dc;
            if (c >= nc) {
                c -= nc;
                ++r;
            }
        }
        __syncthreads();
    }
    int r = q0, c = c0;
    while (r < m) {
        B[r * nc + c] *= rd[r];
        r += dq;
        c += dc;
        if (c >= nc) {
            c -= nc;
            ++r;
        }
    }
    __syncthreads();
}

// G_hat = L^{-1} G L^{-T} from B = L^{-1} G (m x m, in place): column c of
// G_hat solves L z = (row c of B)^T, and only z_0..z_c are formed (each
// needs only the rows above it), in row c.  On return B's lower triangle
// (diagonal included) is G_hat's; its upper triangle is not.
__device__ void cta_trsm_sym_rr(const double *A, const double *rd, double *B, int m) {
    for (int i = 0; i + 1 < m; ++i) {
        const double *Lt = A + i * m;
        const int n = m - 1 - i;   // rows c and columns r in i + 1 .. m - 1, r <= c
        const int tot = ((n + 1) >> 1) * (n + 1);
        for (int q = threadIdx.x; q < tot; q += blockDim.x) {
            int a, b;
            if (!tri_fold(q, n, a, b)) continue;
            const int c = i + 1 + a, r = i + 1 + b;
            B[c * m + r] = fma(-Lt[r], B[c * m + i], B[c * m + r]);
        }
        __syncthreads();
    }
    const int nwarps = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int c = threadIdx.x >> 5; c < m; c += nwarps)
        for (int r = lane; r <= c; r += 32) B[c * m + r] *= rd[r];
    __syncthreads();
}

// Y <- L^{-T} Y (Y: m x nc, row stride ldy) with L from cta_cholesky_rr
// (A's lower triangle: A[i][r] = L_ir / L_ii): back substitution from the
// last row, rows scaled by 1 / L_rr at the end.
__device__ void cta_trsm_bwd_rr(const double *A, const double *rd, double *Y, int m, int nc, int ldy) {
    const int T = blockDim.x, dq = T / nc, dc = T % nc;
    const int q0 = threadIdx.x / nc, c0 = threadIdx.x % nc;
    for (int i = m - 1; i > 0; --i) {
        const double *Li = A + i * m;
        const double *Yi = Y + i * ldy;
        int r = q0, c = c0;
        while (r < i) {
            Y[r * ldy + c] = fma(-Li[r], Yi[c], Y[r * ldy + c]);
            r += dq;
            c += dc;
            if (c >= nc) {
                c -= nc;
                ++r;
            }
        }
        __syncthreads();
    }
    int r = q0, c = c0;
    while (r < m) {
        Y[r * ldy + c] *= rd[r];
        r += dq;
        c += dc;
        if (c >= nc) {
            c -= nc;
            ++r;
        }
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
    // wk: Jacobi rotations and pairs, then the scaling of the eigen route,
    // then the eigensolver's scratch
    __shared__ double wk[3 * EIG_MAXM];
    __shared__ double wsort[EIG_MAXM];
    double *sig = wk + 144;
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
    chol = cta_cholesky_rr(sO, mm, 1e4, rdv);
    if (!chol && p0 < m) {
        mm = p0;
        st = 1;
        load(mm);
        chol = cta_cholesky_rr(sO, mm, 1e4, rdv);
    }
    if (chol) {
        // G_hat = L^{-1} G L^{-T} = L^{-1} (L^{-1} G)^T (G symmetric): a
        // forward substitution, then the lower triangle of the second one
        cta_trsm_fwd_rr(sO, rdv, sG, mm, mm);         // sG = L^{-1} G
        cta_trsm_sym_rr(sO, rdv, sG, mm);             // lower triangle of sG = G_hat
    } else {
        // eigen route on the full pencil
        st = 3;
        mm = m;
        load(mm);
        cta_jacobi(sO, sV, mm, wk, reinterpret_cast<int *>(wk + 96), 30);   // O = U diag(s) U^T, U in sV
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
    if (!chol) {   // U^T G U from two products: symmetrise
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) {
            const int i = e / mm, j = e % mm;
            if (j > i) {
                const double sv = 0.5 * (sG[i * mm + j] + sG[j * mm + i]);
                sG[i * mm + j] = sv;
                sG[j * mm + i] = sv;
            }
        }
        __syncthreads();
    }
    // k smallest eigenpairs of G_hat; eigenvectors (mm x k) into sV
    const int ldv = eig_ldv(mm, k);
    cta_eigh_smallest(sG, mm, k, wsort, sV, ldv, tdd, tee, ttau, tpv, wk);
    // C = L^{-T} Y (Cholesky route) or U s^{-1/2} Y (sO[p][i] = U[i][p]
    // s_p^{-1/2}); rows of a dropped P block are zero; undo the P scaling
    if (chol) cta_trsm_bwd_rr(sO, rdv, sV, mm, k, ldv);
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        double sacc = 0.0;
        if (i < mm) {
            if (chol) {
                sacc = sV[i * ldv + j];
            } else {
                for (int p = 0; p < mm; ++p) sacc += sO[p * mm + i] * sV[p * ldv + j];
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
    if (cta_cholesky_rr(sB, k, 1e7, rdk)) {
        // sL = L^{-1}: the forward solve of the Rayleigh-Ritz step on I
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) sL[e] = (e / k == e % k) ? 1.0 : 0.0;
        __syncthreads();
        cta_trsm_fwd_rr(sB, rdk, sL, k, k);
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
