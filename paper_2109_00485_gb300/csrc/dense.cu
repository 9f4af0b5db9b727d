// Dense steps of block LOBPCG (Algorithm 1) on tall-skinny n x k blocks.
//
//   k_resid      R = HX - X Theta (Algorithm 1, line 10) with the column norms
//                ||r_j||^2, ||x_j||^2 for the convergence test, and the
//                diagonal preconditioner applied on the way (W = K^{-1} R,
//                Section 3.3 with 1x1 tiles)
//   k_gram       M = A^T B for A = [A_0 .. A_{na-1}], B = [B_0 .. B_{nb-1}]
//                (Gram blocks of eq. go and of Cholesky-QR, Section 3.4),
//                accumulated in FP64 across row runs
//   k_combine    Z_o = [A_0 .. A_{na-1}] C_o for up to two outputs sharing
//                the inputs (eqs. xupd, pupd, upd1, upd2; W <- W - X B;
//                W <- W R^{-1}), in place by rows
//   k_small_*    one-CTA FP64 kernels on the k x k / 3k x 3k matrices:
//                Cholesky-QR factor (Section 3.4) and the Rayleigh-Ritz
//                solve of the pencil (G, O) of eq. rreig
//
// Blocks are row-major (row i: k contiguous entries).  T is float (the FP32
// iteration) or double (the FP64 refinement); Gram accumulation is FP64 for
// both, small matrices are always FP64.
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"

namespace lobpcg {

// ---------------------------------------------------------------- residual

// Guarded shifted pivot: g(t) = sign(t) max(|t|, delta), sign(0) = +1,
// delta = 1e-3 max(1, |theta|).
__device__ __forceinline__ double guard_pivot(double t, double theta) {
    const double delta = 1e-3 * fmax(1.0, fabs(theta));
    const double s = (t >= 0.0) ? 1.0 : -1.0;
    return s * fmax(fabs(t), delta);
}

// One thread per element of the n x k block; blockDim is a multiple of k, so
// a thread keeps one column.  norms[j] += ||r_j||^2, norms[k + j] += ||x_j||^2.
// mode 0: W = R; mode 1: W = R / g(d - theta) (diagonal preconditioner).
template <typename T>
__global__ void k_resid(int64_t n, int k, const T *X, const T *HX, const double *theta, const float *d, T *W,
                        int mode, double *norms) {
    extern __shared__ double red[];   // [2k]
    const int per = blockDim.x / k;   // rows per block pass
    const int j = threadIdx.x % k;
    const bool active = threadIdx.x < per * k;
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) red[q] = 0.0;
    __syncthreads();
    double rr = 0.0, xx = 0.0;
    const double th = theta[j];
    if (active) {
        const int64_t stride = static_cast<int64_t>(gridDim.x) * per;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * per + threadIdx.x / k; i < n; i += stride) {
            const int64_t e = i * k + j;
            const double x = static_cast<double>(X[e]);
            const double r = static_cast<double>(HX[e]) - x * th;
            rr += r * r;
            xx += x * x;
            double w = r;
            if (mode == 1) w = r / guard_pivot(static_cast<double>(d[i]) - th, th);
            W[e] = static_cast<T>(w);
        }
        atomicAdd(&red[j], rr);
        atomicAdd(&red[k + j], xx);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) atomicAdd(&norms[q], red[q]);
}

// ---------------------------------------------------------------- Gram

constexpr int GR_ROWS = 64;     // rows staged per pass
constexpr int GR_THREADS = 256; // 16 x 16 thread grid over the output

// M (ma x mb, FP64, row-major, pre-zeroed) += A^T B.  A = [A_0..A_{na-1}],
// B = [B_0..B_{nb-1}], each block n x k.  Thread (tx, ty) owns the outputs
// (tx + 16u, ty + 16v), u < UA, v < UB.  Products are summed in T over one
// staged run of GR_ROWS rows, then added to FP64 accumulators.
template <typename T, int UA, int UB>
__global__ void __launch_bounds__(GR_THREADS) k_gram(int64_t n, int k, int na, GemmBlocks<T> a, int nb,
                                                     GemmBlocks<T> b, double *M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ma = na * k, mb = nb * k;
    T *sa = reinterpret_cast<T *>(smem_raw);   // [GR_ROWS][ma]
    T *sb = sa + GR_ROWS * ma;                 // [GR_ROWS][mb]
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[UA][UB];
#pragma unroll
    for (int u = 0; u < UA; ++u)
#pragma unroll
        for (int v = 0; v < UB; ++v) acc[u][v] = 0.0;
    const int64_t ntile = (n + GR_ROWS - 1) / GR_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t r0 = tile * GR_ROWS;
        const int rows = static_cast<int>(n - r0 < GR_ROWS ? n - r0 : GR_ROWS);
        __syncthreads();
        for (int e = threadIdx.x; e < GR_ROWS * ma; e += blockDim.x) {
            const int r = e / ma, c = e % ma, blk = c / k, cc = c % k;
            sa[e] = (r < rows) ? a.p[blk][(r0 + r) * k + cc] : T(0);
        }
        for (int e = threadIdx.x; e < GR_ROWS * mb; e += blockDim.x) {
            const int r = e / mb, c = e % mb, blk = c / k, cc = c % k;
            sb[e] = (r < rows) ? b.p[blk][(r0 + r) * k + cc] : T(0);
        }
        __syncthreads();
        T part[UA][UB];
#pragma unroll
        for (int u = 0; u < UA; ++u)
#pragma unroll
            for (int v = 0; v < UB; ++v) part[u][v] = T(0);
        for (int r = 0; r < rows; ++r) {
            T av[UA], bv[UB];
#pragma unroll
            for (int u = 0; u < UA; ++u) {
                const int ia = tx + 16 * u;
                av[u] = ia < ma ? sa[r * ma + ia] : T(0);
            }
#pragma unroll
            for (int v = 0; v < UB; ++v) {
                const int ib = ty + 16 * v;
                bv[v] = ib < mb ? sb[r * mb + ib] : T(0);
            }
#pragma unroll
            for (int u = 0; u < UA; ++u)
#pragma unroll
                for (int v = 0; v < UB; ++v) part[u][v] = fma(av[u], bv[v], part[u][v]);
        }
#pragma unroll
        for (int u = 0; u < UA; ++u)
#pragma unroll
            for (int v = 0; v < UB; ++v) acc[u][v] += static_cast<double>(part[u][v]);
    }
#pragma unroll
    for (int u = 0; u < UA; ++u)
#pragma unroll
        for (int v = 0; v < UB; ++v) {
            const int ia = tx + 16 * u, ib = ty + 16 * v;
            if (ia < ma && ib < mb) atomicAdd(&M[ia * mb + ib], acc[u][v]);
        }
}

// ---------------------------------------------------------------- combine

// Four consecutive values from shared memory (16-byte loads; p 16-byte aligned).
__device__ __forceinline__ void load4(const float *p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double *p, double (&v)[4]) {
    const double2 q0 = *reinterpret_cast<const double2 *>(p), q1 = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

constexpr int CB_ROWS = 32;

// For up to two outputs: Z_o[i, :] = sum_c A[i, c0_o + c] C_o[c, :] over the
// staged rows of A = [A_0..A_{na-1}] (columns c0_o .. ma-1); C_o is
// (ma - c0_o) x k FP64, staged transposed (and zero-padded to 4 columns) in
// T.  Thread (row, j) walks c in steps of 4 with 16-byte shared loads.  Rows
// are staged before any output is written, so outputs may alias inputs.
template <typename T>
__global__ void k_combine(int64_t n, int k, int na, GemmBlocks<T> a, int nout, CombineOut<T> out,
                          double *colsq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ma = na * k;
    const int ma4 = (ma + 3) & ~3;
    T *sa = reinterpret_cast<T *>(smem_raw);       // [CB_ROWS][ma4]
    T *sc = sa + CB_ROWS * ma4;                    // [2][k][ma4]  (C transposed)
    for (int o = 0; o < nout; ++o) {
        const int c0 = out.c0[o];
        for (int e = threadIdx.x; e < k * ma4; e += blockDim.x) {
            const int j = e / ma4, c = e % ma4;
            sc[o * k * ma4 + e] = (c >= c0 && c < ma) ? static_cast<T>(out.C[o][(c - c0) * k + j]) : T(0);
        }
    }
    const int64_t ntile = (n + CB_ROWS - 1) / CB_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t r0 = tile * CB_ROWS;
        const int rows = static_cast<int>(n - r0 < CB_ROWS ? n - r0 : CB_ROWS);
        __syncthreads();
        for (int e = threadIdx.x; e < CB_ROWS * ma4; e += blockDim.x) {
            const int r = e / ma4, c = e % ma4;
            T v = T(0);
            if (r < rows && c < ma) v = a.p[c / k][(r0 + r) * k + c % k];
            sa[e] = v;
        }
        __syncthreads();
        for (int o = 0; o < nout; ++o) {
            const int cstart = out.c0[o] & ~3;
            const T *ct = sc + o * k * ma4;
            for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
                const int r = e / k, j = e % k;
                const T *ar = sa + r * ma4;
                const T *cr = ct + j * ma4;
                T s = T(0);
                for (int c = cstart; c < ma4; c += 4) {
                    T x[4], y[4];
                    load4(ar + c, x);
                    load4(cr + c, y);
                    s = fma(x[0], y[0], s);
                    s = fma(x[1], y[1], s);
                    s = fma(x[2], y[2], s);
                    s = fma(x[3], y[3], s);
                }
                out.z[o][(r0 + r) * k + j] = s;
                if (colsq && o == out.norm_of) atomicAdd(&colsq[j], static_cast<double>(s) * static_cast<double>(s));
            }
        }
    }
}

// ---------------------------------------------------------------- small FP64 (one CTA)

// In-place Cholesky of the m x m matrix A (lower triangle used), row-major in
// shared memory.  Returns false if a pivot is not > 0 or the pivots span more
// than `span` (max L_jj / min L_jj).
__device__ bool cta_cholesky(double *A, int m, double span) {
    __shared__ int ok;
    __shared__ double dmin, dmax;
    if (threadIdx.x == 0) { ok = 1; dmin = 1e300; dmax = 0.0; }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (threadIdx.x == 0) {
            double s = A[j * m + j];
            for (int p = 0; p < j; ++p) s -= A[j * m + p] * A[j * m + p];
            if (!(s > 0.0)) ok = 0;
            const double l = ok ? sqrt(s) : 1.0;
            A[j * m + j] = l;
            dmin = fmin(dmin, l);
            dmax = fmax(dmax, l);
        }
        __syncthreads();
        if (!ok) return false;
        const double ljj = A[j * m + j];
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
            double t = A[i * m + j];
            for (int p = 0; p < j; ++p) t -= A[i * m + p] * A[j * m + p];
            A[i * m + j] = t / ljj;
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

// Li = L^{-1} for lower-triangular L (m x m, shared memory): column j by
// forward substitution, one thread per column.
__device__ void cta_tri_inverse(const double *L, double *Li, int m) {
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        for (int i = 0; i < m; ++i) {
            double s = (i == j) ? 1.0 : 0.0;
            if (i < j) { Li[i * m + j] = 0.0; continue; }
            for (int p = j; p < i; ++p) s -= L[i * m + p] * Li[p * m + j];
            Li[i * m + j] = s / L[i * m + i];
        }
    }
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
        if (off <= 1e-15 * fro || off == 0.0) return sweep;
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
    return (off <= 1e-15 * fro || off == 0.0) ? max_sweeps : -1;
}

// Rayleigh-Ritz on the pencil (G, O) of eq. rreig: keep the k leftmost pairs.
// G, O: m x m FP64 (global).  pscale (may be null): scale of the last m - p0
// rows/columns (the P block), applied as D G D, D O D and undone in C.
//   1. Cholesky O = L L^T (pivots within a span of 1e7), G_hat = L^-1 G L^-T,
//      Jacobi G_hat = V D V^T, C = L^-T V[:, :k]
//   2. if O is not numerically positive definite and p0 < m, drop the P
//      block (m -> p0; C's P rows zero)
//   3. if that fails too, go through O = U diag(s) U^T, dropping directions
//      with s < 1e-12 s_max: C = U_r s_r^{-1/2} V[:, :k]
// Out: C (m x k), theta (k), status: 0 ok, 1 P dropped, 3 eigen route,
// 2 breakdown (fewer than k directions left).
__global__ void k_rayleigh_ritz(int m, int k, int p0, const double *G, const double *O, const double *pscale,
                                double *Cout, double *theta, int *status) {
    extern __shared__ __align__(16) double sm[];
    double *sG = sm, *sO = sG + m * m, *sV = sO + m * m;
    __shared__ double cs[2 * 64];
    __shared__ int pairs[2 * 64];
    __shared__ double wsort[96], sig[96];
    __shared__ int order[96];
    __shared__ int kept;
    int mm = m;
    int st = 0;
    bool chol = false;
    auto load = [&](int mdim) {
        for (int e = threadIdx.x; e < mdim * mdim; e += blockDim.x) {
            const int i = e / mdim, j = e % mdim;
            double si = 1.0, sj = 1.0;
            if (pscale && i >= p0) si = pscale[i - p0];
            if (pscale && j >= p0) sj = pscale[j - p0];
            sG[e] = 0.5 * (G[i * m + j] + G[j * m + i]) * si * sj;
            sO[e] = 0.5 * (O[i * m + j] + O[j * m + i]) * si * sj;
        }
        __syncthreads();
    };
    load(mm);
    chol = cta_cholesky(sO, mm, 1e7);
    if (!chol && p0 < m) {
        mm = p0;
        st = 1;
        load(mm);
        chol = cta_cholesky(sO, mm, 1e7);
    }
    if (chol) {
        // G_hat = L^{-1} G L^{-T}
        cta_tri_inverse(sO, sV, mm);                   // sV = L^{-1}
        cta_matmul(sV, false, sG, false, sO, mm);      // sO = L^{-1} G
        cta_matmul(sO, false, sV, true, sG, mm);       // sG = L^{-1} G L^{-T}
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) sO[e] = sV[e];   // keep L^{-1} in sO
        __syncthreads();
    } else {
        // eigen route on the full pencil
        st = 3;
        mm = m;
        load(mm);
        cta_jacobi(sO, sV, mm, cs, pairs, 60);         // O = U diag(s) U^T, U in sV
        if (threadIdx.x == 0) {
            double smax = 0.0;
            for (int i = 0; i < mm; ++i) smax = fmax(smax, sO[i * mm + i]);
            int kc = 0;
            for (int i = 0; i < mm; ++i) {
                const double si = sO[i * mm + i];
                sig[i] = (si > 1e-12 * smax) ? 1.0 / sqrt(si) : 0.0;
                kc += si > 1e-12 * smax;
            }
            kept = kc;
        }
        __syncthreads();
        cta_matmul(sG, false, sV, false, sO, mm);      // sO = G U
        cta_matmul(sV, true, sO, false, sG, mm);       // sG = U^T G U
        for (int e = threadIdx.x; e < mm * mm; e += blockDim.x) {
            const int i = e / mm, j = e % mm;
            double v = sG[e] * sig[i] * sig[j];
            if (sig[i] == 0.0 || sig[j] == 0.0) v = (i == j) ? 1e300 : 0.0;   // dropped directions sort last
            sG[e] = v;
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
    const int sweeps = cta_jacobi(sG, sV, mm, cs, pairs, 60);
    if (sweeps < 0 && st == 0) st = 4;
    for (int i = threadIdx.x; i < mm; i += blockDim.x) wsort[i] = sG[i * mm + i];
    __syncthreads();
    for (int i = threadIdx.x; i < mm; i += blockDim.x) {
        int r = 0;
        for (int j = 0; j < mm; ++j) r += (wsort[j] < wsort[i]) || (wsort[j] == wsort[i] && j < i);
        order[r] = i;
    }
    __syncthreads();
    // C = B V[:, order[0..k)] with B[i][p] = sO[p][i] (L^{-T}, or U s^{-1/2});
    // rows of a dropped P block are zero; undo the P scaling
    const bool lower = chol;   // L^{-1} is lower triangular: B[i][p] = 0 for p < i
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        double sacc = 0.0;
        if (i < mm) {
            const int col = order[j];
            for (int p = lower ? i : 0; p < mm; ++p) sacc += sO[p * mm + i] * sV[p * mm + col];
            if (pscale && i >= p0) sacc *= pscale[i - p0];
        }
        Cout[i * k + j] = sacc;
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x) theta[j] = wsort[order[j]];
    if (threadIdx.x == 0) *status = st;
}

// Orthonormalisation factor for W (Section 3.4), one CTA: B = W^T W (k x k),
// column scaling D = diag(B)^{-1/2} folded in.  Cholesky-QR: D B D = L L^T,
// T = D L^{-T}.  If that breaks down, SVQB (Stathopoulos & Wu 2002):
// D B D = V diag(s) V^T, T = D V diag(s)^{-1/2}, directions with
// s < 1e-12 s_max give zero columns.  W T has orthonormal (or zero) columns.
// status[1] = 0 (Cholesky-QR) or 1 (SVQB).
__global__ void k_orth_factor(int k, const double *B, double *Tout, int *status) {
    __shared__ double sB[32 * 32], sL[32 * 32], dsc[32];
    __shared__ double cs[2 * 16];
    __shared__ int pairs[2 * 16];
    __shared__ double smax;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const double b = B[j * k + j];
        dsc[j] = (b > 0.0) ? 1.0 / sqrt(b) : 1.0;
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
    if (cta_cholesky(sB, k, 1e7)) {
        cta_tri_inverse(sB, sL, k);   // sL = L^{-1}
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int i = e / k, j = e % k;
            Tout[e] = dsc[i] * sL[j * k + i];
        }
        if (threadIdx.x == 0) status[1] = 0;
        return;
    }
    load();
    cta_jacobi(sB, sL, k, cs, pairs, 60);
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

// ---------------------------------------------------------------- launchers

template <typename T>
cudaError_t launch_resid(int64_t n, int k, const T *X, const T *HX, const double *theta, const float *d, T *W,
                         int mode, double *norms, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * k, s);
    if (e != cudaSuccess) return e;
    const int threads = (256 / k) * k;
    const int64_t per = threads / k;
    int blocks = static_cast<int>(std::min<int64_t>((n + per - 1) / per, static_cast<int64_t>(num_sms) * 8));
    if (blocks < 1) blocks = 1;
    k_resid<T><<<blocks, threads, sizeof(double) * 2 * k, s>>>(n, k, X, HX, theta, d, W, mode, norms);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram(int64_t n, int k, int na, GemmBlocks<T> a, int nb, GemmBlocks<T> b, double *M, int num_sms,
                        cudaStream_t s) {
    const int ma = na * k, mb = nb * k;
    cudaError_t e = cudaMemsetAsync(M, 0, sizeof(double) * ma * mb, s);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(T) * GR_ROWS * (ma + mb);
    const int64_t ntile = (n + GR_ROWS - 1) / GR_ROWS;
    int blocks = static_cast<int>(std::min<int64_t>(ntile, static_cast<int64_t>(num_sms) * 4));
    if (blocks < 1) blocks = 1;
    const int ua = (ma + 15) / 16, ub = (mb + 15) / 16;
#define GRAM_CASE(UA, UB)                                                                                     \
    if (ua <= UA && ub <= UB) {                                                                               \
        e = cudaFuncSetAttribute(k_gram<T, UA, UB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                       \
        k_gram<T, UA, UB><<<blocks, GR_THREADS, smem, s>>>(n, k, na, a, nb, b, M);                            \
        return cudaGetLastError();                                                                            \
    }
    GRAM_CASE(1, 1)
    GRAM_CASE(2, 2)
    GRAM_CASE(3, 3)
    GRAM_CASE(4, 4)
    GRAM_CASE(6, 6)
#undef GRAM_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_combine(int64_t n, int k, int na, GemmBlocks<T> a, int nout, CombineOut<T> out, double *colsq,
                           int num_sms, cudaStream_t s) {
    const int ma4 = (na * k + 3) & ~3;
    const size_t smem = sizeof(T) * (CB_ROWS * ma4 + 2 * ma4 * k);
    cudaError_t e = cudaFuncSetAttribute(k_combine<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (colsq) {
        e = cudaMemsetAsync(colsq, 0, sizeof(double) * k, s);
        if (e != cudaSuccess) return e;
    }
    const int64_t ntile = (n + CB_ROWS - 1) / CB_ROWS;
    int blocks = static_cast<int>(std::min<int64_t>(ntile, static_cast<int64_t>(num_sms) * 4));
    if (blocks < 1) blocks = 1;
    k_combine<T><<<blocks, 256, smem, s>>>(n, k, na, a, nout, out, colsq);
    return cudaGetLastError();
}

cudaError_t launch_rayleigh_ritz(int m, int k, int p0, const double *G, const double *O, const double *pscale,
                                 double *C, double *theta, int *status, cudaStream_t s) {
    const size_t smem = sizeof(double) * 3 * m * m;
    cudaError_t e = cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_rayleigh_ritz<<<1, 256, smem, s>>>(m, k, p0, G, O, pscale, C, theta, status);
    return cudaGetLastError();
}

cudaError_t launch_orth_factor(int k, const double *B, double *T, int *status, cudaStream_t s) {
    k_orth_factor<<<1, 128, 0, s>>>(k, B, T, status);
    return cudaGetLastError();
}

template cudaError_t launch_resid<float>(int64_t, int, const float *, const float *, const double *, const float *,
                                         float *, int, double *, int, cudaStream_t);
template cudaError_t launch_resid<double>(int64_t, int, const double *, const double *, const double *,
                                          const float *, double *, int, double *, int, cudaStream_t);
template cudaError_t launch_gram<float>(int64_t, int, int, GemmBlocks<float>, int, GemmBlocks<float>, double *, int,
                                        cudaStream_t);
template cudaError_t launch_gram<double>(int64_t, int, int, GemmBlocks<double>, int, GemmBlocks<double>, double *,
                                         int, cudaStream_t);
template cudaError_t launch_combine<float>(int64_t, int, int, GemmBlocks<float>, int, CombineOut<float>, double *,
                                           int, cudaStream_t);
template cudaError_t launch_combine<double>(int64_t, int, int, GemmBlocks<double>, int, CombineOut<double>,
                                            double *, int, cudaStream_t);

}  // namespace lobpcg
