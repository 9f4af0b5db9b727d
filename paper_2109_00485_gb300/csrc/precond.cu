// Preconditioners K of Algorithm 1 (W = K^{-1} R), Section 3.3: K is block
// diagonal, built from the diagonal tiles of H shifted close to the wanted
// eigenvalues.  Readings: the shift for column j is its Ritz value theta_j;
// a shifted pivot t is guarded as g(t) = sign(t) max(|t|, 1e-3 max(1,|theta|)).
//   diagonal    : 1x1 tiles, w_ij = r_ij / g(d_i - theta_j)
//   block-Jacobi: 64-row tiles solved exactly through their eigen-
//                 decomposition H_T = Q diag(lam) Q^T (computed once, FP64
//                 Jacobi, stored FP32): w_T = Q diag(1/g(lam - theta_j)) Q^T r_T
//   FOM         : the paper's form: s steps (3-5 in Section 3.3) of the Full
//                 Orthogonalization Method on each shifted 64-row tile
//                 H_T - theta_j I, every column of R its own Krylov space
//                 (x_0 = 0), all columns of a tile advanced together
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>
#include "common.cuh"
#include "internal.h"
#include "precond.h"
#include "mlp.h"

namespace lobpcg {

__device__ __forceinline__ double guard_shift(double t, double theta) {
    const double delta = 1e-3 * fmax(1.0, fabs(theta));
    const double s = (t >= 0.0) ? 1.0 : -1.0;
    return s * fmax(fabs(t), delta);
}

// The same guarded pivot in float32 for float32 blocks, theta_j given as two
// floats (hi + lo, split once per CTA): t = (v - hi) - lo.  GB300 runs FP64
// arithmetic and conversions at 1/64 of its FP32 rate, so a float64 division
// per element cost more than the rest of an apply.
__device__ __forceinline__ float guard_shift_f(float v, float thh, float thl) {
    const float t = __fsub_rn(__fsub_rn(v, thh), thl);
    const float delta = 1e-3f * fmaxf(1.f, fabsf(thh));
    return (t >= 0.f) ? fmaxf(t, delta) : -fmaxf(-t, delta);
}

// theta (k <= 32 doubles) split into float pairs in shared memory
__device__ __forceinline__ void split_theta(const double *theta, int k, float *thh, float *thl) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const float hi = __double2float_rn(theta[j]);
        thh[j] = hi;
        thl[j] = __double2float_rn(theta[j] - static_cast<double>(hi));
    }
    __syncthreads();
}

template <typename T>
__global__ void k_precond_diag(int64_t n, int k, const T *R, const double *theta, const float *d, T *W) {
    __shared__ float thh[32], thl[32];
    if constexpr (std::is_same<T, float>::value) split_theta(theta, k, thh, thl);
    const int64_t total = n * k;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = e / k;
        const int j = static_cast<int>(e - i * k);
        if constexpr (std::is_same<T, float>::value) {
            W[e] = R[e] / guard_shift_f(d[i], thh[j], thl[j]);
        } else {
            const double th = theta[j];
            W[e] = static_cast<T>(static_cast<double>(R[e]) / guard_shift(static_cast<double>(d[i]) - th, th));
        }
    }
}

// One CTA per 64-row diagonal tile: dense symmetric tile from the CSR rows
// (entries with col >= tile start), then cyclic Jacobi in FP64 (round-robin
// parallel ordering), eigenvalues ascending-free (any order is fine for the
// solve), Q and lam stored FP32.  A ragged last tile is padded with an
// identity block whose eigenpairs see zero residual.
constexpr int BJ = 64;

__global__ void __launch_bounds__(256) k_bjacobi_setup(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                                       const float *val_f32, const double *val_f64, float *Q,
                                                       float *lam, int *fail) {
    extern __shared__ __align__(16) double smd[];
    double *A = smd, *V = A + BJ * BJ;
    __shared__ double cs[BJ], fro, off;
    __shared__ int pairs[BJ];
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * BJ;
    const int m = static_cast<int>(n - t0 < BJ ? n - t0 : BJ);
    for (int e = threadIdx.x; e < BJ * BJ; e += blockDim.x) {
        A[e] = 0.0;
        V[e] = (e / BJ == e % BJ) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const int64_t i = t0 + r;
        for (int64_t e = row_ptr[i + 1] - 1; e >= row_ptr[i]; --e) {
            const int64_t c = col[e];
            if (c < t0) break;
            const double v = val_f64 ? val_f64[e] : static_cast<double>(val_f32[e]);
            A[r * BJ + (c - t0)] = v;
            A[(c - t0) * BJ + r] = v;
        }
    }
    for (int r = m + threadIdx.x; r < BJ; r += blockDim.x) A[r * BJ + r] = 1.0;   // padding block
    __syncthreads();
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int e = 0; e < BJ * BJ; ++e) f += A[e] * A[e];
        fro = sqrt(f);
    }
    __syncthreads();
    int sweep = 0;
    for (; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) {
            double o = 0.0;
            for (int p = 0; p < BJ; ++p)
                for (int q = p + 1; q < BJ; ++q) o += 2.0 * A[p * BJ + q] * A[p * BJ + q];
            off = sqrt(o);
        }
        __syncthreads();
        if (off <= 1e-14 * fro || off == 0.0) break;
        for (int round = 0; round < BJ - 1; ++round) {
            for (int t = threadIdx.x; t < BJ / 2; t += blockDim.x) {
                const int a = (t == 0) ? 0 : 1 + (t - 1 + round) % (BJ - 1);
                const int b = 1 + (BJ - 2 - t + round) % (BJ - 1);
                const int p = min(a, b), q = max(a, b);
                pairs[2 * t] = p;
                pairs[2 * t + 1] = q;
                const double apq = A[p * BJ + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double tau = (A[q * BJ + q] - A[p * BJ + p]) / (2.0 * apq);
                    const double tt = (tau >= 0.0) ? 1.0 / (tau + sqrt(1.0 + tau * tau))
                                                   : -1.0 / (-tau + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    s = tt * c;
                }
                cs[2 * t] = c;
                cs[2 * t + 1] = s;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (BJ / 2) * BJ; e += blockDim.x) {
                const int t = e / BJ, i = e % BJ;
                const int p = pairs[2 * t], q = pairs[2 * t + 1];
                const double c = cs[2 * t], s = cs[2 * t + 1];
                const double aip = A[i * BJ + p], aiq = A[i * BJ + q];
                A[i * BJ + p] = c * aip - s * aiq;
                A[i * BJ + q] = s * aip + c * aiq;
                const double vip = V[i * BJ + p], viq = V[i * BJ + q];
                V[i * BJ + p] = c * vip - s * viq;
                V[i * BJ + q] = s * vip + c * viq;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (BJ / 2) * BJ; e += blockDim.x) {
                const int t = e / BJ, j = e % BJ;
                const int p = pairs[2 * t], q = pairs[2 * t + 1];
                const double c = cs[2 * t], s = cs[2 * t + 1];
                const double apj = A[p * BJ + j], aqj = A[q * BJ + j];
                A[p * BJ + j] = c * apj - s * aqj;
                A[q * BJ + j] = s * apj + c * aqj;
            }
            __syncthreads();
            for (int t = threadIdx.x; t < BJ / 2; t += blockDim.x) {
                A[pairs[2 * t] * BJ + pairs[2 * t + 1]] = 0.0;
                A[pairs[2 * t + 1] * BJ + pairs[2 * t]] = 0.0;
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0 && sweep >= 40) atomicExch(fail, 1);
    float *Qt = Q + static_cast<int64_t>(blockIdx.x) * BJ * BJ;
    for (int e = threadIdx.x; e < BJ * BJ; e += blockDim.x) Qt[e] = static_cast<float>(V[e]);
    for (int r = threadIdx.x; r < BJ; r += blockDim.x)
        lam[static_cast<int64_t>(blockIdx.x) * BJ + r] = static_cast<float>(A[r * BJ + r]);
}

// One CTA per tile: z = Q^T r_T (64 x k), z_lj /= g(lam_l - theta_j), w_T = Q z.
// R and W may alias (the tile is staged first).
template <typename T>
__global__ void __launch_bounds__(256) k_bjacobi_apply(int64_t n, int k, const float *Q, const float *lam,
                                                       const T *R, const double *theta, T *W) {
    extern __shared__ __align__(16) float smf[];
    float *sQ = smf;                  // [64][64]
    float *sR = sQ + BJ * BJ;         // [64][k]
    float *sZ = sR + BJ * k;          // [64][k]
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * BJ;
    const int m = static_cast<int>(n - t0 < BJ ? n - t0 : BJ);
    const float *Qt = Q + static_cast<int64_t>(blockIdx.x) * BJ * BJ;
    __shared__ float thh[32], thl[32];
    if constexpr (std::is_same<T, float>::value) split_theta(theta, k, thh, thl);
    for (int e = threadIdx.x; e < BJ * BJ / 4; e += blockDim.x)
        reinterpret_cast<float4 *>(sQ)[e] = reinterpret_cast<const float4 *>(Qt)[e];
    for (int e = threadIdx.x; e < BJ * k; e += blockDim.x) {
        const int r = e / k;
        sR[e] = (r < m) ? static_cast<float>(R[t0 * k + e]) : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BJ * k; e += blockDim.x) {
        const int l = e / k, j = e % k;
        float s = 0.f;
        for (int r = 0; r < BJ; ++r) s = fmaf(sQ[r * BJ + l], sR[r * k + j], s);
        if constexpr (std::is_same<T, float>::value) {
            sZ[e] = s / guard_shift_f(lam[t0 + l], thh[j], thl[j]);
        } else {
            const double th = theta[j];
            sZ[e] = static_cast<float>(s / guard_shift(static_cast<double>(lam[t0 + l]) - th, th));
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
        const int r = e / k, j = e % k;
        float s = 0.f;
        for (int l = 0; l < BJ; ++l) s = fmaf(sQ[r * BJ + l], sZ[l * k + j], s);
        W[t0 * k + e] = static_cast<T>(s);
    }
}

cudaError_t bjacobi_setup(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const void *val, bool val_fp64) {
    const int64_t nt = (h->T.n + BJ - 1) / BJ;
    cudaError_t e = dev_alloc(h, reinterpret_cast<void **>(&h->bj_Q), sizeof(float) * nt * BJ * BJ);
    if (e == cudaSuccess) e = dev_alloc(h, reinterpret_cast<void **>(&h->bj_lam), sizeof(float) * nt * BJ);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(double) * 2 * BJ * BJ;
    e = cudaFuncSetAttribute(k_bjacobi_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_bjacobi_setup<<<static_cast<unsigned>(nt), 256, smem, h->stream>>>(
        h->T.n, row_ptr, col, val_fp64 ? nullptr : static_cast<const float *>(val),
        val_fp64 ? static_cast<const double *>(val) : nullptr, h->bj_Q, h->bj_lam, h->d_err + 1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t precond_apply(const lobpcg_ctx *h, int mode, int k, const T *R, const double *theta, T *W,
                          cudaStream_t s) {
    const int64_t n = h->T.n;
    if (mode == 0) {
        if (R != W) return cudaMemcpyAsync(W, R, sizeof(T) * n * k, cudaMemcpyDeviceToDevice, s);
        return cudaSuccess;
    }
    if (mode == 1) {
        int blocks = static_cast<int>(std::min<int64_t>((n * k + 255) / 256, static_cast<int64_t>(h->num_sms) * 8));
        k_precond_diag<T><<<blocks, 256, 0, s>>>(n, k, R, theta, h->T.diag, W);
        return cudaGetLastError();
    }
    if (mode == 2) {
        if (!h->bj_Q) return cudaErrorInvalidValue;
        const int64_t nt = (n + BJ - 1) / BJ;
        const size_t smem = sizeof(float) * (BJ * BJ + 2 * BJ * k);
        cudaError_t e = cudaFuncSetAttribute(k_bjacobi_apply<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_bjacobi_apply<T><<<static_cast<unsigned>(nt), 256, smem, s>>>(n, k, h->bj_Q, h->bj_lam, R, theta, W);
        return cudaGetLastError();
    }
    if (mode == 3) {
        if constexpr (std::is_same<T, float>::value) {
            if (!h->mlp.ready) return cudaErrorInvalidValue;
            return mlp_apply(const_cast<lobpcg_ctx *>(h), k, R, theta, W, s);
        }
    }
    if (mode == 4) return fom_apply<T>(h, k, R, theta, W, s);
    return cudaErrorInvalidValue;
}

template cudaError_t precond_apply<float>(const lobpcg_ctx *, int, int, const float *, const double *, float *,
                                          cudaStream_t);
template cudaError_t precond_apply<double>(const lobpcg_ctx *, int, int, const double *, const double *, double *,
                                           cudaStream_t);

}  // namespace lobpcg
