// Dense steps of the float64 refinement in compensated float32 (df.cuh):
//
//   k_xupdate_df   Z <- Z C + A (Z n x k float64 in place, C k x k float64,
//                  A n x k float32) and Z32 = float32(Z): the X and HX
//                  updates of the refinement
//   k_gram_x_df    G = X^T [HX X] (k x 2k float64) from float64 X and HX:
//                  the Gram blocks the refinement keeps in float64
//
// Each float64 input is split into a float pair on its bit pattern, the
// products summed with error-free transformations in float32 (relative
// error of a few 2^-47 per term), and only the results touch the FP64
// pipe: one float64 addition per output of the update, and per Gram entry
// two every 64 rows (the fold of a float pair into a float64 sum).
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "df.cuh"
#include "dense.h"

namespace lobpcg {

namespace {

constexpr int XU_THREADS = 256;

// thread (row r of the pass, column j); C split once per CTA, the pass's
// rows of Z split once into shared memory
__global__ void __launch_bounds__(XU_THREADS) k_xupdate_df(int64_t n, int k, double *Z, const double *C,
                                                           const float *A, float *Z32) {
    extern __shared__ float xs[];   // ch, cl (k x k each), zh, zl (per x k each)
    const int per = XU_THREADS / k;
    float *ch = xs, *cl = xs + k * k, *zh = xs + 2 * k * k, *zl = zh + per * k;
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) df_split(C[q], ch[q], cl[q]);
    const int r = threadIdx.x / k, j = threadIdx.x % k;
    const bool active = r < per;
    for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * per; i0 < n; i0 += static_cast<int64_t>(gridDim.x) * per) {
        const int rows = static_cast<int>(n - i0 < per ? n - i0 : per);
        __syncthreads();
        if (threadIdx.x < rows * k) df_split(Z[i0 * k + threadIdx.x], zh[threadIdx.x], zl[threadIdx.x]);
        __syncthreads();
        if (active && r < rows) {
            float s = 0.f, c = 0.f;
            for (int l = 0; l < k; ++l) df_mac(zh[r * k + l], zl[r * k + l], ch[l * k + j], cl[l * k + j], s, c);
            const int64_t e = (i0 + r) * k + j;
            // s + a = u + v exactly (TwoSum), then one float64 addition
            const float a = A[e];
            const float u = __fadd_rn(s, a);
            const float ba = __fsub_rn(u, s);
            const float v = __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(u, ba)), __fsub_rn(a, ba)), c);
            Z[e] = df_to_f64(u) + df_to_f64(v);
            Z32[e] = __fadd_rn(u, v);
        }
    }
}

constexpr int GX_THREADS = 256;
constexpr int GX_ROWS = 64;     // rows staged per pass (and folded into float64 per pass)
constexpr int GX_MAXE = 8;      // entries per thread: 2 k^2 <= 8 * 256 (k <= 32)

// G[i][j] = sum_r X[r][i] B[r][j], B = [HX X]: thread t owns entries
// t + 256 q; the CTA's rows in passes of 64, split into shared memory
__global__ void __launch_bounds__(GX_THREADS) k_gram_x_df(int64_t n, int k, const double *X, const double *HX,
                                                          double *G) {
    extern __shared__ float gs[];   // xh, xl, yh, yl: GX_ROWS x k each (y = HX rows)
    float *xh = gs, *xl = gs + GX_ROWS * k, *yh = gs + 2 * GX_ROWS * k, *yl = gs + 3 * GX_ROWS * k;
    const int ne = 2 * k * k;
    double acc[GX_MAXE];
    float s[GX_MAXE], c[GX_MAXE];
#pragma unroll
    for (int q = 0; q < GX_MAXE; ++q) {
        acc[q] = 0.0;
        s[q] = c[q] = 0.f;
    }
    const int64_t per_cta = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * per_cta;
    const int64_t r1 = std::min<int64_t>(n, r0 + per_cta);
    for (int64_t a = r0; a < r1; a += GX_ROWS) {
        const int rows = static_cast<int>(std::min<int64_t>(GX_ROWS, r1 - a));
        __syncthreads();
        for (int q = threadIdx.x; q < rows * k; q += blockDim.x) {
            df_split(X[a * k + q], xh[q], xl[q]);
            df_split(HX[a * k + q], yh[q], yl[q]);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GX_MAXE; ++q) {
            const int en = threadIdx.x + GX_THREADS * q;
            if (en < ne) {
                const int i = en / (2 * k), jj = en % (2 * k);
                const bool hxcol = jj < k;
                const int j = hxcol ? jj : jj - k;
                const float *bh = hxcol ? yh : xh, *bl = hxcol ? yl : xl;
                for (int r = 0; r < rows; ++r)
                    df_mac(xh[r * k + i], xl[r * k + i], bh[r * k + j], bl[r * k + j], s[q], c[q]);
                acc[q] += df_to_f64(s[q]) + df_to_f64(c[q]);
                s[q] = c[q] = 0.f;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < GX_MAXE; ++q) {
        const int en = threadIdx.x + GX_THREADS * q;
        if (en < ne && r0 < r1) atomicAdd(&G[en], acc[q]);
    }
}

}  // namespace

bool mixed_df_ok(int k) { return k >= 1 && k <= 32; }

cudaError_t launch_xupdate_df(int64_t n, int k, double *Z, const double *C, const float *A, float *Z32, int num_sms,
                              cudaStream_t s) {
    if (!mixed_df_ok(k)) return cudaErrorInvalidValue;
    const int per = XU_THREADS / k;
    const size_t smem = sizeof(float) * (2 * k * k + 2 * per * k);
    int blocks = static_cast<int>(std::min<int64_t>((n + per - 1) / per, static_cast<int64_t>(num_sms) * 8));
    if (blocks < 1) blocks = 1;
    k_xupdate_df<<<blocks, XU_THREADS, smem, s>>>(n, k, Z, C, A, Z32);
    return cudaGetLastError();
}

cudaError_t launch_gram_x_df(int64_t n, int k, const double *X, const double *HX, double *G, int num_sms,
                             cudaStream_t s) {
    if (!mixed_df_ok(k)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * 2 * k * k, s);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(float) * 4 * GX_ROWS * k;
    int blocks = static_cast<int>(std::min<int64_t>((n + GX_ROWS - 1) / GX_ROWS, static_cast<int64_t>(num_sms) * 2));
    if (blocks < 1) blocks = 1;
    k_gram_x_df<<<blocks, GX_THREADS, smem, s>>>(n, k, X, HX, G);
    return cudaGetLastError();
}

}  // namespace lobpcg
