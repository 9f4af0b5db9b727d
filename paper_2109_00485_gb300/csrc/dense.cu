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
//   k_combine_reg  the same for float32 and k in {8, 16, 20}, C in registers
//                the inputs (eqs. xupd, pupd, upd1, upd2; W <- W - X B;
//                W <- W R^{-1}), in place by rows
//
// The one-CTA FP64 kernels on the k x k / 3k x 3k matrices (Cholesky-QR
// factor, Rayleigh-Ritz solve) are in small.cu.
//
// Blocks are row-major (row i: k contiguous entries).  T is float (the FP32
// iteration) or double (the FP64 refinement); Gram accumulation is FP64 for
// both, small matrices are always FP64.
#include <cstdint>
#include <cstdlib>
#include <cstring>
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
// a thread keeps one column.  norms[j] += ||r_j||^2, norms[k + j] += ||x_j||^2
// (each thread sums its share in T, then FP64 across threads).
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
    T rr = T(0), xx = T(0);
    const T th = static_cast<T>(theta[j]);
    const T delta = static_cast<T>(1e-3) * (fabs(th) > T(1) ? fabs(th) : T(1));
    if (active) {
        const int64_t stride = static_cast<int64_t>(gridDim.x) * per;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * per + threadIdx.x / k; i < n; i += stride) {
            const int64_t e = i * k + j;
            const T x = X[e];
            const T r = HX[e] - x * th;
            rr = fma(r, r, rr);
            xx = fma(x, x, xx);
            T w = r;
            if (mode == 1) {
                const T t = static_cast<T>(d[i]) - th;   // guarded shifted pivot g(t)
                const T g = (t >= T(0)) ? (t > delta ? t : delta) : (-t > delta ? t : -delta);
                w = r / g;
            }
            W[e] = w;
        }
        atomicAdd(&red[j], static_cast<double>(rr));
        atomicAdd(&red[k + j], static_cast<double>(xx));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) atomicAdd(&norms[q], red[q]);
}

// Residual of the mixed-precision refinement: X, HX float64, W float32.
// r = HX - x theta and the norms in float64 (the cancellation happens here);
// W = r (mode 0) or r / g(d - theta) (mode 1) rounded to float32: W is a
// search direction and needs no more.  R32 (may be NULL) = float32(r).
__global__ void k_resid_mixed(int64_t n, int k, const double *X, const double *HX, const double *theta,
                              const float *d, float *W, float *R32, int mode, double *norms) {
    extern __shared__ double red[];   // [2k]
    const int per = blockDim.x / k;
    const int j = threadIdx.x % k;
    const bool active = threadIdx.x < per * k;
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) red[q] = 0.0;
    __syncthreads();
    double rr = 0.0, xx = 0.0;
    const double th = theta[j];
    const float thf = static_cast<float>(th);
    const float delta = 1e-3f * fmaxf(1.f, fabsf(thf));
    if (active) {
        const int64_t stride = static_cast<int64_t>(gridDim.x) * per;
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * per + threadIdx.x / k; i < n; i += stride) {
            const int64_t e = i * k + j;
            const double x = X[e];
            const double r = fma(-x, th, HX[e]);
            rr = fma(r, r, rr);
            xx = fma(x, x, xx);
            float w = static_cast<float>(r);
            if (R32) R32[e] = w;
            if (mode == 1) {
                const float t = static_cast<float>(static_cast<double>(d[i]) - th);
                const float g = (t >= 0.f) ? fmaxf(t, delta) : -fmaxf(-t, delta);
                w = w / g;
            }
            W[e] = w;
        }
        atomicAdd(&red[j], rr);
        atomicAdd(&red[k + j], xx);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) atomicAdd(&norms[q], red[q]);
}

// Z (n x k, float64, in place) <- Z C + A, C k x k float64 row-major, A
// float32 n x k; Z32 = float32(Z).  The X and HX updates of the mixed
// refinement: Z C carries the converged part in float64, A = [W P] C_23
// (the new P, or HP) the float32 correction.
__global__ void k_xupdate(int64_t n, int k, double *Z, const double *C, const float *A, float *Z32) {
    extern __shared__ double sx[];    // C (k x k), then `per` rows of Z
    double *sC = sx, *sZ = sx + k * k;
    const int per = blockDim.x / k;
    const int r = threadIdx.x / k, j = threadIdx.x % k;
    const bool active = threadIdx.x < per * k;
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) sC[q] = C[q];
    for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * per; i0 < n; i0 += static_cast<int64_t>(gridDim.x) * per) {
        const int rows = static_cast<int>(n - i0 < per ? n - i0 : per);
        __syncthreads();
        if (active && r < rows) sZ[threadIdx.x] = Z[i0 * k + threadIdx.x];
        __syncthreads();
        if (active && r < rows) {
            double acc = 0.0;
            for (int l = 0; l < k; ++l) acc = fma(sZ[r * k + l], sC[l * k + j], acc);
            const int64_t e = (i0 + r) * k + j;
            acc += static_cast<double>(A[e]);
            Z[e] = acc;
            Z32[e] = static_cast<float>(acc);
        }
    }
}

// ---------------------------------------------------------------- Gram

constexpr int GR_ROWS = 64;     // rows staged per pass
constexpr int GR_THREADS = 256; // 16 x 16 thread grid over the output

// Copy rows [r0, r0 + rows) of an n x k block (one contiguous run of rows*k
// values) into shared memory, zero-filling up to nrows rows; 16-byte vector
// loads when k*sizeof(T) is a multiple of 16.
template <typename T>
__device__ __forceinline__ void stage_rows(T *dst, const T *src, int64_t r0, int rows, int nrows, int k) {
    const int total = nrows * k, valid = rows * k;
    constexpr int V = 16 / sizeof(T);
    const T *s0 = src + r0 * k;
    if ((k % V) == 0 && (reinterpret_cast<uintptr_t>(s0) & 15u) == 0) {
        for (int e = threadIdx.x * V; e < total; e += blockDim.x * V) {
            if (e < valid) {
                *reinterpret_cast<float4 *>(dst + e) = __ldg(reinterpret_cast<const float4 *>(s0 + e));
            } else {
#pragma unroll
                for (int q = 0; q < V; ++q) dst[e + q] = T(0);
            }
        }
    } else {
        for (int e = threadIdx.x; e < total; e += blockDim.x) dst[e] = (e < valid) ? s0[e] : T(0);
    }
}

// M (ma x mb, FP64, row-major, pre-zeroed) += A^T B.  A = [A_0..A_{na-1}],
// B = [B_0..B_{nb-1}], each block n x k, staged per block (tile of GR_ROWS
// rows, row stride k).  Thread (tx, ty) owns the outputs (tx + 16u, ty + 16v),
// u < UA, v < UB.  Products are summed in T over one staged tile, then added
// to FP64 accumulators.
template <typename T, int UA, int UB>
__global__ void __launch_bounds__(GR_THREADS) k_gram(int64_t n, int k, int na, GemmBlocks<T> a, int nb,
                                                     GemmBlocks<T> b, double *M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ma = na * k, mb = nb * k;
    T *sa = reinterpret_cast<T *>(smem_raw);   // na tiles [GR_ROWS][k]
    T *sb = sa + na * GR_ROWS * k;             // nb tiles [GR_ROWS][k]
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    // per-output base pointers into the staged tiles
    const T *pa[UA];
    const T *pb[UB];
#pragma unroll
    for (int u = 0; u < UA; ++u) {
        const int ia = min(tx + 16 * u, ma - 1);
        pa[u] = sa + (ia / k) * GR_ROWS * k + ia % k;
    }
#pragma unroll
    for (int v = 0; v < UB; ++v) {
        const int ib = min(ty + 16 * v, mb - 1);
        pb[v] = sb + (ib / k) * GR_ROWS * k + ib % k;
    }
    // Accumulation across tiles in T with Kahan compensation (cheap FP32 adds;
    // the FP64 pipe is reserved for the final reduction across blocks).
    T acc[UA][UB], cmp[UA][UB];
#pragma unroll
    for (int u = 0; u < UA; ++u)
#pragma unroll
        for (int v = 0; v < UB; ++v) acc[u][v] = cmp[u][v] = T(0);
    const int64_t ntile = (n + GR_ROWS - 1) / GR_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t r0 = tile * GR_ROWS;
        const int rows = static_cast<int>(n - r0 < GR_ROWS ? n - r0 : GR_ROWS);
        __syncthreads();
        for (int q = 0; q < na; ++q) stage_rows<T>(sa + q * GR_ROWS * k, a.p[q], r0, rows, GR_ROWS, k);
        for (int q = 0; q < nb; ++q) stage_rows<T>(sb + q * GR_ROWS * k, b.p[q], r0, rows, GR_ROWS, k);
        __syncthreads();
        T part[UA][UB];
#pragma unroll
        for (int u = 0; u < UA; ++u)
#pragma unroll
            for (int v = 0; v < UB; ++v) part[u][v] = T(0);
        for (int r = 0; r < rows; ++r) {
            T av[UA], bv[UB];
#pragma unroll
            for (int u = 0; u < UA; ++u) av[u] = pa[u][r * k];
#pragma unroll
            for (int v = 0; v < UB; ++v) bv[v] = pb[v][r * k];
#pragma unroll
            for (int u = 0; u < UA; ++u)
#pragma unroll
                for (int v = 0; v < UB; ++v) part[u][v] = fma(av[u], bv[v], part[u][v]);
        }
#pragma unroll
        for (int u = 0; u < UA; ++u)
#pragma unroll
            for (int v = 0; v < UB; ++v) {
                const T y = part[u][v] - cmp[u][v];
                const T t = acc[u][v] + y;
                cmp[u][v] = (t - acc[u][v]) - y;
                acc[u][v] = t;
            }
    }
#pragma unroll
    for (int u = 0; u < UA; ++u)
#pragma unroll
        for (int v = 0; v < UB; ++v) {
            const int ia = tx + 16 * u, ib = ty + 16 * v;
            if (ia < ma && ib < mb)
                atomicAdd(&M[ia * mb + ib], static_cast<double>(acc[u][v]) - static_cast<double>(cmp[u][v]));
        }
}

// ---------------------------------------------------------------- Gram on the tensor cores

// M (ma x mb) += A^T B for float32 blocks with k % 4 == 0, ma <= 96,
// mb <= 192, on the tensor cores: mma.sync m16n8k8 TF32 with the 3-term
// split a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (FP32-level products).
// A CTA stages 64-row tiles of [A_0..] and [B_0..] side by side in shared
// memory (cp.async, two stages; row strides = 24 mod 32 words, so fragment
// loads are free of bank conflicts).  Warp w owns output M-tile w % MT and
// N-tiles w / MT + WN t; each 64-row tile's products start from zero and are
// added to Kahan-compensated FP32 sums, FP64 across CTAs (as k_gram).
constexpr int GT_ROWS = 64;

__device__ __forceinline__ int gt_stride(int cols) {   // >= cols, = 24 (mod 32)
    int s = cols + ((24 - cols % 32) + 32) % 32;
    return s;
}

// Split x = hi + lo (two ALU operations): hi = x with its 13 low mantissa
// bits cleared (a TF32 value), lo = x - hi, exact in FP32 and handed to the
// tensor core as it is (the TF32 operand read ignores its low 13 bits, a
// relative error below 2^-10 |lo| < 2^-20 |x|).  Each split product
// a_hi b_hi + a_hi b_lo + a_lo b_hi then errs by less than 3 * 2^-20.
__device__ __forceinline__ void gt_split(float x, uint32_t &hi, uint32_t &lo) {
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}
__device__ __forceinline__ void gt_mma(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                       uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void gt_cp16(void *dst, const void *src, bool valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const int sz = valid ? 16 : 0;   // 0: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(sz) : "memory");
}

__device__ __forceinline__ void gt_cp16s(uint32_t dst, const void *src, bool valid) {
    const int sz = valid ? 16 : 0;   // 0: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(sz) : "memory");
}

// Copy rows [r0, r0 + 64) of every block into stage `stA_off`/`stB_off`
// (float offsets of the stage's A and B regions); rows past n are zeroed.
__device__ __forceinline__ void gt_stage(const float *const *bp, const int *bcol, int nblk, int na, int SA, int SB,
                                         int stA_off, int stB_off, uint32_t sbase, int64_t n, int64_t r0, int k,
                                         int kv, int r_start, int c_start, int dr, int dc) {
    for (int q = 0; q < nblk; ++q) {
        const float *src0 = bp[q];
        const bool isA = q < na;
        const int S = isA ? SA : SB;
        const uint32_t dst0 = sbase + 4u * static_cast<uint32_t>(bcol[q] + (isA ? stA_off : stB_off));
        int r = r_start, c4 = c_start;
        while (r < GT_ROWS) {
            const int64_t row = r0 + r;
            const bool valid = row < n;
            gt_cp16s(dst0 + 4u * static_cast<uint32_t>(r * S + 4 * c4), src0 + (valid ? row : 0) * k + 4 * c4,
                     valid);
            r += dr;
            c4 += dc;
            if (c4 >= kv) {
                c4 -= kv;
                ++r;
            }
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// GT_TPW: most N-tiles per warp (1, 2, 4 or 8)
template <int GT_TPW>
__global__ void __launch_bounds__(384) k_gram_tc(int64_t n, int k, int na, GemmBlocks<float> a, int nb,
                                                 GemmBlocks<float> b, double *M, int MT, int NT, int WN) {
    extern __shared__ __align__(16) float gsm[];
    const int ma = na * k, mb = nb * k;
    const int SA = gt_stride(16 * MT), SB = gt_stride(8 * NT);
    float *const stA0 = gsm, *const stB0 = gsm + 2 * GT_ROWS * SA;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int mi = warp % MT, nj0 = warp / MT;
    // block pointers and their shared-memory destinations (column offsets)
    __shared__ const float *bp[12];
    __shared__ int bcol[12];
    if (threadIdx.x < na + nb) {
        const int q = threadIdx.x;
        bp[q] = q < na ? a.p[q] : b.p[q - na];
        bcol[q] = q < na ? q * k : 2 * GT_ROWS * SA + (q - na) * k;   // offset from gsm (stage 0)
    }
    // zero the padding columns of both stages once (cp.async never writes them)
    for (int e = threadIdx.x; e < 2 * GT_ROWS * (SA - ma); e += blockDim.x) {
        const int st = e / (GT_ROWS * (SA - ma)), q = e % (GT_ROWS * (SA - ma));
        stA0[st * GT_ROWS * SA + (q / (SA - ma)) * SA + ma + q % (SA - ma)] = 0.f;
    }
    for (int e = threadIdx.x; e < 2 * GT_ROWS * (SB - mb); e += blockDim.x) {
        const int st = e / (GT_ROWS * (SB - mb)), q = e % (GT_ROWS * (SB - mb));
        stB0[st * GT_ROWS * SB + (q / (SB - mb)) * SB + mb + q % (SB - mb)] = 0.f;
    }
    __syncthreads();
    const int kv = k / 4;   // 16-byte pieces per row of a block
    // this thread's first (row, piece) of a block tile and the stride of the
    // walk (no divisions inside the copy loops)
    const int r_start = threadIdx.x / kv, c_start = threadIdx.x % kv;
    const int dr = blockDim.x / kv, dc = blockDim.x % kv;
    const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(gsm));
    float sum[GT_TPW][4], cmp[GT_TPW][4];
#pragma unroll
    for (int u = 0; u < GT_TPW; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) sum[u][c] = cmp[u][c] = 0.f;
    const int64_t ntile = (n + GT_ROWS - 1) / GT_ROWS;
    const int nblk = na + nb;
    int64_t tile = blockIdx.x;
    if (tile < ntile)
        gt_stage(bp, bcol, nblk, na, SA, SB, 0, 0, sbase, n, tile * GT_ROWS, k, kv, r_start, c_start, dr, dc);
    int cur = 0;
    for (; tile < ntile; tile += gridDim.x) {
        const int64_t nxt = tile + gridDim.x;
        if (nxt < ntile) {
            gt_stage(bp, bcol, nblk, na, SA, SB, (cur ^ 1) * GT_ROWS * SA, (cur ^ 1) * GT_ROWS * SB, sbase, n,
                     nxt * GT_ROWS, k, kv, r_start, c_start, dr, dc);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const float *sA = stA0 + cur * GT_ROWS * SA, *sB = stB0 + cur * GT_ROWS * SB;
        float part[GT_TPW][4];
#pragma unroll
        for (int u = 0; u < GT_TPW; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c) part[u][c] = 0.f;
#pragma unroll 2
        for (int ks = 0; ks < GT_ROWS / 8; ++ks) {
            // A fragment of (A^T)[16 mi + .., 8 ks + ..]: element (m, kk) = sA[kk][16 mi + m]
            const float *pa = sA + (8 * ks + t) * SA + 16 * mi + g;
            uint32_t ah0, al0, ah1, al1, ah2, al2, ah3, al3;
            gt_split(pa[0], ah0, al0);
            gt_split(pa[8], ah1, al1);
            gt_split(pa[4 * SA], ah2, al2);
            gt_split(pa[4 * SA + 8], ah3, al3);
#pragma unroll
            for (int u = 0; u < GT_TPW; ++u) {
                const int nj = nj0 + WN * u;
                if (nj < NT) {
                    // B fragment: b0 = B[8 ks + t][8 nj + g], b1 = B[8 ks + t + 4][8 nj + g]
                    const float *pb = sB + (8 * ks + t) * SB + 8 * nj + g;
                    uint32_t bh0, bl0, bh1, bl1;
                    gt_split(pb[0], bh0, bl0);
                    gt_split(pb[4 * SB], bh1, bl1);
                    gt_mma(part[u], al0, al1, al2, al3, bh0, bh1);
                    gt_mma(part[u], ah0, ah1, ah2, ah3, bl0, bl1);
                    gt_mma(part[u], ah0, ah1, ah2, ah3, bh0, bh1);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < GT_TPW; ++u)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float y = part[u][c] - cmp[u][c];
                const float tt = sum[u][c] + y;
                cmp[u][c] = (tt - sum[u][c]) - y;
                sum[u][c] = tt;
            }
        __syncthreads();   // stage `cur` is refilled next
        cur ^= 1;
    }
#pragma unroll
    for (int u = 0; u < GT_TPW; ++u) {
        const int nj = nj0 + WN * u;
        if (nj >= NT) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int ia = 16 * mi + g + (c >= 2 ? 8 : 0), ib = 8 * nj + 2 * t + (c & 1);
            if (ia < ma && ib < mb)
                atomicAdd(&M[ia * mb + ib], static_cast<double>(sum[u][c]) - static_cast<double>(cmp[u][c]));
        }
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

// For up to two outputs: Z_o[i, :] = sum_c A[i, c] C_o[c - c0_o, :] over
// columns c >= c0_o of A = [A_0..A_{na-1}]; C_o is (ma - c0_o) x k FP64,
// staged transposed in T.  A is staged per block (tile of CB_ROWS rows, row
// stride k).  Thread (row, j) of a pass; blockDim is a multiple of k, so a
// thread keeps column j and sums ||z_j||^2 for the output norm_of in FP64,
// reduced per block before one global atomic per column.  Rows are staged
// before any output is written, so outputs may alias inputs.
template <typename T>
__global__ void k_combine(int64_t n, int k, int na, GemmBlocks<T> a, int nout, CombineOut<T> out,
                          double *colsq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ma = na * k;
    const int ms = ma | 1;                         // odd row stride of C^T: conflict-free column reads
    T *sa = reinterpret_cast<T *>(smem_raw);       // na tiles [CB_ROWS][k]
    T *sc = sa + na * CB_ROWS * k;                 // [2][k][ms]  (C transposed)
    double *red = reinterpret_cast<double *>(sc + 2 * k * ms + 2);   // [k]
    red = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(red) + 15) & ~uintptr_t(15));
    for (int o = 0; o < nout; ++o) {
        const int c0 = out.c0[o];
        for (int e = threadIdx.x; e < k * ma; e += blockDim.x) {
            const int j = e / ma, c = e % ma;
            sc[o * k * ms + j * ms + c] = (c >= c0) ? static_cast<T>(out.C[o][(c - c0) * k + j]) : T(0);
        }
    }
    for (int j = threadIdx.x; j < k; j += blockDim.x) red[j] = 0.0;
    const int per = blockDim.x / k;
    const int j = threadIdx.x % k, rr = threadIdx.x / k;
    const bool act = threadIdx.x < per * k;
    double nsq = 0.0;
    const int64_t ntile = (n + CB_ROWS - 1) / CB_ROWS;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const int64_t r0 = tile * CB_ROWS;
        const int rows = static_cast<int>(n - r0 < CB_ROWS ? n - r0 : CB_ROWS);
        __syncthreads();
        for (int q = 0; q < na; ++q) stage_rows<T>(sa + q * CB_ROWS * k, a.p[q], r0, rows, CB_ROWS, k);
        __syncthreads();
        if (!act) continue;
        for (int o = 0; o < nout; ++o) {
            const T *ct = sc + o * k * ms + j * ms;
            const int c0 = out.c0[o];
            for (int r = rr; r < rows; r += 2 * per) {   // two rows per thread: two independent chains
                const int r2 = r + per;
                const bool two = r2 < rows;
                T s = T(0), s2 = T(0);
                for (int q = c0 / k; q < na; ++q) {   // c0 is 0 or k
                    const T *arow = sa + q * CB_ROWS * k + r * k;
                    const T *arow2 = sa + q * CB_ROWS * k + (two ? r2 : r) * k;
                    const T *cq = ct + q * k;
                    for (int cc = 0; cc < k; ++cc) {
                        const T cv = cq[cc];
                        s = fma(arow[cc], cv, s);
                        s2 = fma(arow2[cc], cv, s2);
                    }
                }
                out.z[o][(r0 + r) * k + j] = s;
                if (o == out.norm_of) nsq += static_cast<double>(s) * static_cast<double>(s);
                if (two) {
                    out.z[o][(r0 + r2) * k + j] = s2;
                    if (o == out.norm_of) nsq += static_cast<double>(s2) * static_cast<double>(s2);
                }
            }
        }
    }
    if (colsq) {
        __syncthreads();
        if (act) atomicAdd(&red[j], nsq);
        __syncthreads();
        for (int q = threadIdx.x; q < k; q += blockDim.x) atomicAdd(&colsq[q], red[q]);
    }
}

// Float copies of the combine coefficients: Cf[0..n0) = C0, Cf[n0..n0+n1) = C1
// (row offsets as in the FP64 matrices; C1 placed after C0's full NA K x K).
__global__ void k_coef_to_float(int n0, const double *C0, const double *C1, int n1, float *Cf) {
    for (int e = threadIdx.x; e < n0; e += blockDim.x) Cf[e] = static_cast<float>(C0[e]);
    if (C1)
        for (int e = threadIdx.x; e < n1; e += blockDim.x) Cf[n0 + e] = static_cast<float>(C1[e]);
}

// float32, K in {8, 16, 20}: each thread keeps column j of both coefficient
// matrices in registers and walks rows; 64-row tiles of the NA blocks are
// staged by cp.async into two alternating buffers (the next tile loads while
// this one is combined) and read with 16-byte broadcast loads (a row group
// of K threads reads the same row).  Output 1, when present, starts at
// block 1 (c0 = K).  Column norms: float32 per thread and tile, float64
// across tiles.  Semantics as k_combine.
constexpr int CR_ROWS = 64;

template <int K, int NA>
__global__ void __launch_bounds__(128) k_combine_reg(int64_t n, GemmBlocks<float> a, int nout, CombineOut<float> out,
                                                     double *colsq) {
    __shared__ __align__(16) float sa[2][NA * CR_ROWS * K];
    __shared__ double red[K];
    constexpr int G = 128 / K;   // row groups
    constexpr int PV = CR_ROWS * K / 4;   // 16-byte pieces per block tile
    const int j = threadIdx.x % K, grp = threadIdx.x / K;
    const bool act = grp < G;
    float c0[NA * K], c1[NA * K];
#pragma unroll
    for (int c = 0; c < NA * K; ++c) {
        c0[c] = out.Cf[c * K + j];
        c1[c] = (nout > 1 && c >= K) ? out.Cf[NA * K * K + (c - K) * K + j] : 0.f;
    }
    for (int q = threadIdx.x; q < K; q += blockDim.x) red[q] = 0.0;
    auto stage = [&](int st, int64_t r0) {
#pragma unroll
        for (int q = 0; q < NA; ++q)
            for (int e = threadIdx.x; e < PV; e += blockDim.x) {
                const int r = (4 * e) / K;
                const bool valid = r0 + r < n;
                gt_cp16(&sa[st][q * CR_ROWS * K + 4 * e], a.p[q] + (valid ? r0 * K + 4 * e : 0), valid);
            }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    double nsq = 0.0;
    const int64_t ntile = (n + CR_ROWS - 1) / CR_ROWS;
    int64_t tile = blockIdx.x;
    if (tile < ntile) stage(0, tile * CR_ROWS);
    int cur = 0;
    for (; tile < ntile; tile += gridDim.x) {
        const int64_t nxt = tile + gridDim.x;
        if (nxt < ntile) {
            stage(cur ^ 1, nxt * CR_ROWS);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const int64_t r0 = tile * CR_ROWS;
        const int rows = static_cast<int>(n - r0 < CR_ROWS ? n - r0 : CR_ROWS);
        float tsq = 0.f;
        if (act) {
            for (int r = grp; r < rows; r += G) {
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int q = 0; q < NA; ++q) {
                    const float4 *ar = reinterpret_cast<const float4 *>(&sa[cur][q * CR_ROWS * K + r * K]);
#pragma unroll
                    for (int c4 = 0; c4 < K / 4; ++c4) {
                        const float4 v = ar[c4];
                        const int c = q * K + 4 * c4;
                        s0 = fmaf(v.x, c0[c], s0);
                        s0 = fmaf(v.y, c0[c + 1], s0);
                        s0 = fmaf(v.z, c0[c + 2], s0);
                        s0 = fmaf(v.w, c0[c + 3], s0);
                        if (q > 0) {
                            s1 = fmaf(v.x, c1[c], s1);
                            s1 = fmaf(v.y, c1[c + 1], s1);
                            s1 = fmaf(v.z, c1[c + 2], s1);
                            s1 = fmaf(v.w, c1[c + 3], s1);
                        }
                    }
                }
                out.z[0][(r0 + r) * K + j] = s0;
                if (out.norm_of == 0) tsq = fmaf(s0, s0, tsq);
                if (nout > 1) {
                    out.z[1][(r0 + r) * K + j] = s1;
                    if (out.norm_of == 1) tsq = fmaf(s1, s1, tsq);
                }
            }
        }
        nsq += static_cast<double>(tsq);
        __syncthreads();   // buffer `cur` is refilled next
        cur ^= 1;
    }
    if (colsq) {
        if (act) atomicAdd(&red[j], nsq);
        __syncthreads();
        for (int q = threadIdx.x; q < K; q += blockDim.x) atomicAdd(&colsq[q], red[q]);
    }
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

cudaError_t launch_resid_mixed(int64_t n, int k, const double *X, const double *HX, const double *theta,
                               const float *d, float *W, float *R32, int mode, double *norms, int num_sms,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * k, s);
    if (e != cudaSuccess) return e;
    const int threads = (256 / k) * k;
    const int64_t per = threads / k;
    int blocks = static_cast<int>(std::min<int64_t>((n + per - 1) / per, static_cast<int64_t>(num_sms) * 8));
    if (blocks < 1) blocks = 1;
    k_resid_mixed<<<blocks, threads, sizeof(double) * 2 * k, s>>>(n, k, X, HX, theta, d, W, R32, mode, norms);
    return cudaGetLastError();
}

cudaError_t launch_xupdate(int64_t n, int k, double *Z, const double *C, const float *A, float *Z32, int num_sms,
                           cudaStream_t s) {
    const int threads = (256 / k) * k;
    const int64_t per = threads / k;
    int blocks = static_cast<int>(std::min<int64_t>((n + per - 1) / per, static_cast<int64_t>(num_sms) * 8));
    if (blocks < 1) blocks = 1;
    k_xupdate<<<blocks, threads, sizeof(double) * (k * k + threads), s>>>(n, k, Z, C, A, Z32);
    return cudaGetLastError();
}

// The tensor-memory Gram (gram_umma.cu) is chosen with LOBPCG_GRAM=umma; by
// default float32 Grams use k_gram_tc, which is faster on these shapes.
static bool gram_umma_enabled() {
    static const int on = [] {
        const char *v = getenv("LOBPCG_GRAM");
        return (v && strcmp(v, "umma") == 0) ? 1 : 0;
    }();
    return on != 0;
}

// LOBPCG_GRAM=tc keeps float32 Grams on the mma.sync kernel k_gram_tc
// (for comparison); by default they go to the CUDA-core pair kernel
// (gram_ff.cu) when it takes the shape.
static bool gram_tc_forced() {
    static const int on = [] {
        const char *v = getenv("LOBPCG_GRAM");
        return (v && strcmp(v, "tc") == 0) ? 1 : 0;
    }();
    return on != 0;
}

template <typename T>
cudaError_t launch_gram(int64_t n, int k, int na, GemmBlocks<T> a, int nb, GemmBlocks<T> b, double *M, int num_sms,
                        cudaStream_t s, int *err) {
    const int ma = na * k, mb = nb * k;
    if constexpr (std::is_same<T, float>::value) {
        if (err && gram_umma_enabled() && gram_umma_ok(k, na, a.p, nb, b.p))
            return launch_gram_umma(n, k, na, a.p, nb, b.p, M, err, num_sms, s);
        if (err && !gram_tc_forced() && na * nb <= 16) {
            // every (A block, B block) pair on the CUDA-core kernel
            const float *blk[12];
            int nblk = 0;
            auto uq = [&](const float *p) {
                for (int q = 0; q < nblk; ++q)
                    if (blk[q] == p) return q;
                blk[nblk] = p;
                return nblk++;
            };
            GramPair pairs[16];
            int np = 0;
            for (int qa = 0; qa < na; ++qa)
                for (int qb = 0; qb < nb; ++qb) pairs[np++] = GramPair{uq(a.p[qa]), uq(b.p[qb]), qa, qb, 0, 0, 0};
            const int units = np * (k / 4) * (k / 4);
            if (nblk <= 8 && gram_pairs_fit(k, nblk, blk, np, units))
                return launch_gram_pairs(n, k, nblk, blk, np, pairs, M, mb, ma, true, err, num_sms, s);
        }
    }
    cudaError_t e = cudaMemsetAsync(M, 0, sizeof(double) * ma * mb, s);
    if (e != cudaSuccess) return e;
    if constexpr (std::is_same<T, float>::value) {
        bool aligned = true;
        for (int q = 0; q < na; ++q) aligned = aligned && (reinterpret_cast<uintptr_t>(a.p[q]) & 15u) == 0;
        for (int q = 0; q < nb; ++q) aligned = aligned && (reinterpret_cast<uintptr_t>(b.p[q]) & 15u) == 0;
        const int MT = (ma + 15) / 16, NT = (mb + 7) / 8;
        const int WN = std::min(NT, (MT == 5) ? 2 : std::max(1, 12 / MT));   // warps per M-tile
        const int tpw = (NT + WN - 1) / WN;
        if (k % 4 == 0 && aligned && ma <= 96 && mb <= 192 && tpw <= 8) {
            const int W = MT * WN;
            auto stride = [](int cols) { return cols + ((24 - cols % 32) + 32) % 32; };
            const size_t smem = sizeof(float) * 2 * GT_ROWS * (stride(16 * MT) + stride(8 * NT));
            static bool attr = false;
            if (!attr) {
                e = cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(k_gram_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(k_gram_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(k_gram_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
                if (e != cudaSuccess) return e;
                attr = true;
            }
            const int64_t ntile = (n + GT_ROWS - 1) / GT_ROWS;
            // CTAs per SM: as many as shared memory allows, up to 4
            const int per_sm = std::max(1, std::min<int>(4, static_cast<int>((200 * 1024) / smem)));
            int blocks = static_cast<int>(std::min<int64_t>(ntile, static_cast<int64_t>(num_sms) * per_sm));
            if (blocks < 1) blocks = 1;
            if (tpw == 1) k_gram_tc<1><<<blocks, W * 32, smem, s>>>(n, k, na, a, nb, b, M, MT, NT, WN);
            else if (tpw == 2) k_gram_tc<2><<<blocks, W * 32, smem, s>>>(n, k, na, a, nb, b, M, MT, NT, WN);
            else if (tpw <= 4) k_gram_tc<4><<<blocks, W * 32, smem, s>>>(n, k, na, a, nb, b, M, MT, NT, WN);
            else k_gram_tc<8><<<blocks, W * 32, smem, s>>>(n, k, na, a, nb, b, M, MT, NT, WN);
            return cudaGetLastError();
        }
    }
    const size_t smem = sizeof(T) * GR_ROWS * (ma + mb);
    const int64_t ntile = (n + GR_ROWS - 1) / GR_ROWS;   // one tile per block pass
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
    GRAM_CASE(1, 2)
    GRAM_CASE(2, 2)
    GRAM_CASE(2, 4)
    GRAM_CASE(3, 3)
    GRAM_CASE(3, 6)
    GRAM_CASE(4, 4)
    GRAM_CASE(4, 8)
    GRAM_CASE(6, 6)
    GRAM_CASE(6, 12)
#undef GRAM_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_combine(int64_t n, int k, int na, GemmBlocks<T> a, int nout, CombineOut<T> out, double *colsq,
                           int num_sms, cudaStream_t s) {
    cudaError_t e;
    if (colsq) {
        e = cudaMemsetAsync(colsq, 0, sizeof(double) * k, s);
        if (e != cudaSuccess) return e;
    }
    const int64_t ntile = (n + CB_ROWS - 1) / CB_ROWS;
    if constexpr (std::is_same<T, float>::value) {
        // one output from all inputs, no norms: the bulk-copy kernel (update.cu)
        if (nout == 1 && out.c0[0] == 0 && out.err && (out.norm_of != 0 || !colsq) &&
            combine_ff_ok(k, na, a.p, out.z[0]))
            return launch_combine_ff(n, k, na, a.p, out.C[0], out.z[0], out.err, num_sms, s);
        const bool reg_ok = (nout == 1 || out.c0[1] == k) && out.c0[0] == 0 && out.Cf != nullptr;
        int blocks = static_cast<int>(std::min<int64_t>(ntile, static_cast<int64_t>(num_sms) * 8));
        if (blocks < 1) blocks = 1;
#define COMBINE_REG(KK, NN)                                                                              \
        if (reg_ok && k == KK && na == NN) {                                                             \
            k_coef_to_float<<<1, 256, 0, s>>>(NN * KK * KK, out.C[0], nout > 1 ? out.C[1] : nullptr,   \
                                               (NN - 1) * KK * KK, out.Cf);                              \
            k_combine_reg<KK, NN><<<blocks, 128, 0, s>>>(n, a, nout, out, colsq);                        \
            return cudaGetLastError();                                                                   \
        }
        COMBINE_REG(8, 1) COMBINE_REG(8, 2) COMBINE_REG(8, 3)
        COMBINE_REG(16, 1) COMBINE_REG(16, 2) COMBINE_REG(16, 3)
        COMBINE_REG(20, 1) COMBINE_REG(20, 2) COMBINE_REG(20, 3)
#undef COMBINE_REG
    }
    const int ms = (na * k) | 1;
    const size_t smem = sizeof(T) * (na * CB_ROWS * k + 2 * ms * k + 2) + sizeof(double) * (k + 2);
    e = cudaFuncSetAttribute(k_combine<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks = static_cast<int>(std::min<int64_t>(ntile, static_cast<int64_t>(num_sms) * 4));
    if (blocks < 1) blocks = 1;
    const int threads = (256 / k) * k;
    k_combine<T><<<blocks, threads, smem, s>>>(n, k, na, a, nout, out, colsq);
    return cudaGetLastError();
}

template cudaError_t launch_resid<float>(int64_t, int, const float *, const float *, const double *, const float *,
                                         float *, int, double *, int, cudaStream_t);
template cudaError_t launch_resid<double>(int64_t, int, const double *, const double *, const double *,
                                          const float *, double *, int, double *, int, cudaStream_t);
template cudaError_t launch_gram<float>(int64_t, int, int, GemmBlocks<float>, int, GemmBlocks<float>, double *, int,
                                        cudaStream_t, int *);
template cudaError_t launch_gram<double>(int64_t, int, int, GemmBlocks<double>, int, GemmBlocks<double>, double *,
                                         int, cudaStream_t, int *);
template cudaError_t launch_combine<float>(int64_t, int, int, GemmBlocks<float>, int, CombineOut<float>, double *,
                                           int, cudaStream_t);
template cudaError_t launch_combine<double>(int64_t, int, int, GemmBlocks<double>, int, CombineOut<double>,
                                            double *, int, cudaStream_t);

}  // namespace lobpcg
