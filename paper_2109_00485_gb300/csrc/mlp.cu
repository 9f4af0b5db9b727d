// Learned tile preconditioner (not in the paper): one small network shared
// by every 64-row diagonal tile stands in for the exact shifted tile solve
// (H_T - theta_j I)^{-1} r_T of the block-Jacobi form of K (Section 3.3), as
// a correction to the diagonal (1x1-tile) solve D_theta^{-1} r_T:
//
//   x = [ r_T / s , (d_T - theta) / g , theta / g ]  (129, padded to 144)
//   h = relu(W1 x + b1) (256),  y = W2 h + b2 (64)
//   w_T = D_theta^{-1} r_T + (s / g) y
//   s = ||r_T||, g = ||H||_G; target t = clip(g (y_T - D_theta^{-1} r_T) / s, +-1e3)
//
// The output layer starts at zero, so the untrained form is the diagonal one.
//
// All products run on the tensor cores (mma.sync m16n8k16, BF16 operands
// rounded from the FP32 master weights and activations, FP32 accumulation).
// Training: mean squared error, Adam, on pairs harvested from the solver's
// own block-Jacobi iterations.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include "common.cuh"
#include "internal.h"
#include "mlp.h"

namespace lobpcg {

// ------------------------------------------------------------------ GEMM

// C (M x N, fp32, ldc) = op(A) op(B) (+ bias[N]) (relu) (+= C if accumulate)
//   A: a_trans ? stored K x M (row-major, lda) : stored M x K (lda)
//   B: b_nk    ? stored N x K (row-major, ldb) : stored K x N (ldb)
// Tiles of 64 x 64 per CTA (4 warps, 32 x 32 each), K in steps of 32,
// operands rounded to bf16 while staged in shared memory.
struct GemmArgs {
    int M, N, K;
    const float *A;
    int lda;
    int a_trans;
    const float *B;
    int ldb;
    int b_nk;
    float *C;
    int ldc;
    const float *bias;
    int relu;
    int ksplit = 1;              // CTAs along K: each adds its partial product into C (zeroed first)
};

constexpr int GT = 64, GK = 32, GPAD = 8;

__device__ __forceinline__ uint32_t ld_bf16x2(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[GT][GK + GPAD];   // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[GT][GK + GPAD];   // [n][k]
    const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
    // this CTA's K range (split-K: blockIdx.z of ksplit, in GK steps)
    const int ksteps = (g.K + GK - 1) / GK, per = (ksteps + g.ksplit - 1) / g.ksplit;
    const int kbeg = blockIdx.z * per * GK, kend = min(g.K, (blockIdx.z + 1) * per * GK);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += GK) {
        __syncthreads();
        for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
            int mm, kk;
            if (g.a_trans) { kk = e / GT; mm = e % GT; }   // coalesced along M
            else { mm = e / GK; kk = e % GK; }            // coalesced along K
            const int gm = m0 + mm, gk = k0 + kk;
            float v = 0.f;
            if (gm < g.M && gk < kend) v = g.a_trans ? g.A[static_cast<int64_t>(gk) * g.lda + gm]
                                                    : g.A[static_cast<int64_t>(gm) * g.lda + gk];
            As[mm][kk] = __float2bfloat16_rn(v);
        }
        for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
            int nn, kk;
            if (g.b_nk) { nn = e / GK; kk = e % GK; }
            else { kk = e / GT; nn = e % GT; }
            const int gn = n0 + nn, gk = k0 + kk;
            float v = 0.f;
            if (gn < g.N && gk < kend) v = g.b_nk ? g.B[static_cast<int64_t>(gn) * g.ldb + gk]
                                                 : g.B[static_cast<int64_t>(gk) * g.ldb + gn];
            Bs[nn][kk] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < GK; ks += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int r = wm + 16 * a + gq;
                af[a][0] = ld_bf16x2(&As[r][ks + 2 * tq]);
                af[a][1] = ld_bf16x2(&As[r + 8][ks + 2 * tq]);
                af[a][2] = ld_bf16x2(&As[r][ks + 2 * tq + 8]);
                af[a][3] = ld_bf16x2(&As[r + 8][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int c = wn + 8 * b + gq;
                bf[b][0] = ld_bf16x2(&Bs[c][ks + 2 * tq]);
                bf[b][1] = ld_bf16x2(&Bs[c][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) mma_bf16(acc[a][b], af[a][0], af[a][1], af[a][2], af[a][3], bf[b][0], bf[b][1]);
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int r = m0 + wm + 16 * a + gq + (c >= 2 ? 8 : 0);
                const int col = n0 + wn + 8 * b + 2 * tq + (c & 1);
                if (r < g.M && col < g.N) {
                    float v = acc[a][b][c];
                    if (g.ksplit > 1) {
                        atomicAdd(&g.C[static_cast<int64_t>(r) * g.ldc + col], v);
                    } else {
                        if (g.bias) v += g.bias[col];
                        if (g.relu) v = fmaxf(v, 0.f);
                        g.C[static_cast<int64_t>(r) * g.ldc + col] = v;
                    }
                }
            }
}

static cudaError_t gemm(const GemmArgs &g0, cudaStream_t s, int num_sms = 0) {
    GemmArgs g = g0;
    const int tiles = ((g.N + GT - 1) / GT) * ((g.M + GT - 1) / GT);
    // a long reduction (the weight gradients: K = batch rows) over few output
    // tiles is split along K so that about two CTAs per SM run it
    g.ksplit = 1;
    if (num_sms > 0 && !g.bias && !g.relu && tiles < num_sms) {
        const int ksteps = (g.K + GT - 1) / GT;
        g.ksplit = std::max(1, std::min(ksteps / 2, (2 * num_sms + tiles - 1) / tiles));
    }
    if (g.ksplit > 1) {   // C is accumulated into: zero it (rows of N floats, stride ldc)
        const cudaError_t e = cudaMemset2DAsync(g.C, sizeof(float) * g.ldc, 0, sizeof(float) * g.N, g.M, s);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((g.N + GT - 1) / GT, (g.M + GT - 1) / GT, g.ksplit);
    k_gemm_bf16<<<grid, 128, 0, s>>>(g);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ pieces

// Diagonal solve r / g(d - theta) with the guarded pivot
// g(t) = sign(t) max(|t|, 1e-3 max(1, |theta|)); the shift is formed in FP64.
__device__ __forceinline__ float diag_solve(float r, float d, double th) {
    const float t = static_cast<float>(static_cast<double>(d) - th);
    const float delta = 1e-3f * fmaxf(1.f, fabsf(static_cast<float>(th)));
    const float g = (t >= 0.f) ? fmaxf(t, delta) : -fmaxf(-t, delta);
    return r / g;
}

// ------------------------------------------------------------------ fused apply

// The whole apply W = D^{-1} R + c in one kernel, in batches of 64 / k
// whole tiles (at most 64 (tile, column) pairs), the network's weights
// resident in shared memory as bf16 (one CTA per SM): a batch's rows of R
// and d are read coalesced into shared memory, the pairs' inputs built there,
// h = relu(W1 x + b1) and y = W2 h + b2 on the tensor cores (mma.sync
// m16n8k16, FP32 accumulation, k-steps in ascending order as in
// k_gemm_bf16, h rounded to bf16 after the bias and relu as k_gemm_bf16's
// staging rounds it), and the outputs formed in shared memory and written
// back as the batch's contiguous rows of W (W may be R).  Nothing but R, d
// and W leaves the SM (an unfused form through k_gemm_bf16 wrote the
// inputs, a float32 hidden layer and the outputs to memory and read them
// back: 2.5 ms per application at n = 2M, k = 16).
//
// Inputs of pair p = t k + j: x = [r_T / s, (d_T - theta_j) / g,
// theta_j / g, 0...] (s = ||r_T||, g = ||H||_G).  Outputs: w_T = D^{-1} r_T +
// scale (s / g) y, where a non-finite correction is dropped and one whose
// norm over the tile exceeds that of the tile's diagonal solve is scaled
// down to it, so the learned form stays within a factor 2 of the diagonal
// one.
constexpr int FA_PAIRS = 64;
constexpr int FA_WARPS = 16;
constexpr int FA_THREADS = 32 * FA_WARPS;
constexpr int FA_PPW = FA_PAIRS / FA_WARPS;   // pairs a warp builds and finishes
constexpr int FA_XS = MLP_KIN + 8;    // bf16 row strides: 76 and 132 words, so the
constexpr int FA_HS = MLP_NHID + 8;   // eight rows of a fragment load fall in distinct banks

struct FaSmem {
    __nv_bfloat16 w1[MLP_NHID][FA_XS];
    __nv_bfloat16 w2[MLP_NOUT][FA_HS];
    union {                                      // x until the first layer is done, then y
        __nv_bfloat16 x[FA_PAIRS][FA_XS];
        float y[FA_PAIRS][MLP_NOUT + 4];
    } xy;
    __nv_bfloat16 hb[FA_PAIRS][FA_HS];
    float r[FA_PAIRS][MLP_TILE + 1];   // the pairs' residual entries, then their outputs (row stride 65: conflict-free)
    float d[FA_PAIRS * MLP_TILE];      // the batch's diagonal entries
    float b1[MLP_NHID], b2[MLP_NOUT];
    float sc[FA_PAIRS];
    float thf[32], thl[32];   // theta_j = thf + thl (+ 2^-48 |theta_j|), split once per CTA
};

__global__ void __launch_bounds__(FA_THREADS, 1) k_mlp_apply_fused(int64_t n, int k, const float *P, const float *R,
                                                                   const float *d, const double *theta, double normG,
                                                                   float *W) {
    extern __shared__ __align__(16) unsigned char fa_raw[];
    FaSmem &S = *reinterpret_cast<FaSmem *>(fa_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gq = lane >> 2, tq = lane & 3;
    for (int e = threadIdx.x; e < MLP_NHID * MLP_KIN; e += FA_THREADS)
        S.w1[e / MLP_KIN][e % MLP_KIN] = __float2bfloat16_rn(P[MLP_OFF_W1 + e]);
    for (int e = threadIdx.x; e < MLP_NOUT * MLP_NHID; e += FA_THREADS)
        S.w2[e / MLP_NHID][e % MLP_NHID] = __float2bfloat16_rn(P[MLP_OFF_W2 + e]);
    for (int e = threadIdx.x; e < MLP_NHID; e += FA_THREADS) S.b1[e] = P[MLP_OFF_B1 + e];
    for (int e = threadIdx.x; e < MLP_NOUT; e += FA_THREADS) S.b2[e] = P[MLP_OFF_B2 + e];
    for (int e = threadIdx.x; e < k; e += FA_THREADS) {
        const float hi = __double2float_rn(theta[e]);
        S.thf[e] = hi;
        S.thl[e] = __double2float_rn(theta[e] - static_cast<double>(hi));
    }
    // float32 constants: GB300 runs FP64 (and conversions) at 1/64 of the
    // FP32 rate, so nothing in the batch loop is float64
    const float igf = static_cast<float>(1.0 / normG);
    // A batch is T = 64 / k whole tiles (T k <= 64 pairs): its rows of R, d
    // and W are contiguous, read and written with coalesced accesses.
    const int T = FA_PAIRS / k;
    const int64_t ntiles = (n + MLP_TILE - 1) / MLP_TILE;
    for (int64_t t0 = static_cast<int64_t>(blockIdx.x) * T; t0 < ntiles; t0 += static_cast<int64_t>(gridDim.x) * T) {
        const int tb = static_cast<int>(ntiles - t0 < T ? ntiles - t0 : T);
        const int np = tb * k;                               // pairs q = tl k + j
        const int64_t r0 = t0 * MLP_TILE;
        const int rows = static_cast<int>(n - r0 < tb * MLP_TILE ? n - r0 : tb * MLP_TILE);
        __syncthreads();   // the previous batch is done with every buffer
        for (int e = threadIdx.x; e < rows * k; e += FA_THREADS) {
            const int row = e / k, j = e - row * k;
            S.r[(row >> 6) * k + j][row & 63] = R[r0 * k + e];
        }
        for (int e = threadIdx.x; e < rows; e += FA_THREADS) S.d[e] = d[r0 + e];
        __syncthreads();
        // ---- inputs: the warp's pairs (a warp per pair, two rows per lane)
#pragma unroll
        for (int i = 0; i < FA_PPW; ++i) {
            const int q = warp * FA_PPW + i;
            if (q >= np) {
                for (int c = lane; c < MLP_KIN; c += 32) S.xy.x[q][c] = __float2bfloat16_rn(0.f);
                if (lane == 0) S.sc[q] = 0.f;
                continue;
            }
            const int tl = q / k, j = q - tl * k;
            float rv[2], dv[2];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int rl = lane + 32 * hh;
                const bool ok = tl * MLP_TILE + rl < rows;
                rv[hh] = ok ? S.r[q][rl] : 0.f;
                dv[hh] = ok ? S.d[tl * MLP_TILE + rl] : 0.f;
            }
            float ss = rv[0] * rv[0] + rv[1] * rv[1];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            const float sv = sqrtf(ss);
            const float is = sv > 0.f ? 1.f / sv : 0.f;
            const float th = S.thf[j];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                S.xy.x[q][lane + 32 * hh] = __float2bfloat16_rn(rv[hh] * is);
                S.xy.x[q][MLP_TILE + lane + 32 * hh] = __float2bfloat16_rn((dv[hh] - th) * igf);
            }
            if (lane < MLP_KIN - 2 * MLP_TILE)
                S.xy.x[q][2 * MLP_TILE + lane] = __float2bfloat16_rn((lane == 0) ? th * igf : 0.f);
            if (lane == 0) S.sc[q] = sv;
        }
        __syncthreads();
        // ---- h = relu(W1 x + b1): warp w, hidden units [16 w, 16 w + 16)
        {
            float acc[4][2][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
#pragma unroll 3
            for (int ks = 0; ks < MLP_KIN; ks += 16) {
                uint32_t af[4][4], bf[2][2];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int r = 16 * a + gq;
                    af[a][0] = ld_bf16x2(&S.xy.x[r][ks + 2 * tq]);
                    af[a][1] = ld_bf16x2(&S.xy.x[r + 8][ks + 2 * tq]);
                    af[a][2] = ld_bf16x2(&S.xy.x[r][ks + 2 * tq + 8]);
                    af[a][3] = ld_bf16x2(&S.xy.x[r + 8][ks + 2 * tq + 8]);
                }
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int c = 16 * warp + 8 * b + gq;
                    bf[b][0] = ld_bf16x2(&S.w1[c][ks + 2 * tq]);
                    bf[b][1] = ld_bf16x2(&S.w1[c][ks + 2 * tq + 8]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b)
                        mma_bf16(acc[a][b], af[a][0], af[a][1], af[a][2], af[a][3], bf[b][0], bf[b][1]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int r = 16 * a + gq + (c >= 2 ? 8 : 0);
                        const int col = 16 * warp + 8 * b + 2 * tq + (c & 1);
                        S.hb[r][col] = __float2bfloat16_rn(fmaxf(acc[a][b][c] + S.b1[col], 0.f));
                    }
        }
        __syncthreads();
        // ---- y = W2 h + b2: warp w, pairs [16 (w / 4), +16), outputs [16 (w % 4), +16)
        {
            float acc[2][4];
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[b][c] = 0.f;
            const int rm = 16 * (warp >> 2), cn = 16 * (warp & 3);
#pragma unroll 4
            for (int ks = 0; ks < MLP_NHID; ks += 16) {
                const int r = rm + gq;
                const uint32_t a0 = ld_bf16x2(&S.hb[r][ks + 2 * tq]);
                const uint32_t a1 = ld_bf16x2(&S.hb[r + 8][ks + 2 * tq]);
                const uint32_t a2 = ld_bf16x2(&S.hb[r][ks + 2 * tq + 8]);
                const uint32_t a3 = ld_bf16x2(&S.hb[r + 8][ks + 2 * tq + 8]);
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    const int c = cn + 8 * b + gq;
                    mma_bf16(acc[b], a0, a1, a2, a3, ld_bf16x2(&S.w2[c][ks + 2 * tq]),
                             ld_bf16x2(&S.w2[c][ks + 2 * tq + 8]));
                }
            }
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int r = rm + gq + (c >= 2 ? 8 : 0);
                    const int col = cn + 8 * b + 2 * tq + (c & 1);
                    S.xy.y[r][col] = acc[b][c] + S.b2[col];
                }
        }
        __syncthreads();
        // ---- outputs, the warp's pairs, into S.r over their residuals
#pragma unroll
        for (int i = 0; i < FA_PPW; ++i) {
            const int q = warp * FA_PPW + i;
            if (q >= np) break;
            const int tl = q / k, j = q - tl * k;
            const float thf = S.thf[j], thl = S.thl[j];
            const float delta = 1e-3f * fmaxf(1.f, fabsf(thf));
            const float f = S.sc[q] * igf;
            float c[2], wd[2];
            float cc = 0.f, dd = 0.f;
            bool finite = true;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int rl = lane + 32 * hh;
                c[hh] = 0.f;
                wd[hh] = 0.f;
                if (tl * MLP_TILE + rl < rows) {
                    c[hh] = f * S.xy.y[q][rl];
                    // the guarded shifted pivot g(d - theta_j), the shift in two float steps
                    const float t = __fsub_rn(__fsub_rn(S.d[tl * MLP_TILE + rl], thf), thl);
                    const float gp = (t >= 0.f) ? fmaxf(t, delta) : -fmaxf(-t, delta);
                    wd[hh] = S.r[q][rl] / gp;
                    finite = finite && isfinite(c[hh]);
                    cc += c[hh] * c[hh];
                    dd += wd[hh] * wd[hh];
                }
            }
            finite = __all_sync(0xffffffffu, finite);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                cc += __shfl_xor_sync(0xffffffffu, cc, o);
                dd += __shfl_xor_sync(0xffffffffu, dd, o);
            }
            const float scale = !finite ? 0.f : (cc > dd ? sqrtf(dd / cc) : 1.f);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int rl = lane + 32 * hh;
                if (tl * MLP_TILE + rl < rows) S.r[q][rl] = finite ? wd[hh] + scale * c[hh] : wd[hh];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < rows * k; e += FA_THREADS) {
            const int row = e / k, j = e - row * k;
            W[r0 * k + e] = S.r[(row >> 6) * k + j][row & 63];
        }
    }
}

// Harvest training pairs from one iteration: R (residuals) and Wt (exact
// tile solves of the same R).  Pair (t, j) is kept when a 32-bit hash of
// (seed, iteration, t, j) falls below keep (2^32 keeps every pair).
__device__ __forceinline__ uint32_t mix32(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return static_cast<uint32_t>((z ^ (z >> 31)) >> 32);
}

__global__ void k_mlp_harvest(int64_t n, int k, const float *R, const float *Wt, const float *d, const double *theta,
                              double normG, uint64_t seed, int iter, uint64_t keep, int64_t cap, float *Xp, float *Tp,
                              unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    const int64_t P = ((n + MLP_TILE - 1) / MLP_TILE) * k;
    const double ig = 1.0 / normG;
    for (int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; p < P;
         p += (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5) {
        if (static_cast<uint64_t>(mix32(seed ^ (static_cast<uint64_t>(iter) << 40) ^ static_cast<uint64_t>(p))) >= keep) continue;
        const int64_t t = p / k;
        const int j = static_cast<int>(p % k);
        const int64_t r0 = t * MLP_TILE;
        float rv[2], dv[2], yv[2];
        float ss = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t i = r0 + lane + 32 * h;
            rv[h] = (i < n) ? R[i * k + j] : 0.f;
            yv[h] = (i < n) ? Wt[i * k + j] : 0.f;
            dv[h] = (i < n) ? d[i] : 0.f;
            ss += rv[h] * rv[h];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float s = sqrtf(ss);
        if (!(s > 0.f)) continue;
        unsigned long long slot = 0;
        if (lane == 0) slot = atomicAdd(count, 1ull);
        slot = __shfl_sync(0xffffffffu, slot, 0);
        if (static_cast<int64_t>(slot) >= cap) continue;
        const float th = static_cast<float>(theta[j]);
        float *x = Xp + static_cast<int64_t>(slot) * MLP_KIN;
        float *tg = Tp + static_cast<int64_t>(slot) * MLP_NOUT;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            x[lane + 32 * h] = rv[h] / s;
            x[MLP_TILE + lane + 32 * h] = static_cast<float>((dv[h] - th) * ig);
            const float yd = diag_solve(rv[h], dv[h], theta[j]);
            const float tv = static_cast<float>(normG * (yv[h] - yd) / s);
            tg[lane + 32 * h] = fminf(fmaxf(tv, -MLP_CLIP), MLP_CLIP);
        }
        if (lane < MLP_KIN - 2 * MLP_TILE) x[2 * MLP_TILE + lane] = (lane == 0) ? static_cast<float>(th * ig) : 0.f;
    }
}

// Batch gather by an affine permutation of the pair index: q = (a i + c) mod N.
__global__ void k_mlp_gather(int64_t B, int64_t N, uint64_t a, uint64_t c, int64_t b0, const float *Xp,
                             const float *Tp, float *Xb, float *Tb) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < B * (MLP_KIN + MLP_NOUT);
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = e / (MLP_KIN + MLP_NOUT);
        const int f = static_cast<int>(e % (MLP_KIN + MLP_NOUT));
        const int64_t q = static_cast<int64_t>((a * static_cast<uint64_t>(b0 + i) + c) % static_cast<uint64_t>(N));
        if (f < MLP_KIN) Xb[i * MLP_KIN + f] = Xp[q * MLP_KIN + f];
        else Tb[i * MLP_NOUT + (f - MLP_KIN)] = Tp[q * MLP_NOUT + (f - MLP_KIN)];
    }
}

// dY = 2 (Y - T) / (B 64), loss += wl sum (Y - T)^2 (wl = 1 / (B 64) for
// the batch mean).
__global__ void k_mlp_mse(int64_t B, const float *Y, const float *T, float *dY, double *loss, double wl) {
    __shared__ float red[256];
    float acc = 0.f;
    const float sc = 1.f / static_cast<float>(B * MLP_NOUT);
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < B * MLP_NOUT;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float dd = Y[e] - T[e];
        acc += dd * dd;
        dY[e] = 2.f * dd * sc;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, static_cast<double>(red[0]) * wl);
}

// dH *= (H > 0)   (relu'(z) with z > 0 <=> h > 0)
__global__ void k_mlp_relu_bwd(int64_t m, const float *H, float *dH) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        if (!(H[e] > 0.f)) dH[e] = 0.f;
}

// db[c] += sum over rows of D[r][c]   (D: B x N, N <= blockDim; db zeroed
// first): each CTA sums a range of rows for all N columns (thread c reads
// column c: rows are read whole, coalesced), one atomic per column and CTA.
__global__ void k_mlp_colsum(int64_t B, int N, const float *D, float *db) {
    const int c = threadIdx.x;
    if (c >= N) return;
    const int64_t per = (B + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = min(B, r0 + per);
    float acc = 0.f;
    for (int64_t r = r0; r < r1; ++r) acc += D[r * N + c];
    atomicAdd(&db[c], acc);
}

static cudaError_t colsum(int64_t B, int N, const float *D, float *db, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(db, 0, sizeof(float) * N, s);
    if (e != cudaSuccess) return e;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(2 * num_sms, (B + 63) / 64)));
    k_mlp_colsum<<<blocks, N <= 64 ? 64 : 256, 0, s>>>(B, N, D, db);
    return cudaGetLastError();
}

// Adam (Kingma & Ba 2015), bias-corrected, over the packed parameters.
__global__ void k_mlp_adam(int64_t m, float *p, const float *g, float *mo, float *vo, float lr, float bc1, float bc2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * mo[e] + (1.f - b1) * gg;
        const float vv = b2 * vo[e] + (1.f - b2) * gg * gg;
        mo[e] = mm;
        vo[e] = vv;
        p[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
}

// Initial weights: W1 He (Kaiming) normal, W1 ~ N(0, 2 / 129); b1, W2, b2 zero.
// The normal draws come from a counter-based generator: two uniforms from the
// SplitMix64 finaliser of (seed, index), combined by the Box-Muller transform.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void k_mlp_init(uint64_t seed, float *P) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < MLP_NPARAM; e += gridDim.x * blockDim.x) {
        float sd = 0.f;
        if (e < MLP_OFF_B1) sd = (e % MLP_KIN < 129) ? sqrtf(2.f / 129.f) : 0.f;
        float v = 0.f;
        if (sd > 0.f) {
            const uint64_t a = splitmix64(seed * 0x100000001B3ULL + 2ULL * e);
            const uint64_t b = splitmix64(seed * 0x100000001B3ULL + 2ULL * e + 1ULL);
            const float u1 = (static_cast<float>(a >> 40) + 0.5f) * (1.f / 16777216.f);   // (0, 1)
            const float u2 = static_cast<float>(b >> 40) * (1.f / 16777216.f);
            v = sd * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
        }
        P[e] = v;
    }
}

// ------------------------------------------------------------------ host side

static int grid_for(int64_t work, int num_sms) {
    int64_t b = (work + 255) / 256;
    if (b > static_cast<int64_t>(num_sms) * 16) b = static_cast<int64_t>(num_sms) * 16;
    return static_cast<int>(b < 1 ? 1 : b);
}

cudaError_t mlp_setup(lobpcg_ctx *h) {
    Mlp &M = h->mlp;
    if (M.P) return cudaSuccess;
    cudaError_t e = dev_alloc(h, reinterpret_cast<void **>(&M.P), sizeof(float) * MLP_NPARAM * 4);
    if (e != cudaSuccess) return e;
    M.G = M.P + MLP_NPARAM;
    M.Mo = M.G + MLP_NPARAM;
    M.Vo = M.Mo + MLP_NPARAM;
    e = cudaMemsetAsync(M.P, 0, sizeof(float) * MLP_NPARAM * 4, h->stream);
    if (e != cudaSuccess) return e;
    // the fused apply needs no workspace; P is the pair count it is sized for
    M.cap_apply = ((h->T.n + MLP_TILE - 1) / MLP_TILE) * h->params.k;
    return cudaSuccess;
}

// Packed parameter layout on the device (W1 padded to 144 columns):
//   W1 [256][144] | b1 [256] | W2 [64][256] | b2 [64]
// Caller layout (the oracle's): W1 [256][129] | b1 | W2 | b2.
cudaError_t mlp_set_params(lobpcg_ctx *h, const float *src, bool on_host) {
    Mlp &M = h->mlp;
    std::vector<float> host(MLP_NPARAM_CALLER), dev(MLP_NPARAM, 0.f);
    cudaError_t e = cudaMemcpyAsync(host.data(), src, sizeof(float) * MLP_NPARAM_CALLER,
                                    on_host ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    for (int r = 0; r < MLP_NHID; ++r)
        for (int c = 0; c < 129; ++c) dev[MLP_OFF_W1 + r * MLP_KIN + c] = host[r * 129 + c];
    const int cb1 = MLP_NHID * 129;
    for (int r = 0; r < MLP_NHID; ++r) dev[MLP_OFF_B1 + r] = host[cb1 + r];
    const int cw2 = cb1 + MLP_NHID;
    for (int q = 0; q < MLP_NOUT * MLP_NHID; ++q) dev[MLP_OFF_W2 + q] = host[cw2 + q];
    const int cb2 = cw2 + MLP_NOUT * MLP_NHID;
    for (int q = 0; q < MLP_NOUT; ++q) dev[MLP_OFF_B2 + q] = host[cb2 + q];
    e = cudaMemcpyAsync(M.P, dev.data(), sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.Mo, 0, sizeof(float) * MLP_NPARAM * 2, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    M.step = 0;
    M.ready = true;
    return e;
}

// device packed (W1 padded) -> caller layout
static void unpack(const std::vector<float> &dev, float *out) {
    for (int r = 0; r < MLP_NHID; ++r)
        for (int c = 0; c < 129; ++c) out[r * 129 + c] = dev[MLP_OFF_W1 + r * MLP_KIN + c];
    const int cb1 = MLP_NHID * 129;
    for (int r = 0; r < MLP_NHID; ++r) out[cb1 + r] = dev[MLP_OFF_B1 + r];
    const int cw2 = cb1 + MLP_NHID;
    for (int q = 0; q < MLP_NOUT * MLP_NHID; ++q) out[cw2 + q] = dev[MLP_OFF_W2 + q];
    const int cb2 = cw2 + MLP_NOUT * MLP_NHID;
    for (int q = 0; q < MLP_NOUT; ++q) out[cb2 + q] = dev[MLP_OFF_B2 + q];
}

cudaError_t mlp_get_params(lobpcg_ctx *h, float *dst, bool on_host, bool grads) {
    std::vector<float> dev(MLP_NPARAM), host(MLP_NPARAM_CALLER);
    cudaError_t e = cudaMemcpyAsync(dev.data(), grads ? h->mlp.G : h->mlp.P, sizeof(float) * MLP_NPARAM,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    unpack(dev, host.data());
    e = cudaMemcpyAsync(dst, host.data(), sizeof(float) * MLP_NPARAM_CALLER,
                        on_host ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e;
}

// Y (B x 64) = net(X) for X (B x 144, padded rows); H (B x 256) kept.
static cudaError_t forward(lobpcg_ctx *h, const float *X, int64_t B, float *Hh, float *Y, cudaStream_t s) {
    Mlp &M = h->mlp;
    GemmArgs g1{static_cast<int>(B), MLP_NHID, MLP_KIN, X, MLP_KIN, 0, M.P + MLP_OFF_W1, MLP_KIN, 1, Hh, MLP_NHID,
                M.P + MLP_OFF_B1, 1};
    cudaError_t e = gemm(g1, s);
    if (e != cudaSuccess) return e;
    GemmArgs g2{static_cast<int>(B), MLP_NOUT, MLP_NHID, Hh, MLP_NHID, 0, M.P + MLP_OFF_W2, MLP_NHID, 1, Y, MLP_NOUT,
                M.P + MLP_OFF_B2, 0};
    return gemm(g2, s);
}

// Gradients of the batch MSE into M.G (packed); loss added to *loss (device).
static cudaError_t backward(lobpcg_ctx *h, const float *X, const float *T, int64_t B, float *Hh, float *Y, float *dY,
                            float *dH, double *loss) {
    Mlp &M = h->mlp;
    cudaError_t e = forward(h, X, B, Hh, Y, h->stream);
    if (e != cudaSuccess) return e;
    k_mlp_mse<<<grid_for(B * MLP_NOUT, h->num_sms), 256, 0, h->stream>>>(B, Y, T, dY, loss,
                                                                          1.0 / (static_cast<double>(B) * MLP_NOUT));
    // dW2 = dY^T H  (64 x 256)
    GemmArgs gw2{MLP_NOUT, MLP_NHID, static_cast<int>(B), dY, MLP_NOUT, 1, Hh, MLP_NHID, 0, M.G + MLP_OFF_W2,
                 MLP_NHID, nullptr, 0};
    if ((e = gemm(gw2, h->stream, h->num_sms)) != cudaSuccess) return e;
    if ((e = colsum(B, MLP_NOUT, dY, M.G + MLP_OFF_B2, h->num_sms, h->stream)) != cudaSuccess) return e;
    // dH = (dY W2) * relu'
    GemmArgs gh{static_cast<int>(B), MLP_NHID, MLP_NOUT, dY, MLP_NOUT, 0, M.P + MLP_OFF_W2, MLP_NHID, 0, dH, MLP_NHID,
                nullptr, 0};
    if ((e = gemm(gh, h->stream)) != cudaSuccess) return e;
    k_mlp_relu_bwd<<<grid_for(B * MLP_NHID, h->num_sms), 256, 0, h->stream>>>(B * MLP_NHID, Hh, dH);
    // dW1 = dH^T X  (256 x 144)
    GemmArgs gw1{MLP_NHID, MLP_KIN, static_cast<int>(B), dH, MLP_NHID, 1, X, MLP_KIN, 0, M.G + MLP_OFF_W1, MLP_KIN,
                 nullptr, 0};
    if ((e = gemm(gw1, h->stream, h->num_sms)) != cudaSuccess) return e;
    return colsum(B, MLP_NHID, dH, M.G + MLP_OFF_B1, h->num_sms, h->stream);
}

cudaError_t mlp_forward_rows(lobpcg_ctx *h, const float *X129, int64_t B, float *Y) {
    // pad the caller's 129-wide rows to 144 in scratch
    float *buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, sizeof(float) * B * (MLP_KIN + MLP_NHID), h->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(buf, 0, sizeof(float) * B * MLP_KIN, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(buf, sizeof(float) * MLP_KIN, X129, sizeof(float) * 129, sizeof(float) * 129, B,
                              cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = forward(h, buf, B, buf + B * MLP_KIN, Y, h->stream);
    cudaFreeAsync(buf, h->stream);
    return e;
}

cudaError_t mlp_grad_rows(lobpcg_ctx *h, const float *X129, const float *T, int64_t B, double *loss_host) {
    float *buf = nullptr;
    const size_t fl = static_cast<size_t>(B) * (MLP_KIN + 2 * MLP_NHID + 2 * MLP_NOUT) + 8;
    cudaError_t e = cudaMallocAsync(&buf, sizeof(float) * fl, h->stream);
    if (e != cudaSuccess) return e;
    float *X = buf, *Hh = X + B * MLP_KIN, *dH = Hh + B * MLP_NHID, *Y = dH + B * MLP_NHID, *dY = Y + B * MLP_NOUT;
    double *loss = reinterpret_cast<double *>(dY + B * MLP_NOUT + ((B * MLP_NOUT) & 1));
    e = cudaMemsetAsync(X, 0, sizeof(float) * B * MLP_KIN, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(X, sizeof(float) * MLP_KIN, X129, sizeof(float) * 129, sizeof(float) * 129, B,
                              cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = backward(h, X, T, B, Hh, Y, dY, dH, loss);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss_host, loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(buf, h->stream);
    return e;
}

cudaError_t mlp_init(lobpcg_ctx *h, uint64_t seed) {
    Mlp &M = h->mlp;
    k_mlp_init<<<64, 256, 0, h->stream>>>(seed, M.P);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(M.Mo, 0, sizeof(float) * MLP_NPARAM * 2, h->stream);
    M.step = 0;
    M.ready = (e == cudaSuccess);
    return e;
}

cudaError_t mlp_adam(lobpcg_ctx *h, float lr) {
    Mlp &M = h->mlp;
    M.step += 1;
    const float bc1 = 1.f - powf(0.9f, static_cast<float>(M.step));
    const float bc2 = 1.f - powf(0.999f, static_cast<float>(M.step));
    k_mlp_adam<<<grid_for(MLP_NPARAM, h->num_sms), 256, 0, h->stream>>>(MLP_NPARAM, M.P, M.G, M.Mo, M.Vo, lr, bc1, bc2);
    return cudaGetLastError();
}

// W = K_mlp^{-1} R on an n x k float32 block (W may be R): the fused kernel.
cudaError_t mlp_apply(lobpcg_ctx *h, int k, const float *R, const double *theta, float *W, cudaStream_t s) {
    Mlp &M = h->mlp;
    const int64_t n = h->T.n;
    const int64_t P = ((n + MLP_TILE - 1) / MLP_TILE) * k;
    if (P > M.cap_apply) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_mlp_apply_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(sizeof(FaSmem)));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t ntiles = (n + MLP_TILE - 1) / MLP_TILE, T = FA_PAIRS / k;
    const int64_t batches = (ntiles + T - 1) / T;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(batches, h->num_sms)));
    k_mlp_apply_fused<<<blocks, FA_THREADS, sizeof(FaSmem), s>>>(n, k, M.P, R, h->T.diag, theta, h->gershgorin, W);
    return cudaGetLastError();
}

cudaError_t mlp_harvest(lobpcg_ctx *h, int k, const float *R, const float *Wt, const double *theta, int iter) {
    Mlp &M = h->mlp;
    const int64_t n = h->T.n;
    const int64_t P = ((n + MLP_TILE - 1) / MLP_TILE) * k;
    k_mlp_harvest<<<grid_for(P * 32, h->num_sms), 256, 0, h->stream>>>(n, k, R, Wt, h->T.diag, theta, h->gershgorin,
                                                                     h->params.seed, iter, M.keep, M.cap_pairs, M.Xp,
                                                                     M.Tp, M.d_count);
    return cudaGetLastError();
}

cudaError_t mlp_alloc_pairs(lobpcg_ctx *h, int64_t cap, int harvest_iters) {
    Mlp &M = h->mlp;
    if (M.Xp) { cudaFree(M.Xp); M.Xp = nullptr; }
    cudaError_t e = cudaMalloc(&M.Xp, sizeof(float) * (cap * (MLP_KIN + MLP_NOUT)) + 64);
    if (e != cudaSuccess) return e;
    M.Tp = M.Xp + cap * MLP_KIN;
    M.d_count = reinterpret_cast<unsigned long long *>(M.Tp + cap * MLP_NOUT);
    M.d_count = reinterpret_cast<unsigned long long *>((reinterpret_cast<uintptr_t>(M.d_count) + 15) & ~uintptr_t(15));
    M.cap_pairs = cap;
    // keep rate so that harvest_iters iterations yield about cap pairs
    const int64_t per_iter = ((h->T.n + MLP_TILE - 1) / MLP_TILE) * h->params.k;
    double rate = static_cast<double>(cap) / (static_cast<double>(per_iter) * (harvest_iters > 0 ? harvest_iters : 1));
    rate = rate > 1.0 ? 1.0 : rate;
    M.keep = rate >= 1.0 ? (uint64_t(1) << 32) : static_cast<uint64_t>(rate * 4294967296.0);
    return cudaMemsetAsync(M.d_count, 0, sizeof(unsigned long long), h->stream);
}

void mlp_release(lobpcg_ctx *h) {
    if (h->mlp.Xp) cudaFree(h->mlp.Xp);
    h->mlp.Xp = nullptr;
}

// Train on the harvested pairs.  The last tenth (in harvest order) is held
// out; the rest is visited `epochs` times in batches of up to MLP_BATCH rows
// in an affine-permuted order (a new permutation each epoch), one Adam step
// (learning rate lr) per batch.  The held-out mean squared error is measured
// before training and after every epoch (loss_hist, host, epochs + 1
// entries) and the weights with the lowest one are kept (early stopping), so
// training never leaves a form that does worse on held-out pairs than the
// one it started from.
cudaError_t mlp_train(lobpcg_ctx *h, int epochs, float lr, double *loss_hist, int64_t *npairs_out) {
    Mlp &M = h->mlp;
    unsigned long long cnt = 0;
    cudaError_t e = cudaMemcpyAsync(&cnt, M.d_count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return e;
    const int64_t N = static_cast<int64_t>(cnt < static_cast<unsigned long long>(M.cap_pairs) ? cnt : M.cap_pairs);
    if (npairs_out) *npairs_out = N;
    if (N < MLP_BATCH) return cudaErrorInvalidValue;
    const int64_t Nv = N / 10, Ntr = N - Nv;
    const int64_t B = Ntr < MLP_BATCH ? Ntr : MLP_BATCH;
    float *buf = nullptr;
    const size_t fl = static_cast<size_t>(MLP_BATCH) * (MLP_KIN + MLP_NOUT + 2 * MLP_NHID + 2 * MLP_NOUT) +
                      MLP_NPARAM + 16;
    e = cudaMallocAsync(&buf, sizeof(float) * fl, h->stream);
    if (e != cudaSuccess) return e;
    float *Xb = buf, *Tb = Xb + MLP_BATCH * MLP_KIN, *Hh = Tb + MLP_BATCH * MLP_NOUT, *dH = Hh + MLP_BATCH * MLP_NHID,
          *Y = dH + MLP_BATCH * MLP_NHID, *dY = Y + MLP_BATCH * MLP_NOUT, *best = dY + MLP_BATCH * MLP_NOUT;
    double *loss = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(best + MLP_NPARAM) + 15) & ~uintptr_t(15));
    // held-out loss of the current weights
    auto held_out = [&](double &out) -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(loss, 0, sizeof(double), h->stream);
        for (int64_t o = 0; o < Nv && r == cudaSuccess; o += MLP_BATCH) {
            const int64_t bc = (Nv - o < MLP_BATCH) ? Nv - o : MLP_BATCH;
            r = forward(h, M.Xp + (Ntr + o) * MLP_KIN, bc, Hh, Y, h->stream);
            if (r == cudaSuccess)
                k_mlp_mse<<<grid_for(bc * MLP_NOUT, h->num_sms), 256, 0, h->stream>>>(
                    bc, Y, M.Tp + (Ntr + o) * MLP_NOUT, dY, loss, 1.0 / (static_cast<double>(Nv) * MLP_NOUT));
        }
        if (r == cudaSuccess) r = cudaMemcpyAsync(&out, loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (r == cudaSuccess) r = cudaStreamSynchronize(h->stream);
        return r;
    };
    double vbest = 0.0;
    e = held_out(vbest);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best, M.P, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToDevice, h->stream);
    if (loss_hist) loss_hist[0] = vbest;
    const int64_t nb = Ntr / B;
    auto gcd = [](uint64_t x, uint64_t y) { while (y) { uint64_t t = x % y; x = y; y = t; } return x; };
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        // affine permutation q = (a i + c) mod Ntr with a coprime to Ntr
        uint64_t a = (2654435761ULL + 2ULL * static_cast<uint64_t>(ep) * 40503ULL) % static_cast<uint64_t>(Ntr);
        while (gcd(a, static_cast<uint64_t>(Ntr)) != 1) a = (a + 1) % static_cast<uint64_t>(Ntr);
        const uint64_t c = (0x9E3779B97F4A7C15ULL * static_cast<uint64_t>(ep + 1)) % static_cast<uint64_t>(Ntr);
        e = cudaMemsetAsync(loss, 0, sizeof(double), h->stream);
        for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
            k_mlp_gather<<<grid_for(B * (MLP_KIN + MLP_NOUT), h->num_sms), 256, 0, h->stream>>>(B, Ntr, a, c, b * B,
                                                                                               M.Xp, M.Tp, Xb, Tb);
            e = backward(h, Xb, Tb, B, Hh, Y, dY, dH, loss);
            if (e == cudaSuccess) e = mlp_adam(h, lr);
        }
        double v = 0.0;
        if (e == cudaSuccess) e = held_out(v);
        if (loss_hist) loss_hist[ep + 1] = v;
        if (e == cudaSuccess && v < vbest) {
            vbest = v;
            e = cudaMemcpyAsync(best, M.P, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToDevice, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(M.P, best, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(buf, h->stream);
    M.ready = (e == cudaSuccess);
    return e;
}

}  // namespace lobpcg
