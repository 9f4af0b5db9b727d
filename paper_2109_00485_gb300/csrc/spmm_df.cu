// Symmetric SpMM  Y = H X  with float64 vectors, from the stored lower
// triangle (Algorithm 2 with the transpose of Section 3.3), for the float64
// refinement, the explicit re-check of convergence and lobpcg_spmm_sym_f64.
//
// GB300 issues FP64 at about 1/64 of its FP32 rate, so the products are
// formed in float32 with error-free transformations instead:
//   x = x_hi + x_lo + d    (x_hi, x_lo the truncated 24-bit words, |d| < 2^-47 |x|; split once per call)
//   h x_hi = p + e         (p = fl32(h x_hi), e = fma(h, x_hi, -p): exact, h being float32)
//   s + p = s' + t         (TwoSum, Knuth: exact)
//   c <- c + (t + e) + h x_lo
// per term, with (s, c) renormalised by Fast2Sum after each 16-term tile.
// Each term is then exact but for the split's remainder and roundings of
// size 2^-47 |h x|, so an output is within a few 2^-47 sum |h x| of its
// exact value; it is written as the float64 s + c.
//
// Two passes, neither with atomics (so the result does not depend on the
// order warps run in):
//   rows     one warp per row block: Y_R = sum over the row block's chunks of
//            H_t X_C (the diagonal chunk as S = L + L^T - D); Y_R is stored;
//   columns  one warp per column tile: Y_C += sum over the off-diagonal chunks
//            in that column of H_t^T X_R, from a column index of the chunks
//            (built once per handle, each column's chunks in row-block order);
//            Y_C is added to the stored rows.
// Per chunk the warp loads the chunk's words and the 16 rows of x_hi, x_lo
// its product needs into registers one chunk ahead, stages them in shared
// memory, expands the chunk to a dense 16 x 16 tile there, and each lane
// forms k/2 outputs of one row (or column) of the tile product.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"
#include "df.cuh"
#include "internal.h"

namespace lobpcg {

namespace {

constexpr int DF_WARPS = 8;        // warps per block
constexpr int DF_HS = 17;          // row stride of the dense tile

struct DfWarp {
    uint32_t cw[512];              // one chunk's words
    float ht[TILE * DF_HS];        // the dense tile
    float xh[TILE * 32], xl[TILE * 32];   // 16 rows of x_hi, x_lo (row stride k)
};

// x = x_hi + x_lo for the m entries of x (df_split: integer operations on
// the bit pattern, GB300 converting double to float at its FP64 rate),
// zeros for entries m .. mp - 1
__global__ void k_split64(int64_t m, int64_t mp, const double *x, float *xh, float *xl) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < mp;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float hi = 0.f, lo = 0.f;
        if (i < m) df_split(x[i], hi, lo);
        xh[i] = hi;
        xl[i] = lo;
    }
}

// s + c += h (x_hi + x_lo) (the file comment's steps) for two outputs at
// once, as packed f32x2 instructions (each half rounds as the scalar
// operation, and the explicit rounding keeps the compiler from contracting
// or reassociating the error-free steps): hh = (h, h), nh = (-h, -h),
// q = -p, TwoSum(s, p) written as (s - q, (s - (sn - bp)) - (q + bp))
__device__ __forceinline__ void df_term2(float2 hh, float2 nh, float2 xh, float2 xl, float2 &s, float2 &c) {
    const float2 q = df2_mul(nh, xh);
    const float2 e = df2_fma(hh, xh, q);
    const float2 sn = df2_sub(s, q);
    const float2 bp = df2_sub(sn, s);
    const float2 t = df2_sub(df2_sub(s, df2_sub(sn, bp)), df2_add(q, bp));
    s = sn;
    c = df2_fma(hh, xl, df2_add(c, df2_add(t, e)));
}

__device__ __forceinline__ void df_renorm2(float2 &s, float2 &c) {
    const float2 sn = df2_add(s, c);
    c = df2_sub(c, df2_sub(sn, s));
    s = sn;
}

// A chunk and the 16 vector rows of its product, held in registers (one
// chunk ahead of the tile being multiplied).
template <int K>
struct DfPrefetch {
    uint4 w[4];                    // chunk words 4 (lane + 32 q), q < 4
    float4 xh[(K + 7) / 8], xl[(K + 7) / 8];   // the 16 x rows, float4 (lane + 32 q)
    int4 rec;                      // the chunk record
};

template <int K>
__device__ __forceinline__ void df_fetch(DfPrefetch<K> &f, const uint32_t *data, const ChunkRec *chunk, int64_t ci,
                                         int64_t xrow0, int64_t n, const float *xh, const float *xl, int lane) {
    f.rec = __ldg(reinterpret_cast<const int4 *>(chunk + ci));
    const int64_t off = static_cast<int64_t>((static_cast<uint64_t>(static_cast<uint32_t>(f.rec.y)) << 32) |
                                             static_cast<uint32_t>(f.rec.x));
    const int info = f.rec.w;
    const int npad = (info >> NPAD_SHIFT) & 0x3FF;
    const int words = (info & VONLY_FLAG) ? npad : 2 * npad;
    const uint4 *src = reinterpret_cast<const uint4 *>(data + off);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int v = lane + 32 * q;
        f.w[q] = (4 * v < words) ? __ldg(src + v) : make_uint4(0, 0, 0, 0);
    }
    // all 16 rows: the split vectors carry 16 zero rows past row n - 1
    const float4 *sh = reinterpret_cast<const float4 *>(xh + xrow0 * K);
    const float4 *sl = reinterpret_cast<const float4 *>(xl + xrow0 * K);
#pragma unroll
    for (int q = 0; q < (K + 7) / 8; ++q) {
        const int v = lane + 32 * q;
        const bool ok = v < TILE * K / 4;
        f.xh[q] = ok ? __ldg(sh + v) : make_float4(0.f, 0.f, 0.f, 0.f);
        f.xl[q] = ok ? __ldg(sl + v) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// Registers -> shared memory, then the dense tile (diagonal chunks as
// S = L + L^T - D).  Returns the chunk's info word.
template <int K>
__device__ __forceinline__ int df_stage(const DfPrefetch<K> &f, DfWarp *ws, int lane) {
#pragma unroll
    for (int q = 0; q < 4; ++q) reinterpret_cast<uint4 *>(ws->cw)[lane + 32 * q] = f.w[q];
#pragma unroll
    for (int q = 0; q < (K + 7) / 8; ++q) {
        const int v = lane + 32 * q;
        if (v < TILE * K / 4) {
            reinterpret_cast<float4 *>(ws->xh)[v] = f.xh[q];
            reinterpret_cast<float4 *>(ws->xl)[v] = f.xl[q];
        }
    }
    const int info = f.rec.w;
    const int cnt = info & 0xFFFF, npad = (info >> NPAD_SHIFT) & 0x3FF;
    const bool vo = (info & VONLY_FLAG) != 0, diag = (info & DIAG_FLAG) != 0;
    for (int e = lane; e < TILE * DF_HS; e += 32) ws->ht[e] = 0.f;
    __syncwarp();
    const float *val = reinterpret_cast<const float *>(ws->cw) + (vo ? 0 : npad);
    for (int e = lane; e < cnt; e += 32) {
        int r, c;
        if (!vo) {
            const uint32_t u = ws->cw[e];
            r = (u >> 28) & 15;
            c = u & 15;
        } else if (!diag) {
            // complete tile: row e / 16; position p of a row holds column 4 (p % 4) + p / 4
            const int p = e & 15;
            r = e >> 4;
            c = 4 * (p & 3) + (p >> 2);
        } else {
            // complete lower triangle, row-major: row r holds entries r (r + 1) / 2 ..
            int q = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) - 1.f) * 0.5f);
            while (q * (q + 1) / 2 > e) --q;
            while ((q + 1) * (q + 2) / 2 <= e) ++q;
            r = q;
            c = e - q * (q + 1) / 2;
        }
        const float v = val[e];
        ws->ht[r * DF_HS + c] = v;
        if (diag) ws->ht[c * DF_HS + r] = v;
    }
    __syncwarp();
    return info;
}

// acc[q] (+)= sum_t A(o, t) x[t][q0 + q], o = lane / 2, q0 = (lane % 2) K / 2;
// A(o, t) = tile[o][t] (rows pass) or tile[t][o] (columns pass).  The
// outputs in packed pairs (q, q + 1); for odd K / 2 the last pair's second
// half runs on a neighbouring column and is never written.
template <int K>
struct DfAcc {
    static constexpr int KP = (K / 2 + 1) / 2;
    float2 s[KP], c[KP];
};
template <int K, bool TRANS>
__device__ __forceinline__ void df_tile_mac(const DfWarp *ws, int lane, DfAcc<K> &acc) {
    constexpr int KH = K / 2, KP = DfAcc<K>::KP;
    const int o = lane >> 1, q0 = (lane & 1) * KH;
#pragma unroll 4
    for (int t = 0; t < TILE; ++t) {
        const float h = TRANS ? ws->ht[t * DF_HS + o] : ws->ht[o * DF_HS + t];
        const float2 hh = make_float2(h, h), nh = make_float2(-h, -h);
        const float *ph = ws->xh + t * K + q0;
        const float *pl = ws->xl + t * K + q0;
#pragma unroll
        for (int p = 0; p < KP; ++p) {
            float2 xh2, xl2;
            if constexpr (KH % 2 == 0) {
                xh2 = reinterpret_cast<const float2 *>(ph)[p];
                xl2 = reinterpret_cast<const float2 *>(pl)[p];
            } else {
                xh2 = make_float2(ph[2 * p], ph[2 * p + 1]);
                xl2 = make_float2(pl[2 * p], pl[2 * p + 1]);
            }
            df_term2(hh, nh, xh2, xl2, acc.s[p], acc.c[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < KP; ++p) df_renorm2(acc.s[p], acc.c[p]);
}

// output q of the lane's half (s + c as float64)
template <int K>
__device__ __forceinline__ double df_out(const DfAcc<K> &acc, int q) {
    const float2 s = acc.s[q >> 1], c = acc.c[q >> 1];
    return (q & 1) ? static_cast<double>(s.y) + static_cast<double>(c.y)
                   : static_cast<double>(s.x) + static_cast<double>(c.x);
}

// Rows pass: Y[rb] = sum over rb's chunks of H_t X_C.
template <int K>
__global__ void __launch_bounds__(DF_WARPS * 32, 2) k_spmm_df_rows(int64_t n, int64_t R, const uint32_t *data,
                                                               const ChunkRec *chunk, const int64_t *rb_chunk,
                                                               const float *xh, const float *xl, double *Y) {
    extern __shared__ __align__(16) unsigned char df_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DfWarp *ws = reinterpret_cast<DfWarp *>(df_smem) + warp;
    constexpr int KH = K / 2;
    for (int64_t rb = static_cast<int64_t>(blockIdx.x) * DF_WARPS + warp; rb < R;
         rb += static_cast<int64_t>(gridDim.x) * DF_WARPS) {
        DfAcc<K> acc;
#pragma unroll
        for (int q = 0; q < DfAcc<K>::KP; ++q) acc.s[q] = acc.c[q] = make_float2(0.f, 0.f);
        const int64_t c0 = rb_chunk[rb], c1 = rb_chunk[rb + 1];
        DfPrefetch<K> f;
        if (c0 < c1) {
            const int ct = __ldg(reinterpret_cast<const int4 *>(chunk + c0)).z;
            df_fetch<K>(f, data, chunk, c0, static_cast<int64_t>(ct) * TILE, n, xh, xl, lane);
        }
        for (int64_t ci = c0; ci < c1; ++ci) {
            __syncwarp();
            df_stage<K>(f, ws, lane);
            if (ci + 1 < c1) {
                const int ct = __ldg(reinterpret_cast<const int4 *>(chunk + ci + 1)).z;
                df_fetch<K>(f, data, chunk, ci + 1, static_cast<int64_t>(ct) * TILE, n, xh, xl, lane);
            }
            df_tile_mac<K, false>(ws, lane, acc);
        }
        const int o = lane >> 1, q0 = (lane & 1) * KH;
        const int64_t row = rb * TILE + o;
        if (row < n) {
#pragma unroll
            for (int q = 0; q < KH; ++q) Y[row * K + q0 + q] = df_out<K>(acc, q);
        }
    }
}

// Columns pass: Y[ct] += sum over the off-diagonal chunks in column tile ct
// of H_t^T X_R (list[col_ptr[ct] .. col_ptr[ct + 1]): (chunk, row block)).
template <int K>
__global__ void __launch_bounds__(DF_WARPS * 32, 2) k_spmm_df_cols(int64_t n, int64_t R, const uint32_t *data,
                                                               const ChunkRec *chunk, const int64_t *col_ptr,
                                                               const int2 *list, const float *xh, const float *xl,
                                                               double *Y) {
    extern __shared__ __align__(16) unsigned char df_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    DfWarp *ws = reinterpret_cast<DfWarp *>(df_smem) + warp;
    constexpr int KH = K / 2;
    for (int64_t ct = static_cast<int64_t>(blockIdx.x) * DF_WARPS + warp; ct < R;
         ct += static_cast<int64_t>(gridDim.x) * DF_WARPS) {
        const int64_t a0 = col_ptr[ct], a1 = col_ptr[ct + 1];
        if (a0 == a1) continue;
        DfAcc<K> acc;
#pragma unroll
        for (int q = 0; q < DfAcc<K>::KP; ++q) acc.s[q] = acc.c[q] = make_float2(0.f, 0.f);
        DfPrefetch<K> f;
        {
            const int2 e = __ldg(list + a0);
            df_fetch<K>(f, data, chunk, e.x, static_cast<int64_t>(e.y) * TILE, n, xh, xl, lane);
        }
        for (int64_t a = a0; a < a1; ++a) {
            __syncwarp();
            df_stage<K>(f, ws, lane);
            if (a + 1 < a1) {
                const int2 e = __ldg(list + a + 1);
                df_fetch<K>(f, data, chunk, e.x, static_cast<int64_t>(e.y) * TILE, n, xh, xl, lane);
            }
            df_tile_mac<K, true>(ws, lane, acc);
        }
        const int o = lane >> 1, q0 = (lane & 1) * KH;
        const int64_t row = ct * TILE + o;
        if (row < n) {
#pragma unroll
            for (int q = 0; q < KH; ++q) {
                double *y = Y + row * K + q0 + q;
                *y = *y + df_out<K>(acc, q);
            }
        }
    }
}

// ---------------------------------------------------------------- column index

// cnt[ct] = off-diagonal chunks in column tile ct (thread per row block)
__global__ void k_col_count(int64_t R, const ChunkRec *chunk, const int64_t *rb_chunk, int *cnt) {
    const int64_t rb = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (rb >= R) return;
    for (int64_t ci = rb_chunk[rb]; ci < rb_chunk[rb + 1]; ++ci) {
        const ChunkRec r = chunk[ci];
        if (!(r.info & DIAG_FLAG)) atomicAdd(cnt + r.ct, 1);
    }
}

// ptr[0..R] = exclusive prefix sum of cnt[0..R) (one CTA: each thread a
// contiguous segment, then a scan of the segment sums)
__global__ void k_col_scan(int64_t R, const int *cnt, int64_t *ptr) {
    __shared__ int64_t part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int64_t seg = (R + T - 1) / T, a = t * seg, b = (a + seg < R) ? a + seg : R;
    int64_t sum = 0;
    for (int64_t i = a; i < b; ++i) sum += cnt[i];
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {   // inclusive scan (Hillis-Steele)
        const int64_t v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - sum;
    for (int64_t i = a; i < b; ++i) {
        ptr[i] = run;
        run += cnt[i];
    }
    if (t == T - 1) ptr[R] = part[t];
}

// list[ptr[ct] + slot] = (chunk, row block); cur[] counts the slots taken
__global__ void k_col_fill(int64_t R, const ChunkRec *chunk, const int64_t *rb_chunk, const int64_t *ptr, int *cur,
                           int2 *list) {
    const int64_t rb = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (rb >= R) return;
    for (int64_t ci = rb_chunk[rb]; ci < rb_chunk[rb + 1]; ++ci) {
        const ChunkRec r = chunk[ci];
        if (r.info & DIAG_FLAG) continue;
        const int slot = atomicAdd(cur + r.ct, 1);
        list[ptr[r.ct] + slot] = make_int2(static_cast<int>(ci), static_cast<int>(rb));
    }
}

// each column's entries in row-block order (insertion sort, thread per column tile)
__global__ void k_col_sort(int64_t R, const int64_t *ptr, int2 *list) {
    const int64_t ct = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (ct >= R) return;
    const int64_t a = ptr[ct], b = ptr[ct + 1];
    for (int64_t i = a + 1; i < b; ++i) {
        const int2 v = list[i];
        int64_t j = i - 1;
        while (j >= a && list[j].y > v.y) {
            list[j + 1] = list[j];
            --j;
        }
        list[j + 1] = v;
    }
}

template <int K>
cudaError_t launch_df(lobpcg_ctx *h, double *Y, cudaStream_t s) {
    const Tiled &T = h->T;
    const size_t smem = sizeof(DfWarp) * DF_WARPS;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_spmm_df_rows<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_spmm_df_cols<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t wblocks = (T.R + DF_WARPS - 1) / DF_WARPS;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(wblocks, static_cast<int64_t>(h->num_sms) * 8)));
    const float *xh = h->df.xs, *xl = h->df.xs + h->df.xs_stride;
    k_spmm_df_rows<K><<<blocks, DF_WARPS * 32, smem, s>>>(T.n, T.R, T.data, T.chunk, T.rb_chunk, xh, xl, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_spmm_df_cols<K><<<blocks, DF_WARPS * 32, smem, s>>>(T.n, T.R, T.data, T.chunk, h->df.col_ptr, h->df.col_list,
                                                          xh, xl, Y);
    return cudaGetLastError();
}

}  // namespace

bool spmm_df_ok(int k, const double *X, const double *Y) {
    return k >= 2 && k <= 32 && k % 2 == 0 && X && Y;
}

cudaError_t launch_spmm_sym_df(lobpcg_ctx *h, const double *X, double *Y, int k, cudaStream_t s) {
    if (!spmm_df_ok(k, X, Y)) return cudaErrorInvalidValue;
    Tiled &T = h->T;
    DfIndex &D = h->df;
    cudaError_t e;
    if (!D.col_ptr) {   // column index, once per handle
        int *cnt = nullptr;
        e = dev_alloc(h, reinterpret_cast<void **>(&D.col_ptr), sizeof(int64_t) * (T.R + 1));
        if (e == cudaSuccess) e = dev_alloc(h, reinterpret_cast<void **>(&D.col_list), sizeof(int2) * std::max<int64_t>(T.nchunks, 1));
        if (e == cudaSuccess) e = cudaMallocAsync(&cnt, sizeof(int) * T.R, s);
        if (e != cudaSuccess) { D.col_ptr = nullptr; return e; }
        const int tpb = 256;
        const int gb = static_cast<int>((T.R + tpb - 1) / tpb);
        e = cudaMemsetAsync(cnt, 0, sizeof(int) * T.R, s);
        if (e == cudaSuccess) { k_col_count<<<gb, tpb, 0, s>>>(T.R, T.chunk, T.rb_chunk, cnt); e = cudaGetLastError(); }
        if (e == cudaSuccess) { k_col_scan<<<1, 1024, 0, s>>>(T.R, cnt, D.col_ptr); e = cudaGetLastError(); }
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * T.R, s);
        if (e == cudaSuccess) { k_col_fill<<<gb, tpb, 0, s>>>(T.R, T.chunk, T.rb_chunk, D.col_ptr, cnt, D.col_list); e = cudaGetLastError(); }
        if (e == cudaSuccess) { k_col_sort<<<gb, tpb, 0, s>>>(T.R, D.col_ptr, D.col_list); e = cudaGetLastError(); }
        cudaError_t e2 = cudaFreeAsync(cnt, s);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) { D.col_ptr = nullptr; return e; }
    }
    if (D.xs_k < k) {   // x_hi, x_lo for n + 16 rows (the split writes the last 16 as zeros)
        const size_t stride = static_cast<size_t>(T.n + TILE) * k;
        float *p = nullptr;
        e = dev_alloc(h, reinterpret_cast<void **>(&p), sizeof(float) * 2 * stride);
        if (e != cudaSuccess) return e;
        D.xs = p;
        D.xs_k = k;
    }
    D.xs_stride = static_cast<int64_t>(T.n + TILE) * k;   // x_lo after x_hi, laid out for this k
    {
        const int64_t m = T.n * k;
        const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, static_cast<int64_t>(h->num_sms) * 8)));
        k_split64<<<blocks, 256, 0, s>>>(m, D.xs_stride, X, D.xs, D.xs + D.xs_stride);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    switch (k) {
#define DF_CASE(KK) case KK: return launch_df<KK>(h, Y, s);
        DF_CASE(2) DF_CASE(4) DF_CASE(6) DF_CASE(8) DF_CASE(10) DF_CASE(12) DF_CASE(14) DF_CASE(16)
        DF_CASE(18) DF_CASE(20) DF_CASE(22) DF_CASE(24) DF_CASE(26) DF_CASE(28) DF_CASE(30) DF_CASE(32)
#undef DF_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lobpcg
