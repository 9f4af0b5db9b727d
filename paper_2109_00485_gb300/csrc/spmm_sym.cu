// Symmetric SpMM  Y = H X  from the stored lower triangle, one pass.
//
// Every stored h_ij (j <= i) contributes h_ij x_j to y_i (the triangle,
// Algorithm 2) and, for j < i, h_ij x_i to y_j (its transpose, Section 3.3).
// The paper runs the two as separate loops (Section 3.2) for overlap with
// MPI; on one GPU both are applied while the entry sits in shared memory.
//
// Work unit: one "chunk" = the entries of one row block (16 rows) that fall
// in one 16-column tile, streamed HBM -> shared memory by bulk (TMA) copies
// together with the 16 rows of X the tile's columns select.  Per chunk a
// warp forms the 16x16 tile H_t (dense, zero-filled when partial) and its
// transpose in shared memory, then
//     Y_R += H_t X_C     (rows of this row block; kept in registers)
//     Y_C  = H_t^T X_R   (rows of the tile's columns; vector atomics to L2)
// X_R (this row block's 16 rows of X) is held in registers for the row
// block.  The diagonal chunk is expanded to the symmetric tile S = L + L^T - D
// and applied as Y_R += S X_R.  Y_R is flushed once per row block with
// vector atomics, since other warps add transposed parts to the same rows.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"
#include "internal.h"

namespace lobpcg {

template <int K>
struct SpmmCfg {
    static constexpr int GK = K / 4;      // lanes along k (groups of 4 columns)
    static constexpr int RPL = K / 8;     // rows (and tile columns) per lane
    static constexpr int STAGES = 3;
    static constexpr int WARPS = 8;
    static constexpr int MINB = (K <= 16) ? 2 : 1;
};

template <int K>
struct __align__(16) WarpSmem {
    float vals[SpmmCfg<K>::STAGES][256];
    uint32_t idx[SpmmCfg<K>::STAGES][256];
    float xt[SpmmCfg<K>::STAGES][TILE * K];
    float H[256];         // row-major tile for partially filled chunks
    float HT[TILE * 18];  // transposed tile (stride 18: conflict-free scatter and pair loads)
    int4 meta[SpmmCfg<K>::STAGES];   // column tile, info, padded count, valid rows
    uint64_t bar[SpmmCfg<K>::STAGES];
};

struct SpmmArgs {
    int64_t n;
    int k;
    const uint32_t *idx;
    const float *val;
    const int64_t *chunk_off;
    const int32_t *chunk_ct;
    const int32_t *chunk_info;
    const int64_t *rb_chunk;
    const int32_t *warp_rb;
    int W;
    const float *X;
    float *Y;
    int *err;
};

template <int K>
__device__ __forceinline__ void issue_chunk(const SpmmArgs &a, WarpSmem<K> *ws, int64_t c, int s,
                                            uint64_t pol_stream, uint64_t pol_keep) {
    const int64_t off = a.chunk_off[c];
    const int npad = static_cast<int>(a.chunk_off[c + 1] - off);
    const int ct = a.chunk_ct[c];
    const int info = a.chunk_info[c];
    const int64_t r0 = static_cast<int64_t>(ct) * TILE;
    const int rows = static_cast<int>(a.n - r0 < TILE ? a.n - r0 : TILE);
    const uint32_t xbytes = static_cast<uint32_t>(rows) * a.k * 4u;
    ws->meta[s] = make_int4(ct, info, npad, rows);
    mbar_arrive_expect_tx(&ws->bar[s], static_cast<uint32_t>(npad) * 8u + xbytes);
    if (npad > 0) {
        bulk_g2s(ws->vals[s], a.val + off, npad * 4u, &ws->bar[s], pol_stream);
        bulk_g2s(ws->idx[s], a.idx + off, npad * 4u, &ws->bar[s], pol_stream);
    }
    bulk_g2s(ws->xt[s], a.X + r0 * a.k, xbytes, &ws->bar[s], pol_keep);
}

template <int K>
__global__ void __launch_bounds__(SpmmCfg<K>::WARPS * 32, SpmmCfg<K>::MINB) k_spmm_sym_tiled(SpmmArgs a) {
    using C = SpmmCfg<K>;
    constexpr int RPL = C::RPL, GK = C::GK, S = C::STAGES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * C::WARPS + warp;
    if (gw >= a.W) return;
    WarpSmem<K> *ws = reinterpret_cast<WarpSmem<K> *>(smem_raw) + warp;
    const int rb0 = a.warp_rb[gw], rb1 = a.warp_rb[gw + 1];
    if (rb0 >= rb1) return;
    const int64_t c0 = a.rb_chunk[rb0], c1 = a.rb_chunk[rb1];
    const int kg = lane % GK, rg = lane / GK;
    const bool kact = kg * 4 < a.k;
    const int k = a.k;

    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&ws->bar[s], 1);
        fence_proxy_async();
    }
    __syncwarp();
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();
    if (lane == 0)
        for (int s = 0; s < S; ++s)
            if (c0 + s < c1) issue_chunk<K>(a, ws, c0 + s, s, pol_stream, pol_keep);

    float xr[TILE][4];
    float yr[RPL][4];
#pragma unroll
    for (int j = 0; j < RPL; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q) yr[j][q] = 0.f;
#pragma unroll
    for (int r = 0; r < TILE; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) xr[r][q] = 0.f;
    int64_t cur_rb = -1;
    uint32_t phases = 0;

    auto flush_yr = [&](int64_t rb) {
        if (!kact) return;
#pragma unroll
        for (int j = 0; j < RPL; ++j) {
            const int64_t row = rb * TILE + rg * RPL + j;
            if (row < a.n) red_add_v4(a.Y + row * k + kg * 4, yr[j][0], yr[j][1], yr[j][2], yr[j][3]);
        }
    };

    for (int64_t c = c0; c < c1; ++c) {
        const int s = static_cast<int>((c - c0) % S);
        const bool ok = mbar_wait_bounded(&ws->bar[s], (phases >> s) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(a.err, DEV_TIMEOUT);
            // let copies already in flight land before the warp leaves
            for (int64_t cc = c; cc < c1 && cc < c + S; ++cc) {
                const int ss = static_cast<int>((cc - c0) % S);
                mbar_wait_bounded(&ws->bar[ss], (phases >> ss) & 1u);
            }
            return;
        }
        phases ^= 1u << s;
        const int4 m = ws->meta[s];
        const int ct = m.x, cnt = m.y & 0xFFFF, rows = m.w;
        const bool is_diag = (m.y & DIAG_FLAG) != 0;
        const float *xt = ws->xt[s];

        if (is_diag) {
            if (cur_rb >= 0) flush_yr(cur_rb);
            cur_rb = ct;
#pragma unroll
            for (int j = 0; j < RPL; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) yr[j][q] = 0.f;
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (kact && r < rows) v = *reinterpret_cast<const float4 *>(xt + r * k + kg * 4);
                xr[r][0] = v.x; xr[r][1] = v.y; xr[r][2] = v.z; xr[r][3] = v.w;
            }
            // symmetric tile S = L + L^T - D of the diagonal block, in HT
            for (int e = lane; e < TILE * 18; e += 32) ws->HT[e] = 0.f;
            __syncwarp();
            for (int e = lane; e < cnt; e += 32) {
                const uint32_t u = ws->idx[s][e];
                const float v = ws->vals[s][e];
                const int rl = (u >> 28) & 15, cl = u & 15;
                ws->HT[rl * 18 + cl] = v;
                ws->HT[cl * 18 + rl] = v;
            }
            __syncwarp();
#pragma unroll
            for (int cc = 0; cc < TILE; ++cc) {
                float sv[RPL];
#pragma unroll
                for (int j = 0; j < RPL; ++j) sv[j] = ws->HT[cc * 18 + rg * RPL + j];
#pragma unroll
                for (int j = 0; j < RPL; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) yr[j][q] = fmaf(sv[j], xr[cc][q], yr[j][q]);
            }
        } else {
            const bool full = (cnt == 256);
            const float *Hp = full ? ws->vals[s] : ws->H;
            if (!full) {
                for (int e = lane; e < 256; e += 32) ws->H[e] = 0.f;
                for (int e = lane; e < TILE * 18; e += 32) ws->HT[e] = 0.f;
                __syncwarp();
            }
            for (int e = lane; e < cnt; e += 32) {
                const uint32_t u = ws->idx[s][e];
                const float v = ws->vals[s][e];
                const int rl = (u >> 28) & 15, cl = u & 15;
                ws->HT[cl * 18 + rl] = v;
                if (!full) ws->H[rl * 16 + cl] = v;
            }
            __syncwarp();
            // Y_R += H_t X_C
#pragma unroll
            for (int cc = 0; cc < TILE; ++cc) {
                float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                if (kact) x = *reinterpret_cast<const float4 *>(xt + cc * k + kg * 4);
                float hv[RPL];
#pragma unroll
                for (int j = 0; j < RPL; ++j) hv[j] = ws->HT[cc * 18 + rg * RPL + j];
#pragma unroll
                for (int j = 0; j < RPL; ++j) {
                    yr[j][0] = fmaf(hv[j], x.x, yr[j][0]);
                    yr[j][1] = fmaf(hv[j], x.y, yr[j][1]);
                    yr[j][2] = fmaf(hv[j], x.z, yr[j][2]);
                    yr[j][3] = fmaf(hv[j], x.w, yr[j][3]);
                }
            }
            // Y_C = H_t^T X_R
            float yc[RPL][4];
#pragma unroll
            for (int j = 0; j < RPL; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) yc[j][q] = 0.f;
#pragma unroll
            for (int r = 0; r < TILE; ++r) {
                float hv[RPL];
#pragma unroll
                for (int j = 0; j < RPL; ++j) hv[j] = Hp[r * 16 + rg * RPL + j];
#pragma unroll
                for (int j = 0; j < RPL; ++j)
#pragma unroll
                    for (int q = 0; q < 4; ++q) yc[j][q] = fmaf(hv[j], xr[r][q], yc[j][q]);
            }
            if (kact) {
#pragma unroll
                for (int j = 0; j < RPL; ++j) {
                    const int64_t row = static_cast<int64_t>(ct) * TILE + rg * RPL + j;
                    red_add_v4(a.Y + row * k + kg * 4, yc[j][0], yc[j][1], yc[j][2], yc[j][3]);
                }
            }
        }
        __syncwarp();
        if (lane == 0 && c + S < c1) {
            fence_proxy_async();
            issue_chunk<K>(a, ws, c + S, s, pol_stream, pol_keep);
        }
    }
    if (cur_rb >= 0) flush_yr(cur_rb);
}

// ---------------------------------------------------------------------------
// Simple kernel for any k (1..32) and any alignment, float or double vectors:
// one warp per row block, tile and its transpose in shared memory, X rows
// read with plain loads, transposed parts added with scalar atomics.  Used
// for k % 4 != 0, unaligned pointers and the FP64 (check / polish) product.
template <typename T>
struct SimpleSmem {
    float H[256];
    float HT[TILE * 17];
    T xr[TILE * 32];
    T xc[TILE * 32];
};

template <typename T>
__global__ void __launch_bounds__(256) k_spmm_sym_simple(int64_t n, int k, const uint32_t *idx, const float *val,
                                                         const int64_t *chunk_off, const int32_t *chunk_ct,
                                                         const int32_t *chunk_info, const int64_t *rb_chunk,
                                                         int64_t R, const T *X, T *Y) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SimpleSmem<T> *ws = reinterpret_cast<SimpleSmem<T> *>(smem_raw) + warp;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const int nout = TILE * k;  // outputs of one row block: 16 rows x k
    for (int64_t rb = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + warp; rb < R; rb += nwarps) {
        const int rows = static_cast<int>(n - rb * TILE < TILE ? n - rb * TILE : TILE);
        for (int o = lane; o < nout; o += 32) {
            const int r = o / k, q = o % k;
            ws->xr[o] = (r < rows) ? X[(rb * TILE + r) * k + q] : T(0);
        }
        T acc[16];  // outputs o = lane + 32 t, t < 16 (16 x 32 / 32)
#pragma unroll
        for (int t = 0; t < 16; ++t) acc[t] = T(0);
        __syncwarp();
        for (int64_t c = rb_chunk[rb]; c < rb_chunk[rb + 1]; ++c) {
            const int64_t off = chunk_off[c];
            const int info = chunk_info[c];
            const int cnt = info & 0xFFFF;
            const bool is_diag = (info & DIAG_FLAG) != 0;
            const int64_t ct = chunk_ct[c];
            for (int e = lane; e < 256; e += 32) ws->H[e] = 0.f;
            for (int e = lane; e < TILE * 17; e += 32) ws->HT[e] = 0.f;
            __syncwarp();
            for (int e = lane; e < cnt; e += 32) {
                const uint32_t u = idx[off + e];
                const float v = val[off + e];
                const int rl = (u >> 28) & 15, cl = u & 15;
                ws->H[rl * 16 + cl] = v;
                if (is_diag) ws->H[cl * 16 + rl] = v;
                else ws->HT[cl * 17 + rl] = v;
            }
            if (!is_diag)
                for (int o = lane; o < nout; o += 32) ws->xc[o] = X[(ct * TILE) * k + o];
            __syncwarp();
            const T *xs = is_diag ? ws->xr : ws->xc;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int o = lane + 32 * t;
                if (o < nout) {
                    const int r = o / k, q = o % k;
                    T sum = T(0);
                    for (int cc = 0; cc < TILE; ++cc) sum += static_cast<T>(ws->H[r * 16 + cc]) * xs[cc * k + q];
                    acc[t] += sum;
                }
            }
            if (!is_diag) {
                for (int o = lane; o < nout; o += 32) {
                    const int cl = o / k, q = o % k;
                    T sum = T(0);
                    for (int r = 0; r < TILE; ++r) sum += static_cast<T>(ws->HT[cl * 17 + r]) * ws->xr[r * k + q];
                    atomicAdd(Y + (ct * TILE + cl) * k + q, sum);
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int o = lane + 32 * t;
            if (o < nout) {
                const int r = o / k, q = o % k;
                if (r < rows) atomicAdd(Y + (rb * TILE + r) * k + q, acc[t]);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------

template <int K>
static cudaError_t launch_tiled(const lobpcg_ctx *h, const float *X, float *Y, int k, cudaStream_t s) {
    using C = SpmmCfg<K>;
    const size_t smem = sizeof(WarpSmem<K>) * C::WARPS;
    static bool attr_set[64] = {false};
    int dev = h->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(k_spmm_sym_tiled<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr_set[dev & 63] = true;
    }
    SpmmArgs a;
    a.n = h->T.n; a.k = k; a.idx = h->T.idx; a.val = h->T.val; a.chunk_off = h->T.chunk_off;
    a.chunk_ct = h->T.chunk_ct; a.chunk_info = h->T.chunk_info; a.rb_chunk = h->T.rb_chunk;
    a.warp_rb = h->T.warp_rb; a.W = h->T.warps; a.X = X; a.Y = Y; a.err = h->d_err;
    const int blocks = (h->T.warps + C::WARPS - 1) / C::WARPS;
    k_spmm_sym_tiled<K><<<blocks, C::WARPS * 32, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_simple(const lobpcg_ctx *h, const T *X, T *Y, int k, cudaStream_t s) {
    const size_t smem = sizeof(SimpleSmem<T>) * 8;
    static bool attr_set[64] = {false};
    int dev = h->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(k_spmm_sym_simple<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr_set[dev & 63] = true;
    }
    const int64_t R = h->T.R;
    int blocks = static_cast<int>(std::min<int64_t>((R + 7) / 8, static_cast<int64_t>(h->num_sms) * 8));
    if (blocks < 1) blocks = 1;
    k_spmm_sym_simple<T><<<blocks, 256, smem, s>>>(h->T.n, k, h->T.idx, h->T.val, h->T.chunk_off, h->T.chunk_ct,
                                                   h->T.chunk_info, h->T.rb_chunk, R, X, Y);
    return cudaGetLastError();
}

cudaError_t launch_spmm_sym_f32(const lobpcg_ctx *h, const float *X, float *Y, int k, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(Y, 0, sizeof(float) * static_cast<size_t>(h->T.n) * k, s);
    if (e != cudaSuccess) return e;
    const bool aligned = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) == 0;
    if (aligned && k % 4 == 0) {
        if (k <= 8) return launch_tiled<8>(h, X, Y, k, s);
        if (k <= 16) return launch_tiled<16>(h, X, Y, k, s);
        return launch_tiled<32>(h, X, Y, k, s);
    }
    return launch_simple<float>(h, X, Y, k, s);
}

cudaError_t launch_spmm_sym_f64(const lobpcg_ctx *h, const double *X, double *Y, int k, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(Y, 0, sizeof(double) * static_cast<size_t>(h->T.n) * k, s);
    if (e != cudaSuccess) return e;
    return launch_simple<double>(h, X, Y, k, s);
}

}  // namespace lobpcg
