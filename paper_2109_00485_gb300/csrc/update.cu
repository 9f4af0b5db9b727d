// The LOBPCG update after the Rayleigh-Ritz step and the residual of the
// next iteration, in one pass over the blocks (float32, k = 8, 16 or 20):
//
//   X  <- S C,            HX <- HS C            (eqs. xupd, upd1)
//   P  <- S[:, k:] C[k:], HP <- HS[:, k:] C[k:] (eqs. pupd, upd2)
//   R  =  HX - X Theta                          (Algorithm 1, line 10)
//   W  =  R, or R / g(d - theta_j) per column   (line 6 with 1x1 tiles)
//
// with S = [X W P] (or [X W] without a P block), HS = [HX HW HP], C the
// (na k) x k Ritz coefficients (FP64, rounded to float32), and the column
// sums ||r_j||^2, ||x_j||^2 (norms) and ||p_j||^2 (colsq) in FP64.  X, P,
// HX, HP and W are overwritten in place: a tile's input rows are staged in
// shared memory before any of its outputs is written, and every row is read
// once.
//
// The same coefficient column serves all four outputs (P uses the lower rows
// of C), so a thread keeps column j of C in registers and computes, per row,
// p = S[k:] C[k:, j] and x = p + S[:k] C[:k, j] (and hp, hx from HS): 2 na k
// FMAs for four outputs.  Rows are staged by a producer warp in tiles of 128
// rows per block (bulk copies completing on an mbarrier, 4 KB pieces: a
// tile's handshake is a fixed cost, 8 KB or more per block keeps the six
// streams at HBM speed), into up to four stages; consumer warps release a
// stage on its `empty` mbarrier.  Waits are bounded; on a timeout the kernel
// records DEV_TIMEOUT, lets its copies land and returns.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"

namespace lobpcg {

namespace {

constexpr int UP_ROWS = 128;
constexpr int UP_MAXSTAGES = 4;
constexpr int UP_CONS = 16;                  // consumer warps
constexpr int UP_THREADS = 32 * (UP_CONS + 1);

struct UpArgs {
    int64_t n;
    int na, mode, stages;
    const float *in[6];          // S blocks (na), then HS blocks (na)
    float *X, *P, *HX, *HP, *W;  // outputs
    const double *C, *theta;
    const float *d;
    double *norms, *colsq;
    int *err;
};

template <int K, int NA>
__global__ void __launch_bounds__(UP_THREADS, 1) k_update_post(const __grid_constant__ UpArgs a) {
    extern __shared__ __align__(16) float up_smem[];
    __shared__ __align__(8) uint64_t full[UP_MAXSTAGES], empty[UP_MAXSTAGES];
    __shared__ double red[3 * K];
    __shared__ int abort_flag;
    const int NS = a.stages;
    constexpr int nblk = 2 * NA;
    constexpr int TILE_F = UP_ROWS * K;                    // floats per block and tile
    const int stage_f = nblk * TILE_F + UP_ROWS;           // + the tile's diagonal entries
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntile = (a.n + UP_ROWS - 1) / UP_ROWS;
    const int my_tiles = (blockIdx.x < ntile) ? static_cast<int>((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], UP_CONS);
        }
        abort_flag = 0;
        fence_proxy_async();
    }
    for (int q = threadIdx.x; q < 3 * K; q += blockDim.x) red[q] = 0.0;
    __syncthreads();

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            bool bad = false;
            int issued = 0;
            for (int i = 0; i < my_tiles; ++i) {
                const int s = i % NS;
                if (i >= NS && !mbar_wait_sleep_bounded(&empty[s], ((i / NS) - 1) & 1)) {
                    bad = true;
                    break;
                }
                if (*reinterpret_cast<volatile int *>(&abort_flag)) break;
                const int64_t r0 = (blockIdx.x + static_cast<int64_t>(i) * gridDim.x) * UP_ROWS;
                const int rows = static_cast<int>(a.n - r0 < UP_ROWS ? a.n - r0 : UP_ROWS);
                const uint32_t bytes = static_cast<uint32_t>(rows * K) * 4u;
                // the diagonal entries of the tile's rows, rounded up to 4
                // (the diagonal array is padded for it); consumers read them
                // from shared memory: a global load before the stage release
                // (an mbarrier arrive, with release semantics) would wait a
                // memory round trip per tile
                const uint32_t dbytes = a.mode == 1 ? static_cast<uint32_t>((rows + 3) / 4 * 4) * 4u : 0u;
                mbar_arrive_expect_tx(&full[s], bytes * static_cast<uint32_t>(nblk) + dbytes);
                for (int q = 0; q < nblk; ++q) {
                    const char *src = reinterpret_cast<const char *>(a.in[q] + r0 * K);
                    char *dst = reinterpret_cast<char *>(up_smem + s * stage_f + q * TILE_F);
                    for (uint32_t o = 0; o < bytes; o += 4096u)
                        bulk_g2s(dst + o, src + o, bytes - o < 4096u ? bytes - o : 4096u, &full[s], pol);
                }
                if (dbytes) bulk_g2s(up_smem + s * stage_f + nblk * TILE_F, a.d + r0, dbytes, &full[s], pol);
                issued = i + 1;
            }
            if (bad) {
                atomicExch(a.err, DEV_TIMEOUT);
                abort_flag = 1;
            }
            for (int i = (issued > NS ? issued - NS : 0); i < issued; ++i)
                mbar_wait_bounded(&full[i % NS], (i / NS) & 1);
        }
    } else {
        // ---------------------------------------------------------- consumers
        const int ct = threadIdx.x - 32;
        constexpr int G = (UP_CONS * 32) / K;              // row groups
        const int j = ct % K, g = ct / K;
        const bool act = g < G;
        float c[NA * K];
#pragma unroll
        for (int q = 0; q < NA * K; ++q) c[q] = static_cast<float>(a.C[q * K + j]);
        const float th = static_cast<float>(a.theta[j]);
        const float delta = 1e-3f * (fabsf(th) > 1.f ? fabsf(th) : 1.f);
        double rr_d = 0.0, xx_d = 0.0, pp_d = 0.0;
        float rr_f = 0.f, xx_f = 0.f, pp_f = 0.f;
        bool bad = false;
        for (int i = 0; i < my_tiles; ++i) {
            const int s = i % NS;
            if (!mbar_wait_sleep_bounded(&full[s], (i / NS) & 1)) bad = true;
            if (__any_sync(0xffffffffu, bad) || *reinterpret_cast<volatile int *>(&abort_flag)) {
                bad = true;
                break;
            }
            const int64_t r0 = (blockIdx.x + static_cast<int64_t>(i) * gridDim.x) * UP_ROWS;
            const int rows = static_cast<int>(a.n - r0 < UP_ROWS ? a.n - r0 : UP_ROWS);
            const float *st = up_smem + s * stage_f;
            float rr = 0.f, xx = 0.f, pp = 0.f;
            if (act) {
                const float *sd = st + nblk * TILE_F;   // the tile's diagonal entries
#pragma unroll 1
                for (int r = g; r < rows; r += G) {
                    // the S and HS rows block by block, P blocks first (p is
                    // the partial sum of x), each block's 4-vectors loaded
                    // before its FMAs; packed pairs (even and odd columns)
                    float2 p2 = make_float2(0.f, 0.f), hp2 = p2;
#pragma unroll
                    for (int q = 1; q < NA; ++q) {
                        float4 v[K / 4], w[K / 4];
                        const float4 *sr = reinterpret_cast<const float4 *>(st + q * TILE_F + r * K);
                        const float4 *hr = reinterpret_cast<const float4 *>(st + (NA + q) * TILE_F + r * K);
#pragma unroll
                        for (int c4 = 0; c4 < K / 4; ++c4) v[c4] = sr[c4];
#pragma unroll
                        for (int c4 = 0; c4 < K / 4; ++c4) w[c4] = hr[c4];
#pragma unroll
                        for (int c4 = 0; c4 < K / 4; ++c4) {
                            const int cc = q * K + 4 * c4;
                            const float2 c01 = make_float2(c[cc], c[cc + 1]), c23 = make_float2(c[cc + 2], c[cc + 3]);
                            p2 = fma2(make_float2(v[c4].x, v[c4].y), c01, p2);
                            hp2 = fma2(make_float2(w[c4].x, w[c4].y), c01, hp2);
                            p2 = fma2(make_float2(v[c4].z, v[c4].w), c23, p2);
                            hp2 = fma2(make_float2(w[c4].z, w[c4].w), c23, hp2);
                        }
                    }
                    const float p = p2.x + p2.y, hp = hp2.x + hp2.y;
                    float2 x2 = make_float2(p, 0.f), hx2 = make_float2(hp, 0.f);
                    {
                        float4 v[K / 4], w[K / 4];
                        const float4 *sr = reinterpret_cast<const float4 *>(st + r * K);
                        const float4 *hr = reinterpret_cast<const float4 *>(st + NA * TILE_F + r * K);
#pragma unroll
                        for (int c4 = 0; c4 < K / 4; ++c4) v[c4] = sr[c4];
#pragma unroll
                        for (int c4 = 0; c4 < K / 4; ++c4) w[c4] = hr[c4];
#pragma unroll
                        for (int c4 = 0; c4 < K / 4; ++c4) {
                            const int cc = 4 * c4;
                            const float2 c01 = make_float2(c[cc], c[cc + 1]), c23 = make_float2(c[cc + 2], c[cc + 3]);
                            x2 = fma2(make_float2(v[c4].x, v[c4].y), c01, x2);
                            hx2 = fma2(make_float2(w[c4].x, w[c4].y), c01, hx2);
                            x2 = fma2(make_float2(v[c4].z, v[c4].w), c23, x2);
                            hx2 = fma2(make_float2(w[c4].z, w[c4].w), c23, hx2);
                        }
                    }
                    const float x = x2.x + x2.y, hx = hx2.x + hx2.y;
                    const int64_t e = (r0 + r) * K + j;
                    const float res = hx - x * th;
                    float w = res;
                    if (a.mode == 1) {
                        const float t = sd[r] - th;   // guarded shifted pivot g(t)
                        const float gp = (t >= 0.f) ? (t > delta ? t : delta) : (-t > delta ? t : -delta);
                        w = res * __frcp_rn(gp);      // a search direction: two roundings are enough
                    }
                    a.X[e] = x;
                    a.P[e] = p;
                    a.HX[e] = hx;
                    a.HP[e] = hp;
                    a.W[e] = w;
                    rr = fmaf(res, res, rr);
                    xx = fmaf(x, x, xx);
                    pp = fmaf(p, p, pp);
                }
            }
            rr_f += rr;
            xx_f += xx;
            pp_f += pp;
            if ((i & 3) == 3 || i == my_tiles - 1) {   // FP64 every 4 tiles (<= 16 rows in float)
                rr_d += static_cast<double>(rr_f);
                xx_d += static_cast<double>(xx_f);
                pp_d += static_cast<double>(pp_f);
                rr_f = xx_f = pp_f = 0.f;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (bad && lane == 0) {
            atomicExch(a.err, DEV_TIMEOUT);
            abort_flag = 1;
        }
        if (act && !bad) {
            atomicAdd(&red[j], rr_d);
            atomicAdd(&red[K + j], xx_d);
            atomicAdd(&red[2 * K + j], pp_d);
        }
    }
    __syncthreads();
    if (*reinterpret_cast<volatile int *>(&abort_flag)) return;
    for (int q = threadIdx.x; q < 2 * K; q += blockDim.x) atomicAdd(&a.norms[q], red[q]);
    for (int q = threadIdx.x; q < K; q += blockDim.x) atomicAdd(&a.colsq[q], red[2 * K + q]);
}

// Z = [A_0 .. A_{na-1}] C (na <= 3 blocks, one output, float32), in place
// (Z may be one of the A blocks): the same staging as k_update_post, a
// thread per output column with its column of C in registers.
struct LcArgs {
    int64_t n;
    int na, stages, rows_t;      // rows per tile: about 48 KB of inputs per tile
    const float *in[3];
    float *Z;
    const double *C;             // (na K) x K, row-major
    int *err;
};

template <int K, int NA>
__global__ void __launch_bounds__(UP_THREADS, 1) k_combine_ff(const __grid_constant__ LcArgs a) {
    extern __shared__ __align__(16) float lc_smem[];
    __shared__ __align__(8) uint64_t full[UP_MAXSTAGES], empty[UP_MAXSTAGES];
    __shared__ int abort_flag;
    const int NS = a.stages, TR = a.rows_t;
    const int TILE_F = TR * K;
    const int stage_f = NA * TILE_F;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntile = (a.n + TR - 1) / TR;
    const int my_tiles = (blockIdx.x < ntile) ? static_cast<int>((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], UP_CONS);
        }
        abort_flag = 0;
        fence_proxy_async();
    }
    __syncthreads();
    if (warp == 0) {
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            bool bad = false;
            int issued = 0;
            for (int i = 0; i < my_tiles; ++i) {
                const int s = i % NS;
                if (i >= NS && !mbar_wait_sleep_bounded(&empty[s], ((i / NS) - 1) & 1)) {
                    bad = true;
                    break;
                }
                if (*reinterpret_cast<volatile int *>(&abort_flag)) break;
                const int64_t r0 = (blockIdx.x + static_cast<int64_t>(i) * gridDim.x) * TR;
                const int rows = static_cast<int>(a.n - r0 < TR ? a.n - r0 : TR);
                const uint32_t bytes = static_cast<uint32_t>(rows * K) * 4u;
                mbar_arrive_expect_tx(&full[s], bytes * static_cast<uint32_t>(NA));
                for (int q = 0; q < NA; ++q) {
                    const char *src = reinterpret_cast<const char *>(a.in[q] + r0 * K);
                    char *dst = reinterpret_cast<char *>(lc_smem + s * stage_f + q * TILE_F);
                    for (uint32_t o = 0; o < bytes; o += 4096u)
                        bulk_g2s(dst + o, src + o, bytes - o < 4096u ? bytes - o : 4096u, &full[s], pol);
                }
                issued = i + 1;
            }
            if (bad) {
                atomicExch(a.err, DEV_TIMEOUT);
                abort_flag = 1;
            }
            for (int i = (issued > NS ? issued - NS : 0); i < issued; ++i)
                mbar_wait_bounded(&full[i % NS], (i / NS) & 1);
        }
    } else {
        const int ct = threadIdx.x - 32;
        constexpr int G = (UP_CONS * 32) / K;
        const int j = ct % K, g = ct / K;
        const bool act = g < G;
        float c[NA * K];
#pragma unroll
        for (int q = 0; q < NA * K; ++q) c[q] = static_cast<float>(a.C[q * K + j]);
        // rows per step: every row's 4-vectors are loaded before any FMA, so
        // a thread has RPS independent chains in flight (the loop is bound by
        // the shared-load latency otherwise)
        constexpr int RPS = NA == 1 ? 4 : (NA == 2 ? 2 : 1);
        bool bad = false;
        for (int i = 0; i < my_tiles; ++i) {
            const int s = i % NS;
            if (!mbar_wait_sleep_bounded(&full[s], (i / NS) & 1)) bad = true;
            if (__any_sync(0xffffffffu, bad) || *reinterpret_cast<volatile int *>(&abort_flag)) {
                bad = true;
                break;
            }
            const int64_t r0 = (blockIdx.x + static_cast<int64_t>(i) * gridDim.x) * TR;
            const int rows = static_cast<int>(a.n - r0 < TR ? a.n - r0 : TR);
            const float *st = lc_smem + s * stage_f;
            if (act) {
#pragma unroll 1
                for (int r = g; r < rows; r += RPS * G) {
                    float4 v[RPS][NA * (K / 4)];
#pragma unroll
                    for (int u = 0; u < RPS; ++u) {
                        const int ru = r + u * G < rows ? r + u * G : r;   // past the tile: reload row r
#pragma unroll
                        for (int q = 0; q < NA; ++q) {
                            const float4 *sr = reinterpret_cast<const float4 *>(st + q * TILE_F + ru * K);
#pragma unroll
                            for (int c4 = 0; c4 < K / 4; ++c4) v[u][q * (K / 4) + c4] = sr[c4];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < RPS; ++u) {
                        // packed pairs: (v.x, v.y) (c0, c1) and (v.z, v.w) (c2, c3)
                        float2 z = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c4 = 0; c4 < NA * (K / 4); ++c4) {
                            z = fma2(make_float2(v[u][c4].x, v[u][c4].y), make_float2(c[4 * c4], c[4 * c4 + 1]), z);
                            z = fma2(make_float2(v[u][c4].z, v[u][c4].w), make_float2(c[4 * c4 + 2], c[4 * c4 + 3]), z);
                        }
                        if (r + u * G < rows) a.Z[(r0 + r + u * G) * K + j] = z.x + z.y;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        if (bad && lane == 0) {
            atomicExch(a.err, DEV_TIMEOUT);
            abort_flag = 1;
        }
    }
}

template <int K, int NA>
cudaError_t launch_lc(const LcArgs &a0, int num_sms, cudaStream_t s) {
    LcArgs a = a0;
    // about 48 KB of inputs per tile (a multiple of the row groups so full
    // tiles split evenly): a tile's handshake is a fixed cost
    constexpr int G = (UP_CONS * 32) / K;
    a.rows_t = std::max(G, (49152 / (a.na * K * 4)) / G * G);
    const size_t stage_bytes = sizeof(float) * a.na * a.rows_t * K;
    a.stages = static_cast<int>(std::min<size_t>(UP_MAXSTAGES, (192u * 1024u) / stage_bytes));
    if (a.stages < 2) return cudaErrorInvalidValue;
    const size_t smem = a.stages * stage_bytes;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_combine_ff<K, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t ntile = (a.n + a.rows_t - 1) / a.rows_t;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ntile, num_sms)));
    k_combine_ff<K, NA><<<blocks, UP_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <int K, int NA>
cudaError_t launch_k(const UpArgs &a0, int num_sms, cudaStream_t s) {
    UpArgs a = a0;
    const size_t stage_bytes = sizeof(float) * (2 * a.na * UP_ROWS * K + UP_ROWS);
    a.stages = static_cast<int>(std::min<size_t>(UP_MAXSTAGES, (196u * 1024u) / stage_bytes));
    if (a.stages < 2) return cudaErrorInvalidValue;
    const size_t smem = a.stages * stage_bytes;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_update_post<K, NA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t ntile = (a.n + UP_ROWS - 1) / UP_ROWS;
    const int blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(ntile, num_sms)));
    k_update_post<K, NA><<<blocks, UP_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool combine_ff_ok(int k, int na, const float *const *blocks, const float *Z) {
    if (!(k == 8 || k == 16 || k == 20) || na < 1 || na > 3 || !Z || (reinterpret_cast<uintptr_t>(Z) & 15u))
        return false;
    for (int q = 0; q < na; ++q)
        if (!blocks[q] || (reinterpret_cast<uintptr_t>(blocks[q]) & 15u)) return false;
    return true;
}

cudaError_t launch_combine_ff(int64_t n, int k, int na, const float *const *A, const double *C, float *Z, int *err,
                              int num_sms, cudaStream_t s) {
    LcArgs a{};
    a.n = n;
    a.na = na;
    for (int q = 0; q < na; ++q) a.in[q] = A[q];
    a.Z = Z;
    a.C = C;
    a.err = err;
    switch (k * 4 + na) {
        case 8 * 4 + 1: return launch_lc<8, 1>(a, num_sms, s);
        case 8 * 4 + 2: return launch_lc<8, 2>(a, num_sms, s);
        case 8 * 4 + 3: return launch_lc<8, 3>(a, num_sms, s);
        case 16 * 4 + 1: return launch_lc<16, 1>(a, num_sms, s);
        case 16 * 4 + 2: return launch_lc<16, 2>(a, num_sms, s);
        case 16 * 4 + 3: return launch_lc<16, 3>(a, num_sms, s);
        case 20 * 4 + 1: return launch_lc<20, 1>(a, num_sms, s);
        case 20 * 4 + 2: return launch_lc<20, 2>(a, num_sms, s);
        case 20 * 4 + 3: return launch_lc<20, 3>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

bool update_post_ok(int k, int na, const float *const *blocks) {
    if (!(k == 8 || k == 16 || k == 20) || (na != 2 && na != 3)) return false;
    for (int q = 0; q < 2 * na; ++q)
        if (!blocks[q] || (reinterpret_cast<uintptr_t>(blocks[q]) & 15u)) return false;
    return true;
}

cudaError_t launch_update_post(int64_t n, int k, int na, const float *const *S, const float *const *HS,
                               float *X, float *P, float *HX, float *HP, float *W, const double *C,
                               const double *theta, const float *d, int mode, double *norms, double *colsq,
                               int *err, int num_sms, cudaStream_t s) {
    UpArgs a{};
    a.n = n;
    a.na = na;
    a.mode = mode;
    for (int q = 0; q < na; ++q) {
        a.in[q] = S[q];
        a.in[na + q] = HS[q];
    }
    a.X = X; a.P = P; a.HX = HX; a.HP = HP; a.W = W;
    a.C = C;
    a.theta = theta;
    a.d = d;
    a.norms = norms;
    a.colsq = colsq;
    a.err = err;
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * k, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(colsq, 0, sizeof(double) * k, s);
    if (e != cudaSuccess) return e;
    switch (k * 4 + na) {
        case 8 * 4 + 2: return launch_k<8, 2>(a, num_sms, s);
        case 8 * 4 + 3: return launch_k<8, 3>(a, num_sms, s);
        case 16 * 4 + 2: return launch_k<16, 2>(a, num_sms, s);
        case 16 * 4 + 3: return launch_k<16, 3>(a, num_sms, s);
        case 20 * 4 + 2: return launch_k<20, 2>(a, num_sms, s);
        case 20 * 4 + 3: return launch_k<20, 3>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lobpcg
