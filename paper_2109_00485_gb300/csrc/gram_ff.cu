// Gram blocks M = A^T B of tall-skinny float32 blocks (Section 3.4: the
// blocks of G = S^T HS and O = S^T S of eq. go, and Cholesky-QR's X^T W and
// W^T W) on the CUDA cores, for a list of (A-block, B-block) pairs.
//
// Each pair is a k x k product over all n rows.  The products a_i b_j are
// exact FP32 FMAs (no operand rounding), summed in FP32 over at most 64 of
// a lane's rows, then added into Kahan-compensated FP32 sums; the CTA sums
// go to the FP64 result with one atomic per entry.  For the Gram shapes of
// the iteration this needs about 8 FMA per byte read at k = 16 -- a little
// above the FP32 FMA : HBM byte balance of GB300 (40 T FMA/s : 6.7 TB/s),
// so exact products cost no more than the operand rounding a tensor-core
// split would need.
//
// Layout of the work: a lane owns a 4 x 4 sub-tile of one pair's output (a
// "unit"); a warp's two half-warps hold the same 16 units and take
// neighbouring rows, so each row needs two 16-byte shared loads per lane
// (a 4-vector of the A row and of the B row, broadcast within the
// half-warp, both rows in one 128-byte line) for 16 FMAs.  A pair flagged
// SYM (a diagonal block of a symmetric Gram) computes only its lower
// sub-tiles and writes each off-diagonal one twice (transposed); MIRROR
// writes the whole block again transposed at (co, ro) -- the Rayleigh-Ritz
// step averages M[i][j] and M[j][i], so a mirrored block counts once.
//
// One CTA per SM.  Rows are staged in tiles of about 48 KB (128 rows per
// distinct block for six blocks at k = 16, more for fewer) by bulk copies
// (TMA, 4 KB pieces, completing on an mbarrier) into up to eight stages; a
// producer warp refills a stage once every consumer warp has released it.
// Consumer warps: the unit warps times row groups (up to 24 warps), each
// group taking every other pair of rows.  Every wait is bounded; on a
// timeout the kernel records DEV_TIMEOUT, lets its copies in flight land
// and returns.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"

namespace lobpcg {

namespace {

constexpr int GF_MAXSTAGES = 8;
constexpr int GF_MAXBLK = 8;
constexpr int GF_MAXPAIRS = 16;
constexpr int GF_MAXWARPS = 24;                 // consumer warps per CTA
constexpr int GF_THREADS = 32 * (GF_MAXWARPS + 1);

struct GfArgs {
    int64_t n;
    int k, T;                    // T = k / 4 sub-tiles per side
    int rows_t;                  // rows per staged tile (a multiple of 64)
    int stages;
    int nblk;
    const float *blk[GF_MAXBLK];
    int npairs;
    int pa[GF_MAXPAIRS], pb[GF_MAXPAIRS], ro[GF_MAXPAIRS], co[GF_MAXPAIRS], flags[GF_MAXPAIRS];
    int mro[GF_MAXPAIRS], mco[GF_MAXPAIRS];
    int piece;                   // bytes per bulk copy (a tile's block run is cut into pieces)
    int units;                   // sum over pairs of their sub-tiles
    int wpg;                     // consumer warps per row group (ceil(units / 16))
    int groups;                  // row groups per CTA
    double *M;
    int ldm;
    int *err;
};

// Sub-tile (p, si, sj) of unit u (pairs in list order; in a pair, sub-tiles
// row by row, lower ones only for SYM pairs).
__device__ __forceinline__ bool unit_of(const GfArgs &a, int u, int &p, int &si, int &sj) {
    const int T = a.T;
    for (int q = 0; q < a.npairs; ++q) {
        const bool sym = a.flags[q] & GRAM_SYM;
        const int cnt = sym ? T * (T + 1) / 2 : T * T;
        if (u < cnt) {
            p = q;
            if (!sym) {
                si = u / T;
                sj = u % T;
            } else {
                int r = 0;
                while (u >= r + 1) {
                    u -= r + 1;
                    ++r;
                }
                si = r;
                sj = u;
            }
            return true;
        }
        u -= cnt;
    }
    return false;
}

// part[4 i + j] += x_i y_j, as packed pairs (x_i, x_i) (y_0, y_1) and
// (x_i, x_i) (y_2, y_3): eight fma.rn.f32x2 for the sixteen products
__device__ __forceinline__ void fma16(float (&part)[16], const float4 x, const float4 y) {
    const float xv[4] = {x.x, x.y, x.z, x.w};
    const float2 y01 = make_float2(y.x, y.y), y23 = make_float2(y.z, y.w);
#pragma unroll
    for (int i2 = 0; i2 < 4; ++i2) {
        const float2 xx = make_float2(xv[i2], xv[i2]);
        float2 a = fma2(xx, y01, make_float2(part[i2 * 4], part[i2 * 4 + 1]));
        float2 b = fma2(xx, y23, make_float2(part[i2 * 4 + 2], part[i2 * 4 + 3]));
        part[i2 * 4] = a.x;
        part[i2 * 4 + 1] = a.y;
        part[i2 * 4 + 2] = b.x;
        part[i2 * 4 + 3] = b.y;
    }
}

// Warp 0 is the producer (lane 0 issues the bulk copies of each tile into a
// free stage); warps 1.. consume.  A consumer warp waits for its tile's
// stage to fill, accumulates its rows, and releases the stage (one arrival
// per consumer warp on the stage's `empty` barrier); no CTA-wide barrier
// inside the loop, so a warp that finishes early runs ahead.
// 80 registers: 25 warps (800 threads) fit one SM's register file
__global__ void __maxnreg__(80) k_gram_ff(const __grid_constant__ GfArgs a) {
    extern __shared__ __align__(16) float gf_smem[];
    __shared__ __align__(8) uint64_t full[GF_MAXSTAGES], empty[GF_MAXSTAGES];
    const int k = a.k, TR = a.rows_t, NS = a.stages;
    const int tile_floats = TR * k;                           // one block's tile
    const int stage_floats = a.nblk * tile_floats;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncons = a.wpg * a.groups;                       // consumer warps
    const int64_t ntile = (a.n + TR - 1) / TR;
    const int my_tiles = (blockIdx.x < ntile) ? static_cast<int>((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], ncons);
        }
        abort_flag = 0;
        fence_proxy_async();
    }
    __syncthreads();

    float sum[16], cmp[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) sum[e] = cmp[e] = 0.f;
    const int cw = warp - 1;                                  // consumer index
    const int half = lane >> 4, hl = lane & 15;
    const int grp = cw / a.wpg, wig = cw % a.wpg;
    const int u = wig * 16 + hl;
    int p = 0, si = 0, sj = 0;
    const bool act = warp >= 1 && cw < ncons && u < a.units && unit_of(a, u, p, si, sj);

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
                const int64_t r0 = (blockIdx.x + static_cast<int64_t>(i) * gridDim.x) * TR;
                const int rows = static_cast<int>(a.n - r0 < TR ? a.n - r0 : TR);
                const uint32_t bytes = static_cast<uint32_t>(rows * k) * 4u;
                mbar_arrive_expect_tx(&full[s], bytes * static_cast<uint32_t>(a.nblk));
                for (int q = 0; q < a.nblk; ++q) {
                    const char *src = reinterpret_cast<const char *>(a.blk[q] + r0 * k);
                    char *dst = reinterpret_cast<char *>(gf_smem + s * stage_floats + q * tile_floats);
                    for (uint32_t o = 0; o < bytes; o += a.piece)
                        bulk_g2s(dst + o, src + o, bytes - o < static_cast<uint32_t>(a.piece) ? bytes - o : a.piece,
                                 &full[s], pol);
                }
                issued = i + 1;
            }
            if (bad) {
                atomicExch(a.err, DEV_TIMEOUT);
                abort_flag = 1;
            }
            // copies still landing must finish before the CTA's shared memory goes
            for (int i = (issued > NS ? issued - NS : 0); i < issued; ++i)
                mbar_wait_bounded(&full[i % NS], (i / NS) & 1);
        }
    } else if (cw < ncons) {
        // ---------------------------------------------------------- consumers
        const int offA = act ? a.pa[p] * tile_floats + 4 * si : 0;
        const int offB = act ? a.pb[p] * tile_floats + 4 * sj : 0;
        const int rstep = 2 * a.groups;                       // rows between a lane's rows
        const int rfirst = 2 * grp + half;
        float part[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) part[e] = 0.f;
        int since = 0;                                        // rows in part
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
            if (act) {
                const float *st = gf_smem + s * stage_floats;
                const float4 *pA = reinterpret_cast<const float4 *>(st + offA + rfirst * k);
                const float4 *pB = reinterpret_cast<const float4 *>(st + offB + rfirst * k);
                const int vstep = rstep * k / 4;                 // float4s between a lane's rows
                // this lane's rows: rfirst + m rstep < rows (a full tile: the
                // same count for every lane, rows_t being a multiple of rstep)
                const int cnt = rows > rfirst ? (rows - rfirst + rstep - 1) / rstep : 0;
                int m = 0;
                for (; m + 2 <= cnt; m += 2) {                    // two rows per step, loads first
                    const float4 x0 = pA[0], y0 = pB[0], x1 = pA[vstep], y1 = pB[vstep];
                    fma16(part, x0, y0);
                    fma16(part, x1, y1);
                    pA += 2 * vstep;
                    pB += 2 * vstep;
                }
                if (m < cnt) fma16(part, pA[0], pB[0]);
                since += cnt;
                if (since >= 64 || i == my_tiles - 1) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float yk = part[e] - cmp[e];
                        const float t = sum[e] + yk;
                        cmp[e] = (t - sum[e]) - yk;
                        sum[e] = t;
                        part[e] = 0.f;
                    }
                    since = 0;
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
    __syncthreads();
    if (*reinterpret_cast<volatile int *>(&abort_flag)) return;
    // every lane's sums into shared memory (entry-major, lanes contiguous:
    // no bank conflicts), then each entry summed over the row groups and the
    // two half-warps, one FP64 atomic per entry and CTA
    double *red = reinterpret_cast<double *>(gf_smem);
    const int U2 = a.units * 2;
    if (act) {
#pragma unroll
        for (int e = 0; e < 16; ++e)
            red[(grp * 16 + e) * U2 + u * 2 + half] = static_cast<double>(sum[e]) - static_cast<double>(cmp[e]);
    }
    __syncthreads();
    const int nred = a.units * 16;
    for (int e = threadIdx.x; e < nred; e += blockDim.x) {
        const int uu = e / 16, q = e % 16;
        int pp, ssi, ssj;
        if (!unit_of(a, uu, pp, ssi, ssj)) continue;
        double v = 0.0;
        for (int g = 0; g < a.groups; ++g) v += red[(g * 16 + q) * U2 + uu * 2] + red[(g * 16 + q) * U2 + uu * 2 + 1];
        const int i2 = q / 4, j2 = q % 4;
        const int row = a.ro[pp] * k + 4 * ssi + i2, col = a.co[pp] * k + 4 * ssj + j2;
        atomicAdd(&a.M[static_cast<int64_t>(row) * a.ldm + col], v);
        const int fl = a.flags[pp];
        if ((fl & GRAM_SYM) && ssi != ssj) {   // transposed inside the block
            const int row2 = a.ro[pp] * k + 4 * ssj + j2, col2 = a.co[pp] * k + 4 * ssi + i2;
            atomicAdd(&a.M[static_cast<int64_t>(row2) * a.ldm + col2], v);
        }
        if (fl & GRAM_MIRROR) {                // transposed at block (mro, mco)
            const int row2 = a.mro[pp] * k + 4 * ssj + j2, col2 = a.mco[pp] * k + 4 * ssi + i2;
            atomicAdd(&a.M[static_cast<int64_t>(row2) * a.ldm + col2], v);
        }
    }
}

}  // namespace

// Bytes per bulk copy: LOBPCG_GF_PIECE (a multiple of 16, 1024..65536)
// overrides the default for tuning.
int gf_piece_bytes() {
    static const int v = [] {
        const char *e = getenv("LOBPCG_GF_PIECE");
        const int x = e ? atoi(e) : 0;
        return (x >= 1024 && x <= 65536 && x % 16 == 0) ? x : 4096;
    }();
    return v;
}

// Consumer warps the kernel can launch with (its register use decides;
// 0 if the query fails).
int gf_max_consumers() {
    static int v = -1;
    if (v < 0) {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, k_gram_ff) != cudaSuccess) {
            cudaGetLastError();
            v = 0;
        } else {
            v = std::max(0, std::min(GF_MAXWARPS, fa.maxThreadsPerBlock / 32 - 1));
        }
    }
    return v;
}

bool gram_pairs_fit(int k, int nblk, const float *const *blk, int npairs, int units) {
    return gram_pairs_ok(k, nblk, blk, npairs) && units <= 16 * gf_max_consumers();
}

bool gram_pairs_ok(int k, int nblk, const float *const *blk, int npairs) {
    if (k % 4 != 0 || k < 4 || k > 32 || nblk < 1 || nblk > GF_MAXBLK || npairs < 1 || npairs > GF_MAXPAIRS)
        return false;
    for (int q = 0; q < nblk; ++q)
        if (!blk[q] || (reinterpret_cast<uintptr_t>(blk[q]) & 15u)) return false;
    return true;
}

cudaError_t launch_gram_pairs(int64_t n, int k, int nblk, const float *const *blk, int npairs, const GramPair *pairs,
                              double *M, int ldm, int ldm_rows, bool zero, int *err, int num_sms, cudaStream_t s) {
    if (!gram_pairs_ok(k, nblk, blk, npairs) || !err) return cudaErrorInvalidValue;
    GfArgs a{};
    a.n = n;
    a.k = k;
    a.T = k / 4;
    a.nblk = nblk;
    for (int q = 0; q < nblk; ++q) a.blk[q] = blk[q];
    a.npairs = npairs;
    a.units = 0;
    for (int q = 0; q < npairs; ++q) {
        a.pa[q] = pairs[q].a;
        a.pb[q] = pairs[q].b;
        a.ro[q] = pairs[q].ro;
        a.co[q] = pairs[q].co;
        a.flags[q] = pairs[q].flags;
        a.mro[q] = pairs[q].mro;
        a.mco[q] = pairs[q].mco;
        a.units += (pairs[q].flags & GRAM_SYM) ? a.T * (a.T + 1) / 2 : a.T * a.T;
    }
    a.M = M;
    a.ldm = ldm;
    a.err = err;
    a.piece = gf_piece_bytes();
    const int max_cons = gf_max_consumers();
    a.wpg = (a.units + 15) / 16;
    if (a.wpg > max_cons) return cudaErrorInvalidValue;   // too many units: not taken
    a.groups = max_cons / a.wpg;
    // tiles of about 24 KB whatever the number of blocks (bytes in flight),
    // stages filling up to 192 KB of shared memory (one CTA per SM)
    {
        // ~48 KB per tile and at least 8 KB per block: a tile costs a fixed
        // handshake (measured: 4 KB tiles stream at 1.5 TB/s, 32 KB tiles at
        // 6.5 TB/s), and 4 KB pieces from six arrays stream slower than 8 KB
        // ones (3.9 vs 6.0 TB/s)
        const int row_bytes = k * 4;
        int base = std::max(8192 / row_bytes, 49152 / (nblk * row_bytes));
        const int rs = 2 * a.groups;
        a.rows_t = (base + rs - 1) / rs * rs;   // every lane the same number of rows of a full tile
    }
    const size_t stage_bytes = sizeof(float) * static_cast<size_t>(nblk) * a.rows_t * k;
    a.stages = static_cast<int>(std::min<size_t>(GF_MAXSTAGES, (192u * 1024u) / stage_bytes));
    if (a.stages < 2) return cudaErrorInvalidValue;
    size_t smem = a.stages * stage_bytes;
    const size_t red_bytes = sizeof(double) * static_cast<size_t>(a.units) * 32 * a.groups;
    if (red_bytes > smem) smem = red_bytes;
    const int threads = 32 * (1 + a.wpg * a.groups);
    if (threads > GF_THREADS) return cudaErrorInvalidValue;
    cudaError_t e;
    if (zero) {
        e = cudaMemsetAsync(M, 0, sizeof(double) * static_cast<size_t>(ldm) * ldm_rows, s);
        if (e != cudaSuccess) return e;
    }
    static bool attr = false;
    if (!attr) {
        e = cudaFuncSetAttribute(k_gram_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t ntile = (n + a.rows_t - 1) / a.rows_t;
    int blocks = static_cast<int>(std::min<int64_t>(ntile, num_sms));
    if (blocks < 1) blocks = 1;
    k_gram_ff<<<blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lobpcg
