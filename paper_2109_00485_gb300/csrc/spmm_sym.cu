// Symmetric SpMM  Y = H X  from the stored lower triangle, one pass.
//
// Every stored h_ij (j <= i) contributes h_ij x_j to y_i (the triangle,
// Algorithm 2) and, for j < i, h_ij x_i to y_j (its transpose, Section 3.3).
// The paper runs the two as separate loops (Section 3.2) for overlap with
// MPI; on one GPU both are applied while the entry sits in shared memory.
//
// Work unit: one "chunk" = the entries of one row block (16 rows) that fall
// in one 16-column tile.  One bulk (TMA) copy streams the chunk (indices and
// values) HBM -> shared memory, a second brings the 16 rows of X the tile's
// columns select.  The warp scatters the entries into the dense 16x16 tile
// H_t and its transpose (zero-filled when the chunk is partial), then
//     Y_R += H_t X_C    (this row block's rows; accumulated over its chunks)
//     Y_C  = H_t^T X_R  (the tile's column rows, added to Y by 16-byte
//                        vector reductions in L2)
// Both are 16x16x16 products on the tensor cores (mma.sync m16n8k8, TF32).
// FP32 accuracy comes from the 3-term split a = a_hi + a_lo: a_hi is a with
// its 13 low mantissa bits cleared (a TF32 value), a_lo = a - a_hi (exact in
// FP32, |a_lo| < 2^-10 |a|), and a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi with
// FP32 accumulation.  The tensor core reads a_lo as TF32 (its top 19 bits),
// so each product carries a relative error below 3 * 2^-20.  X_R (this row
// block's 16 rows of X) stays in registers as split B fragments.  The
// diagonal chunk is expanded to S = L + L^T - D and applied as
// Y_R += S X_R.  Y_R of a row block is added to Y by vector reductions too,
// since other warps add transposed parts to the same rows.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"
#include "internal.h"

namespace lobpcg {

// Pipeline depth and residency (tunable at build time; the row-block
// partition made at create assumes SPMM_WARPS_PER_SM resident warps).
#ifndef SPMM_STAGES
#define SPMM_STAGES 4
#endif
#ifndef SPMM_WARPS
#define SPMM_WARPS 8
#endif
#ifndef SPMM_MINB
#define SPMM_MINB 2
#endif

constexpr int HS = 20;   // row stride of the scattered tile (fragment loads of T: bank-conflict free)

// NT = number of 8-column n-tiles of the vector block (k <= 8 NT).
template <int NT>
struct SpmmCfg {
    static constexpr int K = 8 * NT;
    // k <= 16: four stages; k = 17..24: three, so that two blocks still fit
    static constexpr int STAGES = NT <= 2 ? SPMM_STAGES : (NT == 3 ? 3 : SPMM_STAGES);
    static constexpr int WARPS = SPMM_WARPS;
    // two blocks fit in shared memory up to k = 24 (three stages past 16)
    static constexpr int MINB = NT <= 3 ? SPMM_MINB : 1;
};

// Shared memory of one warp.  A partial chunk is scattered into the stage
// it arrived in (its entries are first read into registers), so the
// scattered tile needs no buffer of its own.
template <int NT>
struct __align__(16) WarpSmem {
    uint32_t cd[SpmmCfg<NT>::STAGES][512];        // one chunk: npad index words, then npad value words
    float xt[SpmmCfg<NT>::STAGES][TILE * 8 * NT];  // X rows of the chunk's column tile (row stride k)
    int4 meta[SpmmCfg<NT>::STAGES];                 // column tile, info, padded count, valid rows
    uint64_t bar[SpmmCfg<NT>::STAGES];              // stage filled (bulk-copy bytes landed)
};
static_assert(TILE * HS <= 512, "a scattered tile fits in one chunk stage");

// Row blocks are handed out in order, SPMM_GROUP at a time, from a counter
// in device memory (zeroed before each launch): all warps then work on a
// narrow band of rows at any moment, so the X rows the band's tiles read and
// the Y rows their transposed parts update stay in L2.
#ifndef SPMM_GROUP
#define SPMM_GROUP 1
#endif

struct SpmmArgs {
    int64_t n;
    int64_t R;          // row blocks
    int k;
    const uint32_t *data;
    const ChunkRec *chunk;
    const int64_t *rb_chunk;
    int *sched;         // next row-block group to hand out
    const float *X;
    float *Y;
    int *err;
};

// Split x = hi + lo for the 3-term product (two ALU operations): hi = x
// with its 13 low mantissa bits cleared, lo = x - hi, exact in FP32.  lo is
// handed to the tensor core as it is; the TF32 operand read ignores its low
// 13 bits (a relative error below 2^-10 |lo| < 2^-20 |x|).
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// d += a b  (m16n8k8, TF32 inputs, FP32 accumulate)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += A B with A, B given as (hi, lo) splits: three products, small first.
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint32_t bh0,
                                     uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, al, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
    mma_tf32(d, ah, bh0, bh1);
}

// A fragment (16x8 slice ks) of a 16x16 tile T stored with row stride RS:
// a0 = T[g][8ks+t], a1 = T[g+8][8ks+t], a2 = T[g][8ks+t+4], a3 = T[g+8][8ks+t+4].
template <int RS>
__device__ __forceinline__ void load_a(const float *T, int ks, int g, int t, uint32_t (&ah)[4], uint32_t (&al)[4]) {
    const float *p = T + g * RS + 8 * ks + t;
    split_tf32(p[0], ah[0], al[0]);
    split_tf32(p[8 * RS], ah[1], al[1]);
    split_tf32(p[4], ah[2], al[2]);
    split_tf32(p[8 * RS + 4], ah[3], al[3]);
}
// The same fragment of the TRANSPOSE of T (T stored with row stride RS):
// a0 = T[8ks+t][g], a1 = T[8ks+t][g+8], a2 = T[8ks+t+4][g], a3 = T[8ks+t+4][g+8].
template <int RS>
__device__ __forceinline__ void load_at(const float *T, int ks, int g, int t, uint32_t (&ah)[4], uint32_t (&al)[4]) {
    const float *p = T + (8 * ks + t) * RS + g;
    split_tf32(p[0], ah[0], al[0]);
    split_tf32(p[8], ah[1], al[1]);
    split_tf32(p[4 * RS], ah[2], al[2]);
    split_tf32(p[4 * RS + 8], ah[3], al[3]);
}

// A full chunk stores column c of each row at position pc(c) = 4 (c mod 4) +
// c / 4, so lane (g, t)'s four A-fragment columns t, t + 4, t + 8, t + 12 of
// row g are one 16-byte word (both k-slices): two conflict-free vector loads.
__device__ __forceinline__ void load_a_full(const float *v, int g, int t, uint32_t (&ah)[2][4], uint32_t (&al)[2][4]) {
    const float4 r0 = *reinterpret_cast<const float4 *>(v + g * 16 + 4 * t);
    const float4 r1 = *reinterpret_cast<const float4 *>(v + (g + 8) * 16 + 4 * t);
    split_tf32(r0.x, ah[0][0], al[0][0]);
    split_tf32(r1.x, ah[0][1], al[0][1]);
    split_tf32(r0.y, ah[0][2], al[0][2]);
    split_tf32(r1.y, ah[0][3], al[0][3]);
    split_tf32(r0.z, ah[1][0], al[1][0]);
    split_tf32(r1.z, ah[1][1], al[1][1]);
    split_tf32(r0.w, ah[1][2], al[1][2]);
    split_tf32(r1.w, ah[1][3], al[1][3]);
}
// The transposed fragment (slice ks) from a full chunk: T[8ks+t][g] sits at
// row 8ks+t, position pc(g); column g + 8 two positions further on.
__device__ __forceinline__ void load_at_full(const float *v, int ks, int g, int t, uint32_t (&ah)[4],
                                             uint32_t (&al)[4]) {
    const float *p = v + (8 * ks + t) * 16 + 4 * (g & 3) + (g >> 2);
    split_tf32(p[0], ah[0], al[0]);
    split_tf32(p[2], ah[1], al[1]);
    split_tf32(p[64], ah[2], al[2]);
    split_tf32(p[66], ah[3], al[3]);
}

// Offset of S[r][c] (S = L + L^T - D) in a complete diagonal chunk, whose
// 136 entries are the lower triangle in row-major order.
__device__ __forceinline__ int tri_off(int r, int c) {
    const int a = max(r, c), b = min(r, c);
    return ((a * (a + 1)) >> 1) + b;
}
// A fragment (slice ks) of S read straight from a complete diagonal chunk.
__device__ __forceinline__ void load_a_tri(const float *v, int ks, int g, int t, uint32_t (&ah)[4],
                                           uint32_t (&al)[4]) {
    const int c = 8 * ks + t;
    split_tf32(v[tri_off(g, c)], ah[0], al[0]);
    split_tf32(v[tri_off(g + 8, c)], ah[1], al[1]);
    split_tf32(v[tri_off(g, c + 4)], ah[2], al[2]);
    split_tf32(v[tri_off(g + 8, c + 4)], ah[3], al[3]);
}

// Issue the bulk copies of one chunk into stage s (one lane).
template <int NT>
__device__ __forceinline__ void issue_chunk(const SpmmArgs &a, int k, WarpSmem<NT> *ws, int4 rec, int s, uint64_t pol_stream,
                                            uint64_t pol_keep) {
    const int64_t off = static_cast<int64_t>((static_cast<uint64_t>(static_cast<uint32_t>(rec.y)) << 32) |
                                             static_cast<uint32_t>(rec.x));
    const int ct = rec.z, info = rec.w;
    const int npad = (info >> NPAD_SHIFT) & 0x3FF;
    const bool vo = (info & VONLY_FLAG) != 0;    // value words only
    const int64_t r0 = static_cast<int64_t>(ct) * TILE;
    const int rows = static_cast<int>(a.n - r0 < TILE ? a.n - r0 : TILE);
    const uint32_t xbytes = static_cast<uint32_t>(rows) * k * 4u;
    const uint32_t cbytes = static_cast<uint32_t>(npad) * (vo ? 4u : 8u);
    ws->meta[s] = make_int4(ct, info, vo ? 0 : npad, rows);   // .z: first value word in the stage
    mbar_arrive_expect_tx(&ws->bar[s], cbytes + xbytes);
    if (npad > 0) bulk_g2s(ws->cd[s], a.data + off, cbytes, &ws->bar[s], pol_stream);
    bulk_g2s(ws->xt[s], a.X + r0 * k, xbytes, &ws->bar[s], pol_keep);
}

__device__ __forceinline__ int4 load_rec(const ChunkRec *p, int64_t c) {
    return __ldg(reinterpret_cast<const int4 *>(p + c));
}

// KC: k as a compile-time constant (0: read from the arguments).
template <int NT, int KC>
__global__ void __launch_bounds__(SpmmCfg<NT>::WARPS * 32, SpmmCfg<NT>::MINB) k_spmm_sym_tiled(SpmmArgs a) {
    using C = SpmmCfg<NT>;
    constexpr int S = C::STAGES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<NT> *ws = reinterpret_cast<WarpSmem<NT> *>(smem_raw) + warp;
    const int g = lane >> 2, t = lane & 3;   // mma fragment coordinates
    const int k = KC > 0 ? KC : a.k;

    if (lane == 0) {
        for (int st = 0; st < S; ++st) mbar_init(&ws->bar[st], 1);
        fence_proxy_async();
    }
    __syncwarp();
    const uint64_t pol_stream = policy_evict_first();
    const uint64_t pol_keep = policy_evict_last();

    // Lane 0 is the producer.  Its cursor [ic, ic_end) walks the chunks of
    // the row-block group in hand; `pending` holds the record of chunk ic.
    // The next group is requested (atomic) when a group is taken up, and
    // its chunk bounds are read one chunk later, so neither latency lands
    // on the switch from one group to the next.
    int64_t ic = 0, ic_end = 0, res_rb = 0, res_lo = 0, res_hi = 0;
    int res_state = 0;   // 0: no further group, 1: requested, 2: bounds read
    bool pend_ok = false;
    int4 pending = make_int4(0, 0, 0, 0);
    auto request = [&]() {
        res_rb = static_cast<int64_t>(atomicAdd(a.sched, 1)) * SPMM_GROUP;
        res_state = 1;
    };
    auto resolve = [&]() {
        if (res_state != 1) return;
        if (res_rb >= a.R) { res_state = 0; return; }
        res_lo = a.rb_chunk[res_rb];
        res_hi = a.rb_chunk[res_rb + SPMM_GROUP < a.R ? res_rb + SPMM_GROUP : a.R];
        res_state = 2;
    };
    auto take_group = [&]() -> bool {
        resolve();
        if (res_state != 2) return false;
        ic = res_lo;
        ic_end = res_hi;
        request();
        return true;
    };
    auto advance = [&]() {   // move the cursor to the next chunk
        resolve();
        if (++ic >= ic_end && !take_group()) {
            pend_ok = false;
            return;
        }
        pending = load_rec(a.chunk, ic);
    };
    int inflight = 0;   // lane 0: chunks issued and not yet consumed
    if (lane == 0) {
        request();
        pend_ok = take_group();
        if (pend_ok) pending = load_rec(a.chunk, ic);
        for (int st = 0; st < S && pend_ok; ++st) {
            issue_chunk<NT>(a, k, ws, pending, st, pol_stream, pol_keep);
            ++inflight;
            advance();
        }
    }

    float yr[NT][4];      // Y_R accumulators (D fragments)
    uint32_t xbh[2][NT][2], xbl[2][NT][2];   // X_R as split B fragments [k-step][n-tile][b0,b1]
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) yr[nt][q] = 0.f;
    int64_t cur_rb = -1;
    int cur_rows = 0;
    uint32_t phases = 0;
    int s = 0;

    // Add a 16 x k tile from registers (D-fragment layout) to Y rows r0..
    // r0 + rows - 1 with 16-byte vector reductions in L2 (red.global.add.v4):
    // lanes t and t^1 trade halves so that each holds four consecutive
    // columns of one row.  For a pair of n-tiles (2p, 2p+1) an even lane
    // takes row g of tile 2p and an odd lane row g of tile 2p+1 (then rows
    // g + 8); a last unpaired n-tile goes to even lanes for row g and odd
    // lanes for row g + 8.  (A bulk reduce per tile is one more operation
    // for the SM's TMA unit, whose operations bound this kernel.)
    auto reduce_tile = [&](const float (&d)[NT][4], int64_t r0, int rows) {
        const bool odd = t & 1;
#pragma unroll
        for (int pq = 0; pq + 1 < NT; pq += 2) {
            const int c0 = odd ? 8 * (pq + 1) + 2 * (t - 1) : 8 * pq + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float s0 = odd ? d[pq][2 * h] : d[pq + 1][2 * h];
                const float s1 = odd ? d[pq][2 * h + 1] : d[pq + 1][2 * h + 1];
                const float v0 = __shfl_xor_sync(0xffffffffu, s0, 1);
                const float v1 = __shfl_xor_sync(0xffffffffu, s1, 1);
                const int row = g + 8 * h;
                const float4 v = odd ? make_float4(v0, v1, d[pq + 1][2 * h], d[pq + 1][2 * h + 1])
                                     : make_float4(d[pq][2 * h], d[pq][2 * h + 1], v0, v1);
                if (row < rows && c0 + 4 <= k) red_add_v4(a.Y + (r0 + row) * k + c0, v.x, v.y, v.z, v.w);
            }
        }
        if (NT & 1) {
            constexpr int nt = NT - 1;
            const float s0 = odd ? d[nt][0] : d[nt][2];
            const float s1 = odd ? d[nt][1] : d[nt][3];
            const float v0 = __shfl_xor_sync(0xffffffffu, s0, 1);
            const float v1 = __shfl_xor_sync(0xffffffffu, s1, 1);
            const int row = odd ? g + 8 : g;
            const int c0 = 8 * nt + 2 * (odd ? t - 1 : t);
            const float4 v = odd ? make_float4(v0, v1, d[nt][2], d[nt][3]) : make_float4(d[nt][0], d[nt][1], v0, v1);
            if (row < rows && c0 + 4 <= k) red_add_v4(a.Y + (r0 + row) * k + c0, v.x, v.y, v.z, v.w);
        }
    };

    while (true) {
        const int nfl = __shfl_sync(0xffffffffu, inflight, 0);
        if (nfl == 0) break;
        const bool ok = mbar_wait_bounded(&ws->bar[s], (phases >> s) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(a.err, DEV_TIMEOUT);
            // let copies already in flight land before the warp leaves
            int ss = s;
            for (int q = 0; q < nfl; ++q) {
                mbar_wait_bounded(&ws->bar[ss], (phases >> ss) & 1u);
                ss = (ss + 1 == S) ? 0 : ss + 1;
            }
            return;
        }
        phases ^= 1u << s;
        const int4 m = ws->meta[s];
        const int ct = m.x, cnt = m.y & 0xFFFF, rows = m.w;
        const bool is_diag = (m.y & DIAG_FLAG) != 0;
        const float *xt = ws->xt[s];
        const uint32_t *sidx = ws->cd[s];
        const float *sval = reinterpret_cast<const float *>(ws->cd[s] + m.z);

        // A chunk holding all 256 entries of its off-diagonal tile is that tile
        // (rows in order, columns permuted as load_a_full reads them), and a diagonal chunk
        // holding all 136 entries of its lower triangle is that triangle in
        // row-major order, so their fragments are read straight from the
        // staged values.  Any other chunk (fewer than 256 entries) is read
        // into registers, then scattered by its indices into a zeroed tile
        // (a diagonal one into the symmetric S = L + L^T - D) that takes the
        // place of the chunk in its stage.
        const bool full = !is_diag && cnt == 256;
        const bool tri = is_diag && cnt == TILE * (TILE + 1) / 2;   // complete diagonal tile, canonical order
        float *Hs = reinterpret_cast<float *>(ws->cd[s]);
        if (!full && !tri) {
            uint32_t eu[8];
            float ev[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = lane + 32 * q;
                eu[q] = (e < cnt) ? sidx[e] : IDX_PAD;
                ev[q] = (e < cnt) ? sval[e] : 0.f;
            }
            __syncwarp();
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int e = lane; e < TILE * HS / 4; e += 32) reinterpret_cast<float4 *>(Hs)[e] = z;
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (eu[q] == IDX_PAD) continue;
                const int rl = (eu[q] >> 28) & 15, cl = eu[q] & 15;
                Hs[rl * HS + cl] = ev[q];
                if (is_diag) Hs[cl * HS + rl] = ev[q];
            }
            fence_proxy_async();   // the stage is refilled by a bulk copy later
            __syncwarp();
        }

        if (is_diag) {
            if (cur_rb >= 0) reduce_tile(yr, cur_rb * TILE, cur_rows);
            cur_rb = ct;
            cur_rows = rows;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) yr[nt][q] = 0.f;
            // X_R B fragments: b0 = X_R[8ks+t][8nt+g], b1 = X_R[8ks+t+4][8nt+g]
#pragma unroll
            for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int col = 8 * nt + g, r0 = 8 * ks + t;
                    const float v0 = (col < k && r0 < rows) ? xt[r0 * k + col] : 0.f;
                    const float v1 = (col < k && r0 + 4 < rows) ? xt[(r0 + 4) * k + col] : 0.f;
                    split_tf32(v0, xbh[ks][nt][0], xbl[ks][nt][0]);
                    split_tf32(v1, xbh[ks][nt][1], xbl[ks][nt][1]);
                }
            // Y_R += S X_R
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t ah[4], al[4];
                if (tri) load_a_tri(sval, ks, g, t, ah, al);
                else load_a<HS>(Hs, ks, g, t, ah, al);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
                    mma3(yr[nt], ah, al, xbh[ks][nt][0], xbh[ks][nt][1], xbl[ks][nt][0], xbl[ks][nt][1]);
            }
        } else {
            // Each tile product starts from a zero accumulator and is added to
            // Y_R with ordinary FP32 adds: the tensor-core accumulation then
            // only ever sums the 48 terms of one tile product.
            float yc[NT][4], yt4[NT][4];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) yc[nt][q] = yt4[nt][q] = 0.f;
            uint32_t fah[2][4], fal[2][4];   // H_t fragments of both k-slices
            if (full) load_a_full(sval, g, t, fah, fal);
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t ah[4], al[4], th[4], tl[4];
                if (full) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) { ah[q] = fah[ks][q]; al[q] = fal[ks][q]; }   // H_t
                    load_at_full(sval, ks, g, t, th, tl);                                    // H_t^T
                } else {
                    load_a<HS>(Hs, ks, g, t, ah, al);
                    load_at<HS>(Hs, ks, g, t, th, tl);
                }
                uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int col = 8 * nt + g, r0 = 8 * ks + t;
                    split_tf32(col < k ? xt[r0 * k + col] : 0.f, bh[nt][0], bl[nt][0]);
                    split_tf32(col < k ? xt[(r0 + 4) * k + col] : 0.f, bh[nt][1], bl[nt][1]);
                }
                // small terms first, independent accumulators interleaved
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    mma_tf32(yt4[nt], al, bh[nt][0], bh[nt][1]);                          // Y_R += H_t X_C
                    mma_tf32(yc[nt], tl, xbh[ks][nt][0], xbh[ks][nt][1]);                 // Y_C = H_t^T X_R
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    mma_tf32(yt4[nt], ah, bl[nt][0], bl[nt][1]);
                    mma_tf32(yc[nt], th, xbl[ks][nt][0], xbl[ks][nt][1]);
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    mma_tf32(yt4[nt], ah, bh[nt][0], bh[nt][1]);
                    mma_tf32(yc[nt], th, xbh[ks][nt][0], xbh[ks][nt][1]);
                }
            }
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) yr[nt][q] += yt4[nt][q];
            reduce_tile(yc, static_cast<int64_t>(ct) * TILE, TILE);   // off-diagonal tiles lie inside 0..n-1
        }
        __syncwarp();
        if (lane == 0) {
            --inflight;
            if (pend_ok) {
                fence_proxy_async();
                issue_chunk<NT>(a, k, ws, pending, s, pol_stream, pol_keep);
                ++inflight;
                advance();
            }
        }
        s = (s + 1 == S) ? 0 : s + 1;
    }
    if (cur_rb >= 0) reduce_tile(yr, cur_rb * TILE, cur_rows);
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
__global__ void __launch_bounds__(256) k_spmm_sym_simple(int64_t n, int k, const uint32_t *data,
                                                         const ChunkRec *chunk, const int64_t *rb_chunk,
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
            const ChunkRec rec = chunk[c];
            const int64_t off = rec.off;
            const int info = rec.info;
            const int64_t npad = (info >> NPAD_SHIFT) & 0x3FF;
            const bool vo = (info & VONLY_FLAG) != 0;
            const uint32_t *cidx = data + off;
            const uint32_t *cval = vo ? cidx : cidx + npad;
            const int cnt = info & 0xFFFF;
            const bool is_diag = (info & DIAG_FLAG) != 0;
            const int64_t ct = rec.ct;
            for (int e = lane; e < 256; e += 32) ws->H[e] = 0.f;
            for (int e = lane; e < TILE * 17; e += 32) ws->HT[e] = 0.f;
            __syncwarp();
            for (int e = lane; e < cnt; e += 32) {
                const float v = __uint_as_float(cval[e]);
                int rl, cl;
                if (!vo) {
                    const uint32_t u = cidx[e];
                    rl = (u >> 28) & 15;
                    cl = u & 15;
                } else if (!is_diag) {
                    // complete tile: row e / 16; position p within the row holds column 4 (p % 4) + p / 4
                    const int p = e & 15;
                    rl = e >> 4;
                    cl = 4 * (p & 3) + (p >> 2);
                } else {
                    // complete lower triangle, row-major: row r holds entries r (r + 1) / 2 ..
                    int r = static_cast<int>((sqrtf(8.f * static_cast<float>(e) + 1.f) - 1.f) * 0.5f);
                    while (r * (r + 1) / 2 > e) --r;
                    while ((r + 1) * (r + 2) / 2 <= e) ++r;
                    rl = r;
                    cl = e - r * (r + 1) / 2;
                }
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

template <int NT, int KC>
static cudaError_t launch_tiled(const lobpcg_ctx *h, const float *X, float *Y, int k, cudaStream_t s) {
    using C = SpmmCfg<NT>;
    const size_t smem = sizeof(WarpSmem<NT>) * C::WARPS;
    static bool attr_set[64] = {false};
    int dev = h->device;
    if (!attr_set[dev & 63]) {
        cudaError_t e = cudaFuncSetAttribute(k_spmm_sym_tiled<NT, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr_set[dev & 63] = true;
    }
    SpmmArgs a;
    a.n = h->T.n; a.R = h->T.R; a.k = k; a.data = h->T.data; a.chunk = h->T.chunk; a.rb_chunk = h->T.rb_chunk;
    a.sched = h->T.sched; a.X = X; a.Y = Y; a.err = h->d_err;
    cudaError_t e = cudaMemsetAsync(h->T.sched, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    const int blocks = (h->T.warps + C::WARPS - 1) / C::WARPS;
    k_spmm_sym_tiled<NT, KC><<<blocks, C::WARPS * 32, smem, s>>>(a);
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
    k_spmm_sym_simple<T><<<blocks, 256, smem, s>>>(h->T.n, k, h->T.data, h->T.chunk, h->T.rb_chunk, R, X, Y);
    return cudaGetLastError();
}

cudaError_t launch_spmm_sym_f32(const lobpcg_ctx *h, const float *X, float *Y, int k, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(Y, 0, sizeof(float) * static_cast<size_t>(h->T.n) * k, s);
    if (e != cudaSuccess) return e;
    const bool aligned = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15u) == 0;
    if (aligned && k % 4 == 0) {
        switch (k) {   // the common block sizes with k known at compile time
            case 8: return launch_tiled<1, 8>(h, X, Y, k, s);
            case 16: return launch_tiled<2, 16>(h, X, Y, k, s);
            case 20: return launch_tiled<3, 20>(h, X, Y, k, s);
            case 32: return launch_tiled<4, 32>(h, X, Y, k, s);
            default: break;
        }
        if (k <= 8) return launch_tiled<1, 0>(h, X, Y, k, s);
        if (k <= 16) return launch_tiled<2, 0>(h, X, Y, k, s);
        if (k <= 24) return launch_tiled<3, 0>(h, X, Y, k, s);
        return launch_tiled<4, 0>(h, X, Y, k, s);
    }
    return launch_simple<float>(h, X, Y, k, s);
}

cudaError_t launch_spmm_sym_f64(lobpcg_ctx *h, const double *X, double *Y, int k, cudaStream_t s) {
    if (spmm_df_ok(k, X, Y)) return launch_spmm_sym_df(h, X, Y, k, s);   // writes every row of Y
    cudaError_t e = cudaMemsetAsync(Y, 0, sizeof(double) * static_cast<size_t>(h->T.n) * k, s);
    if (e != cudaSuccess) return e;
    return launch_simple<double>(h, X, Y, k, s);
}

}  // namespace lobpcg
