// The paper's preconditioner (Section 3.3): K is block diagonal, K_T the
// diagonal tile H_T of a row partition, shifted by the Ritz value theta_j of
// the column it is applied to, and K_T^{-1} r is approximated by s steps
// (three to five in the paper) of the Full Orthogonalization Method from
// x_0 = 0 -- one Krylov space per tile and column, all columns of a tile
// advanced together (the paper's FOM_thread).
//
// Per tile and column: beta = ||r||, v_0 = r / beta; step j forms
// w = (H_T - theta I) v_j, orthogonalises it against v_0..v_j (classical
// Gram-Schmidt applied twice: the same Galerkin space as the modified form
// in exact arithmetic, and as accurate), h_{j+1,j} = ||w||, and stops the
// column (s = j + 1) when h_{j+1,j} <= 1e-6 ||(H_T - theta I) v_j|| (an
// invariant Krylov space).  The s x s Hessenberg system H_s y = beta e_1 is
// solved by Gaussian elimination with partial pivoting, each pivot guarded
// as g(t) = sign(t) max(|t|, 1e-3 max(1, |theta|)), and x = V_s y.
//
// Tiles of at most 64 rows run in k_fom_small (one CTA per tile, the tile
// dense in shared memory, every column's basis in registers); larger tiles
// (the paper's run to thousands of rows) in the k_fl_* kernels: all large
// tiles advance together, one grid-wide kernel per phase of a step over
// 64-row segments, each tile as a local CSR of both triangles and the basis
// vectors in a global scratch.
#include <algorithm>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "internal.h"
#include "precond.h"

namespace lobpcg {
namespace {

constexpr int BS = FOM_SMALL;            // rows of a small tile's dense block
constexpr int PITCH = 68;                // shared row pitch (floats): 16-byte rows, 4-bank step per row
constexpr int MS = FOM_MAX_STEPS;
constexpr int NV = MS + 1;               // reduction slots: MS dot products + one squared norm (slot MS)
constexpr float BREAKDOWN = 1e-6f;

// Sum the NV per-thread partials over the row groups of one column (L lanes
// per row group, NW warps).  Butterfly shuffles inside a warp, then one pass
// through shared memory over the warps.  Every thread of a column ends with
// bitwise identical sums (pairwise adds are commutative; then the same
// reads in the same order), so the per-column decisions below agree.
template <int L, int NW>
__device__ __forceinline__ void colsum(float (&v)[NV], float *red, int warp, int lane) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = L; o < 32; o <<= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    if (lane < L) {
#pragma unroll
        for (int i = 0; i < NV; ++i) red[(warp * NV + i) * 32 + lane] = v[i];
    }
    __syncthreads();
    const int j = lane % L;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float x = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) x += red[(w * NV + i) * 32 + j];
        v[i] = x;
    }
}

__device__ __forceinline__ float guarded(float p, float delta) {
    return (p >= 0.f ? 1.f : -1.f) * fmaxf(fabsf(p), delta);
}

// y with H_s y = beta e_1 (H upper Hessenberg, s = sdim): Gaussian
// elimination with partial pivoting -- column i has nonzeros in rows i and
// i + 1 only, so the pivot search is one comparison and an exchange of those
// two rows -- guarded pivots, back substitution.  (Without the exchanges a
// small leading pivot of an indefinite tile multiplies the float32 rounding
// by its growth factor.)
__device__ __forceinline__ void hess_solve(float (&H)[NV][MS], int sdim, float beta, float delta, float (&y)[MS]) {
    float b[MS];
#pragma unroll
    for (int i = 0; i < MS; ++i) b[i] = (i == 0) ? beta : 0.f;
#pragma unroll
    for (int i = 0; i < MS; ++i) {
        if (i < sdim) {
            if (i + 1 < sdim && fabsf(H[i + 1][i]) > fabsf(H[i][i])) {
#pragma unroll
                for (int c = i; c < MS; ++c) {
                    const float t = H[i][c];
                    H[i][c] = H[i + 1][c];
                    H[i + 1][c] = t;
                }
                const float t = b[i];
                b[i] = b[i + 1];
                b[i + 1] = t;
            }
            const float gp = guarded(H[i][i], delta);
            H[i][i] = gp;
            if (i + 1 < sdim) {
                const float l = H[i + 1][i] / gp;
#pragma unroll
                for (int c = i + 1; c < MS; ++c) H[i + 1][c] = fmaf(-l, H[i][c], H[i + 1][c]);
                b[i + 1] = fmaf(-l, b[i], b[i + 1]);
            }
        }
    }
#pragma unroll
    for (int i = MS - 1; i >= 0; --i) {
        y[i] = 0.f;
        if (i < sdim) {
            float t = b[i];
#pragma unroll
            for (int c = i + 1; c < MS; ++c)
                if (c < sdim) t = fmaf(-H[i][c], y[c], t);
            y[i] = t / H[i][i];
        }
    }
}

// Record column st of H from the two Gram-Schmidt passes (h: first-pass
// coefficients, acc[0..st]: second-pass ones, acc[MS]: ||w after pass 1||^2)
// and decide breakdown.  Returns h_{st+1,st}.
__device__ __forceinline__ float hess_column(float (&H)[NV][MS], const float (&h)[MS], const float (&acc)[NV], int st,
                                             float wn, bool &active, int &sdim) {
    float c2 = 0.f;
#pragma unroll
    for (int i = 0; i < MS; ++i)
        if (i <= st) c2 = fmaf(acc[i], acc[i], c2);
    const float hs = sqrtf(fmaxf(acc[MS] - c2, 0.f));   // ||w1 - V c||^2 = ||w1||^2 - ||c||^2 (V orthonormal)
    if (active) {
#pragma unroll
        for (int c = 0; c < MS; ++c) {
            if (c == st) {
#pragma unroll
                for (int i = 0; i <= c; ++i) H[i][c] = h[i] + acc[i];
                H[c + 1][c] = hs;
            }
        }
        if (hs <= BREAKDOWN * wn) {
            sdim = st + 1;
            active = false;
        }
    }
    return hs;
}

// ---------------------------------------------------------------- small tiles
// One CTA (256 threads) per tile of m <= 64 rows.  Thread t serves column
// j = t % L (L >= k, a power of two) and rows [g RPT, g RPT + RPT) with
// g = t / L, so a column's basis lives in the registers of its 256/L threads.
template <int L, typename T>
__global__ void __launch_bounds__(256) k_fom_small(int k, int steps, const int64_t *s_t0, const int32_t *s_m,
                                                   const float *Atiles, const T *R, const double *theta, T *W) {
    constexpr int G = 256 / L;
    constexpr int RPT = BS / G;
    extern __shared__ __align__(16) float smf[];
    float *sA = smf;                           // [64][PITCH]
    float *sV = sA + BS * PITCH;               // [L][PITCH]: v_st of every column, rows contiguous
    float *red = sV + L * PITCH;               // [2][8 warps][NV][32]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = tid % L, r0 = (tid / L) * RPT;
    const int64_t t0 = s_t0[blockIdx.x];
    const int m = s_m[blockIdx.x];
    {
        const float4 *src = reinterpret_cast<const float4 *>(Atiles + static_cast<int64_t>(blockIdx.x) * BS * BS);
        for (int e = tid; e < BS * BS / 4; e += 256) {
            const int row = e / (BS / 4), c4 = e % (BS / 4);
            *reinterpret_cast<float4 *>(sA + row * PITCH + 4 * c4) = src[e];
        }
    }
    const bool colok = j < k;
    const float th = colok ? static_cast<float>(theta[j]) : 0.f;
    const float delta = 1e-3f * fmaxf(1.f, fabsf(th));
    float vb[MS][RPT];
    float w[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int r = r0 + q;
        w[q] = (colok && r < m) ? static_cast<float>(R[(t0 + r) * k + j]) : 0.f;
#pragma unroll
        for (int i = 0; i < MS; ++i) vb[i][q] = 0.f;
    }
    float acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.f;
#pragma unroll
    for (int q = 0; q < RPT; ++q) acc[MS] = fmaf(w[q], w[q], acc[MS]);
    colsum<L, 8>(acc, red, warp, lane);
    const float beta = sqrtf(acc[MS]);
    const float rb = beta > 0.f ? 1.f / beta : 0.f;
#pragma unroll
    for (int q = 0; q < RPT; ++q) vb[0][q] = w[q] * rb;
    float H[NV][MS];
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
        for (int b = 0; b < MS; ++b) H[a][b] = 0.f;
    int sdim = steps, par = 1;
    bool active = true;
#pragma unroll
    for (int st = 0; st < MS; ++st) {
        if (st >= steps) break;
#pragma unroll
        for (int q = 0; q < RPT; ++q) sV[j * PITCH + r0 + q] = vb[st][q];
        __syncthreads();
        // w = A v - theta v over own rows (float4 reads of the tile rows and of v)
#pragma unroll
        for (int q = 0; q < RPT; ++q) w[q] = 0.f;
        const float *vcol = sV + j * PITCH;
#pragma unroll 4
        for (int l = 0; l < BS; l += 4) {
            const float4 x = *reinterpret_cast<const float4 *>(vcol + l);
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                const float4 a = *reinterpret_cast<const float4 *>(sA + (r0 + q) * PITCH + l);
                w[q] = fmaf(a.x, x.x, fmaf(a.y, x.y, fmaf(a.z, x.z, fmaf(a.w, x.w, w[q]))));
            }
        }
#pragma unroll
        for (int q = 0; q < RPT; ++q) w[q] = fmaf(-th, vb[st][q], w[q]);
        // pass 1: h_i = v_i . w and ||w||^2
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = 0.f;
#pragma unroll
        for (int i = 0; i <= st; ++i)
#pragma unroll
            for (int q = 0; q < RPT; ++q) acc[i] = fmaf(vb[i][q], w[q], acc[i]);
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[MS] = fmaf(w[q], w[q], acc[MS]);
        colsum<L, 8>(acc, red + par * 8 * NV * 32, warp, lane);
        par ^= 1;
        const float wn = sqrtf(acc[MS]);
        float h[MS];
#pragma unroll
        for (int i = 0; i < MS; ++i) {
            h[i] = (i <= st) ? acc[i] : 0.f;
            if (i <= st) {
#pragma unroll
                for (int q = 0; q < RPT; ++q) w[q] = fmaf(-h[i], vb[i][q], w[q]);
            }
        }
        // pass 2: c_i = v_i . w1 and ||w1||^2
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] = 0.f;
#pragma unroll
        for (int i = 0; i <= st; ++i)
#pragma unroll
            for (int q = 0; q < RPT; ++q) acc[i] = fmaf(vb[i][q], w[q], acc[i]);
#pragma unroll
        for (int q = 0; q < RPT; ++q) acc[MS] = fmaf(w[q], w[q], acc[MS]);
        colsum<L, 8>(acc, red + par * 8 * NV * 32, warp, lane);
        par ^= 1;
        const bool was_active = active;
        const float hs = hess_column(H, h, acc, st, wn, active, sdim);
        if (st + 1 < MS) {
            const float rh = (was_active && active) ? 1.f / hs : 0.f;
#pragma unroll
            for (int q = 0; q < RPT; ++q) {
                float x = w[q];
#pragma unroll
                for (int i = 0; i <= st; ++i) x = fmaf(-acc[i], vb[i][q], x);
                vb[st + 1][q] = x * rh;
            }
        }
    }
    float y[MS];
    hess_solve(H, sdim, beta, delta, y);
    if (!colok) return;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const int r = r0 + q;
        if (r >= m) break;
        float x = 0.f;
#pragma unroll
        for (int i = 0; i < MS; ++i)
            if (i < sdim) x = fmaf(y[i], vb[i][q], x);
        W[(t0 + r) * k + j] = static_cast<T>(beta > 0.f ? x : 0.f);
    }
}

// ---------------------------------------------------------------- large tiles
// Tiles of more than 64 rows advance together, one grid-wide kernel per
// phase of a FOM step, so that a tile of thousands of rows is spread over
// the whole GPU instead of one CTA (the paper notes that the spread of tile
// sizes, 1 to thousands, unbalances its one-tile-per-gang loop).  Their
// rows are packed one tile after another (packed row p) and cut into
// segments of at most 64 rows inside one tile; one CTA of 64 G threads takes
// a segment, thread t serving row t / G of it and the four columns
// 4 (t % G) .. 4 (t % G) + 3 (G = the power of two >= ceil(k / 4)), so
// every vector access is one 16-byte load or store.  Per step: the product
// (k_fl_matvec), two Gram-Schmidt passes (k_fl_dots1, k_fl_dots2) and the
// next basis vector (k_fl_next).  Per-tile sums (norms
// and Gram-Schmidt coefficients) are CTA partial sums added atomically into
// acc, one slot set per step and pass; every later kernel reads complete
// sums and replays the same per-column decisions from them.
//   scratch: kp = k rounded up to 4 columns (the padding stays zero);
//            basis v_q at V + q nl kp, work vector w at V + MS nl kp,
//            element (p, j) at p kp + j
//   acc    : [MS steps][2 passes][large tiles][NV][32]; slot i < MS is
//            v_i . w, slot MS a squared norm; accb [large tiles][32] = ||r||^2
struct LargeArgs {
    int k, kp, steps;
    int64_t nl, nlt;
    const int64_t *seg_p0;      // first packed row of each segment
    const int32_t *seg_n;       // rows of each segment (<= 64)
    const int32_t *seg_t;       // large tile of each segment
    const int64_t *l_t0;        // first matrix row of each large tile
    const int64_t *l_base;      // first packed row of each large tile
    const int64_t *rp;          // local CSR of each tile, both triangles (packed rows)
    const int32_t *lcol;        // column within the tile
    const float *lval;
    float *V;
    float *acc;
    float *accb;
};

constexpr int SEG = 64;

__device__ __forceinline__ float *acc_at(const LargeArgs &a, int st, int pass, int tile) {
    return a.acc + ((static_cast<int64_t>(st) * 2 + pass) * a.nlt + tile) * (NV * 32);
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 fma4v(float4 a, float4 x, float4 y) {
    return make_float4(fmaf(a.x, x.x, y.x), fmaf(a.y, x.y, y.y), fmaf(a.z, x.z, y.z), fmaf(a.w, x.w, y.w));
}
__device__ __forceinline__ float comp(float4 v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }

// Replay steps 0 .. upto-1 of one tile column from the sums: H, s, and
// whether the Krylov space still grows.  Every kernel that needs them calls
// this on the same complete sums, so all segments of a tile agree.
__device__ __forceinline__ void replay(const LargeArgs &a, int tile, int j, int upto, float (&H)[NV][MS], int &sdim,
                                       bool &active) {
#pragma unroll
    for (int r = 0; r < NV; ++r)
#pragma unroll
        for (int c = 0; c < MS; ++c) H[r][c] = 0.f;
    sdim = a.steps;
    active = true;
    for (int st = 0; st < upto; ++st) {
        const float *a1 = acc_at(a, st, 0, tile);
        const float *a2 = acc_at(a, st, 1, tile);
        float h[MS], c[NV];
#pragma unroll
        for (int i = 0; i < MS; ++i) {
            h[i] = (i <= st) ? a1[i * 32 + j] : 0.f;
            c[i] = (i <= st) ? a2[i * 32 + j] : 0.f;
        }
        c[MS] = a2[MS * 32 + j];
        const float wn = sqrtf(a1[MS * 32 + j]);
        hess_column(H, h, c, st, wn, active, sdim);
    }
}

// Sum NV float4 partials over the 64 rows of a segment (lane groups of G in
// a warp, then the 2G warps through shared memory) and add slots 0..nd-1
// and MS of every real column atomically into dst[slot * 32 + j].
template <int G>
__device__ __forceinline__ void seg_sum_add(float4 (&v)[NV], int nd, float *red, float *dst, int k) {
    constexpr int NWP = 2 * G;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = tid % G;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = G; o < 32; o <<= 1) {
            v[i].x += __shfl_xor_sync(0xffffffffu, v[i].x, o);
            v[i].y += __shfl_xor_sync(0xffffffffu, v[i].y, o);
            v[i].z += __shfl_xor_sync(0xffffffffu, v[i].z, o);
            v[i].w += __shfl_xor_sync(0xffffffffu, v[i].w, o);
        }
    }
    if (lane < G) {
#pragma unroll
        for (int i = 0; i < NV; ++i) st4(red + (warp * NV + i) * 32 + 4 * g, v[i]);
    }
    __syncthreads();
    if (tid < G) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            if (i < nd || i == MS) {
                float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int w = 0; w < NWP; ++w) {
                    const float4 x = ld4(red + (w * NV + i) * 32 + 4 * g);
                    s.x += x.x;
                    s.y += x.y;
                    s.z += x.z;
                    s.w += x.w;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    if (4 * g + c < k) atomicAdd(dst + i * 32 + 4 * g + c, comp(s, c));
            }
        }
    }
}

struct SegPos {
    int tile, n, r, g;
    int64_t p0, p;
};
template <int G>
__device__ __forceinline__ SegPos seg_pos(const LargeArgs &a) {
    SegPos q;
    q.tile = a.seg_t[blockIdx.x];
    q.p0 = a.seg_p0[blockIdx.x];
    q.n = a.seg_n[blockIdx.x];
    q.r = threadIdx.x / G;
    q.g = threadIdx.x % G;
    q.p = q.p0 + q.r;
    return q;
}

// ||r||^2 per tile column
template <int G, typename T>
__global__ void __launch_bounds__(64 * G) k_fl_norm(LargeArgs a, const T *R) {
    __shared__ __align__(16) float red[2 * G * NV * 32];
    const SegPos q = seg_pos<G>(a);
    float4 v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q.r < q.n) {
        const int64_t row = a.l_t0[q.tile] + (q.p - a.l_base[q.tile]);
        float x[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) x[c] = (4 * q.g + c < a.k) ? static_cast<float>(R[row * a.k + 4 * q.g + c]) : 0.f;
        v[MS] = make_float4(x[0] * x[0], x[1] * x[1], x[2] * x[2], x[3] * x[3]);
    }
    // only slot MS is added: aim it at accb[tile][.] (the pointer stays inside acc)
    seg_sum_add<G>(v, 0, red, a.accb + static_cast<int64_t>(q.tile) * 32 - MS * 32, a.k);
}

// v_0 = r / ||r||
template <int G, typename T>
__global__ void __launch_bounds__(64 * G) k_fl_start(LargeArgs a, const T *R) {
    const SegPos q = seg_pos<G>(a);
    if (q.r >= q.n || 4 * q.g >= a.kp) return;
    const int64_t row = a.l_t0[q.tile] + (q.p - a.l_base[q.tile]);
    float x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = 4 * q.g + c;
        const float beta = (j < a.k) ? sqrtf(a.accb[static_cast<int64_t>(q.tile) * 32 + j]) : 0.f;
        x[c] = (j < a.k && beta > 0.f) ? static_cast<float>(R[row * a.k + j]) / beta : 0.f;
    }
    st4(a.V + q.p * a.kp + 4 * q.g, make_float4(x[0], x[1], x[2], x[3]));
}

// w = (H_T - theta I) v_st as a pure row gather over each tile's full
// symmetric local CSR (both triangles, built at create): the segment's
// rows of v_st are staged in shared memory, columns inside the segment are
// read from there, the others from global memory; no atomics.
template <int G>
__global__ void __launch_bounds__(64 * G) k_fl_matvec(LargeArgs a, int st, const double *theta) {
    __shared__ __align__(16) float sv[SEG * 4 * G];
    const SegPos q = seg_pos<G>(a);
    const int64_t base = a.l_base[q.tile], vs = a.nl * a.kp;
    const float *v = a.V + st * vs;
    const bool mine = q.r < q.n && 4 * q.g < a.kp;
    const int seg0 = static_cast<int>(q.p0 - base);          // first tile row of the segment
    float4 vp = make_float4(0.f, 0.f, 0.f, 0.f);
    if (mine) vp = ld4(v + q.p * a.kp + 4 * q.g);
    st4(sv + q.r * 4 * G + 4 * q.g, vp);
    __syncthreads();
    if (!mine) return;
    float th[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) th[c] = (4 * q.g + c < a.k) ? static_cast<float>(theta[4 * q.g + c]) : 0.f;
    float4 s0 = make_float4(-th[0] * vp.x, -th[1] * vp.y, -th[2] * vp.z, -th[3] * vp.w);
    float4 s1 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t e1 = a.rp[q.p + 1];
    int64_t e = a.rp[q.p];
    for (; e + 1 < e1; e += 2) {
        const int c0 = a.lcol[e] - seg0, c1 = a.lcol[e + 1] - seg0;
        const float a0 = a.lval[e], a1 = a.lval[e + 1];
        const float4 x0 = (c0 >= 0 && c0 < q.n) ? ld4(sv + c0 * 4 * G + 4 * q.g)
                                               : ld4(v + (q.p0 + c0) * a.kp + 4 * q.g);
        const float4 x1 = (c1 >= 0 && c1 < q.n) ? ld4(sv + c1 * 4 * G + 4 * q.g)
                                               : ld4(v + (q.p0 + c1) * a.kp + 4 * q.g);
        s0 = fma4(a0, x0, s0);
        s1 = fma4(a1, x1, s1);
    }
    if (e < e1) {
        const int c0 = a.lcol[e] - seg0;
        const float4 x0 = (c0 >= 0 && c0 < q.n) ? ld4(sv + c0 * 4 * G + 4 * q.g)
                                               : ld4(v + (q.p0 + c0) * a.kp + 4 * q.g);
        s0 = fma4(a.lval[e], x0, s0);
    }
    st4(a.V + MS * vs + q.p * a.kp + 4 * q.g, make_float4(s0.x + s1.x, s0.y + s1.y, s0.z + s1.z, s0.w + s1.w));
}

// pass 1 partial sums: v_i . w (i <= st) and ||w||^2
template <int G>
__global__ void __launch_bounds__(64 * G) k_fl_dots1(LargeArgs a, int st) {
    __shared__ __align__(16) float red[2 * G * NV * 32];
    const SegPos q = seg_pos<G>(a);
    const int64_t vs = a.nl * a.kp;
    float4 v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q.r < q.n && 4 * q.g < a.kp) {
        const int64_t o = q.p * a.kp + 4 * q.g;
        const float4 x = ld4(a.V + MS * vs + o);
#pragma unroll
        for (int i = 0; i < MS; ++i)
            if (i <= st) v[i] = fma4v(ld4(a.V + i * vs + o), x, v[i]);
        v[MS] = fma4v(x, x, v[MS]);
    }
    seg_sum_add<G>(v, st + 1, red, acc_at(a, st, 0, q.tile), a.k);
}

// w1 = w - V h (stored) and the pass 2 partial sums v_i . w1, ||w1||^2
template <int G>
__global__ void __launch_bounds__(64 * G) k_fl_dots2(LargeArgs a, int st) {
    __shared__ __align__(16) float red[2 * G * NV * 32];
    const SegPos q = seg_pos<G>(a);
    const int64_t vs = a.nl * a.kp;
    float4 v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (q.r < q.n && 4 * q.g < a.kp) {
        const float *a1 = acc_at(a, st, 0, q.tile) + 4 * q.g;
        const int64_t o = q.p * a.kp + 4 * q.g;
        float4 vq[MS];
        float4 x = ld4(a.V + MS * vs + o);
#pragma unroll
        for (int i = 0; i < MS; ++i) {
            if (i <= st) {
                vq[i] = ld4(a.V + i * vs + o);
                const float4 h = ld4(a1 + i * 32);
                x = fma4v(make_float4(-h.x, -h.y, -h.z, -h.w), vq[i], x);
            }
        }
        st4(a.V + MS * vs + o, x);
#pragma unroll
        for (int i = 0; i < MS; ++i)
            if (i <= st) v[i] = fma4v(vq[i], x, v[i]);
        v[MS] = fma4v(x, x, v[MS]);
    }
    seg_sum_add<G>(v, st + 1, red, acc_at(a, st, 1, q.tile), a.k);
}

// v_{st+1} = (w1 - V c) / h_{st+1,st}, zero once the column has stopped.
// One thread per column replays the tile's history; the scale goes through
// shared memory to the rest of the CTA.
template <int G>
__global__ void __launch_bounds__(64 * G) k_fl_next(LargeArgs a, int st) {
    __shared__ float s_rh[32];
    const SegPos q = seg_pos<G>(a);
    const float *a1 = acc_at(a, st, 0, q.tile);
    const float *a2 = acc_at(a, st, 1, q.tile);
    const int t = threadIdx.x;
    if (t < 32) {
        float rh = 0.f;
        if (t < a.k) {
            float H[NV][MS];
            int sdim;
            bool active;
            replay(a, q.tile, t, st, H, sdim, active);
            const bool was_active = active;
            float h[MS], cc[NV];
#pragma unroll
            for (int i = 0; i < MS; ++i) {
                h[i] = (i <= st) ? a1[i * 32 + t] : 0.f;
                cc[i] = (i <= st) ? a2[i * 32 + t] : 0.f;
            }
            cc[MS] = a2[MS * 32 + t];
            const float hs = hess_column(H, h, cc, st, sqrtf(a1[MS * 32 + t]), active, sdim);
            rh = (was_active && active) ? 1.f / hs : 0.f;
        }
        s_rh[t] = rh;
    }
    __syncthreads();
    if (q.r >= q.n || 4 * q.g >= a.kp) return;
    const int64_t vs = a.nl * a.kp;
    const int64_t o = q.p * a.kp + 4 * q.g;
    float4 x = ld4(a.V + MS * vs + o);
#pragma unroll
    for (int i = 0; i < MS; ++i) {
        if (i <= st) {
            const float4 c = ld4(a2 + i * 32 + 4 * q.g);
            x = fma4v(make_float4(-c.x, -c.y, -c.z, -c.w), ld4(a.V + i * vs + o), x);
        }
    }
    const float4 rh = ld4(s_rh + 4 * q.g);
    st4(a.V + (st + 1) * vs + o, make_float4(x.x * rh.x, x.y * rh.y, x.z * rh.z, x.w * rh.w));
}

// x = V_s y with H_s y = beta e_1: one thread per column replays the tile's
// history and solves the small system; y goes through shared memory.
template <int G, typename T>
__global__ void __launch_bounds__(64 * G) k_fl_finish(LargeArgs a, const double *theta, T *W) {
    __shared__ __align__(16) float s_y[MS][32];
    const SegPos q = seg_pos<G>(a);
    const int t = threadIdx.x;
    if (t < 32) {
        float y[MS];
#pragma unroll
        for (int i = 0; i < MS; ++i) y[i] = 0.f;
        if (t < a.k) {
            float H[NV][MS];
            int sdim;
            bool active;
            replay(a, q.tile, t, a.steps, H, sdim, active);
            const float beta = sqrtf(a.accb[static_cast<int64_t>(q.tile) * 32 + t]);
            const float th = static_cast<float>(theta[t]);
            hess_solve(H, sdim, beta, 1e-3f * fmaxf(1.f, fabsf(th)), y);
            if (!(beta > 0.f)) {
#pragma unroll
                for (int i = 0; i < MS; ++i) y[i] = 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < MS; ++i) s_y[i][t] = y[i];
    }
    __syncthreads();
    if (q.r >= q.n || 4 * q.g >= a.kp) return;
    const int64_t vs = a.nl * a.kp;
    const int64_t row = a.l_t0[q.tile] + (q.p - a.l_base[q.tile]);
    const int64_t o = q.p * a.kp + 4 * q.g;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < MS; ++i)
        if (i < a.steps) x = fma4v(ld4(&s_y[i][4 * q.g]), ld4(a.V + i * vs + o), x);
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (4 * q.g + c < a.k) W[row * a.k + 4 * q.g + c] = static_cast<T>(comp(x, c));
}

// ---------------------------------------------------------------- set-up
// Dense copy (both triangles) of each small tile, one CTA per tile.
template <typename VT>
__global__ void __launch_bounds__(256) k_fom_dense(const int64_t *s_t0, const int32_t *s_m, const int64_t *row_ptr,
                                                   const int32_t *col, const VT *val, float *Atiles) {
    __shared__ __align__(16) float sT[BS * BS];
    const int64_t t0 = s_t0[blockIdx.x];
    const int m = s_m[blockIdx.x];
    for (int e = threadIdx.x; e < BS * BS; e += blockDim.x) sT[e] = 0.f;
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const int64_t i = t0 + r;
        for (int64_t e = row_ptr[i + 1] - 1; e >= row_ptr[i]; --e) {
            const int64_t c = col[e];
            if (c < t0) break;
            const float v = static_cast<float>(val[e]);
            sT[r * BS + (c - t0)] = v;
            sT[(c - t0) * BS + r] = v;
        }
    }
    __syncthreads();
    float4 *dst = reinterpret_cast<float4 *>(Atiles + static_cast<int64_t>(blockIdx.x) * BS * BS);
    for (int e = threadIdx.x; e < BS * BS / 4; e += blockDim.x) dst[e] = reinterpret_cast<const float4 *>(sT)[e];
}

// Entries of each large-tile row inside its tile (the suffix of the sorted
// CSR row with col >= tile start): count (fill = false) or copy (fill = true).
template <bool FILL, typename VT>
__global__ void k_fom_rows(const int64_t *l_t0, const int32_t *l_m, const int64_t *l_base, const int64_t *row_ptr,
                           const int32_t *col, const VT *val, int64_t *cnt, const int64_t *rp, int32_t *lcol,
                           float *lval) {
    const int64_t t0 = l_t0[blockIdx.x];
    const int m = l_m[blockIdx.x];
    const int64_t base = l_base[blockIdx.x];
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const int64_t i = t0 + r;
        int64_t e0 = row_ptr[i + 1];
        while (e0 > row_ptr[i] && col[e0 - 1] >= t0) --e0;
        if (!FILL) {
            cnt[base + r] = row_ptr[i + 1] - e0;
        } else {
            int64_t o = rp[base + r];
            for (int64_t e = e0; e < row_ptr[i + 1]; ++e, ++o) {
                lcol[o] = static_cast<int32_t>(col[e] - t0);
                lval[o] = static_cast<float>(val[e]);
            }
        }
    }
}

template <typename VT>
cudaError_t fom_setup_impl(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const VT *val,
                           const int64_t *tile_ptr, int64_t ntiles) {
    FomTiles &F = h->fom;
    cudaStream_t s = h->stream;
    const int64_t n = h->T.n;
    std::vector<int64_t> tp;
    if (tile_ptr) {
        tp.assign(tile_ptr, tile_ptr + ntiles + 1);
    } else {
        for (int64_t a = 0; a < n; a += BS) tp.push_back(a);
        tp.push_back(n);
    }
    std::vector<int64_t> s_t0;
    std::vector<int32_t> s_m;
    std::vector<std::pair<int64_t, int64_t>> large;   // (size, start)
    for (size_t t = 0; t + 1 < tp.size(); ++t) {
        const int64_t m = tp[t + 1] - tp[t];
        if (m <= BS) {
            s_t0.push_back(tp[t]);
            s_m.push_back(static_cast<int32_t>(m));
        } else {
            large.emplace_back(m, tp[t]);
        }
    }
    std::stable_sort(large.begin(), large.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    F.n_small = static_cast<int64_t>(s_t0.size());
    F.n_large = static_cast<int64_t>(large.size());
    std::vector<int64_t> l_t0, l_base;
    std::vector<int32_t> l_m;
    int64_t nl = 0;
    for (const auto &q : large) {
        l_t0.push_back(q.second);
        l_m.push_back(static_cast<int32_t>(q.first));
        l_base.push_back(nl);
        nl += q.first;
        F.max_large = std::max<int32_t>(F.max_large, static_cast<int32_t>(q.first));
    }
    F.large_rows = nl;
    cudaError_t e = cudaSuccess;
    auto up_ = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
        cudaError_t r = dev_alloc(h, dst, std::max<size_t>(bytes, 16));
        if (r == cudaSuccess && bytes) r = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s);
        return r;
    };
    if (F.n_small) {
        e = up_(reinterpret_cast<void **>(&F.s_t0), s_t0.data(), sizeof(int64_t) * F.n_small);
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.s_m), s_m.data(), sizeof(int32_t) * F.n_small);
        if (e == cudaSuccess) e = dev_alloc(h, reinterpret_cast<void **>(&F.A), sizeof(float) * F.n_small * BS * BS);
        if (e != cudaSuccess) return e;
        k_fom_dense<VT><<<static_cast<unsigned>(F.n_small), 256, 0, s>>>(F.s_t0, F.s_m, row_ptr, col, val, F.A);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (F.n_large) {
        e = up_(reinterpret_cast<void **>(&F.l_t0), l_t0.data(), sizeof(int64_t) * F.n_large);
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.l_m), l_m.data(), sizeof(int32_t) * F.n_large);
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.l_base), l_base.data(), sizeof(int64_t) * F.n_large);
        if (e != cudaSuccess) return e;
        int64_t *d_cnt = nullptr;
        e = cudaMallocAsync(&d_cnt, sizeof(int64_t) * nl, s);
        if (e != cudaSuccess) return e;
        k_fom_rows<false, VT><<<static_cast<unsigned>(F.n_large), 256, 0, s>>>(
            F.l_t0, F.l_m, F.l_base, row_ptr, col, val, d_cnt, nullptr, nullptr, nullptr);
        e = cudaGetLastError();
        std::vector<int64_t> cnt(nl), rp(nl + 1);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int64_t) * nl, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(d_cnt, s);
        if (e != cudaSuccess) return e;
        rp[0] = 0;
        for (int64_t p = 0; p < nl; ++p) rp[p + 1] = rp[p] + cnt[p];
        const int64_t lnnz = rp[nl];
        // the tiles' lower triangles (local columns) into temporaries ...
        int64_t *d_rp = nullptr;
        int32_t *d_col = nullptr;
        float *d_val = nullptr;
        e = cudaMallocAsync(&d_rp, sizeof(int64_t) * (nl + 1), s);
        if (e == cudaSuccess) e = cudaMallocAsync(&d_col, sizeof(int32_t) * std::max<int64_t>(lnnz, 4), s);
        if (e == cudaSuccess) e = cudaMallocAsync(&d_val, sizeof(float) * std::max<int64_t>(lnnz, 4), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_rp, rp.data(), sizeof(int64_t) * (nl + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            k_fom_rows<true, VT><<<static_cast<unsigned>(F.n_large), 256, 0, s>>>(
                F.l_t0, F.l_m, F.l_base, row_ptr, col, val, nullptr, d_rp, d_col, d_val);
            e = cudaGetLastError();
        }
        std::vector<int32_t> lc(lnnz);
        std::vector<float> lv(lnnz);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lc.data(), d_col, sizeof(int32_t) * lnnz, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lv.data(), d_val, sizeof(float) * lnnz, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(d_rp, s);
        cudaFreeAsync(d_col, s);
        cudaFreeAsync(d_val, s);
        if (e != cudaSuccess) return e;
        // ... expanded on the host to both triangles: row c = its stored
        // entries (columns <= c, ascending) followed by the transposes of
        // the entries (r, c), r > c, in increasing r (so rows stay sorted)
        std::vector<int64_t> up(nl, 0), frp(nl + 1, 0);
        for (int64_t q = 0; q < F.n_large; ++q)
            for (int64_t r = 0; r < l_m[q]; ++r) {
                const int64_t p = l_base[q] + r;
                for (int64_t e2 = rp[p]; e2 < rp[p + 1]; ++e2)
                    if (lc[e2] < r) ++up[l_base[q] + lc[e2]];
            }
        for (int64_t p = 0; p < nl; ++p) frp[p + 1] = frp[p] + cnt[p] + up[p];
        F.large_nnz = frp[nl];
        std::vector<int32_t> fc(F.large_nnz);
        std::vector<float> fv(F.large_nnz);
        std::vector<int64_t> cur(nl);
        for (int64_t p = 0; p < nl; ++p) {
            cur[p] = frp[p];
            for (int64_t e2 = rp[p]; e2 < rp[p + 1]; ++e2, ++cur[p]) {
                fc[cur[p]] = lc[e2];
                fv[cur[p]] = lv[e2];
            }
        }
        for (int64_t q = 0; q < F.n_large; ++q)
            for (int64_t r = 0; r < l_m[q]; ++r) {
                const int64_t p = l_base[q] + r;
                for (int64_t e2 = rp[p]; e2 < rp[p + 1]; ++e2)
                    if (lc[e2] < r) {
                        const int64_t t = l_base[q] + lc[e2];
                        fc[cur[t]] = static_cast<int32_t>(r);
                        fv[cur[t]] = lv[e2];
                        ++cur[t];
                    }
            }
        e = up_(reinterpret_cast<void **>(&F.rp), frp.data(), sizeof(int64_t) * (nl + 1));
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.col), fc.data(), sizeof(int32_t) * F.large_nnz);
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.val), fv.data(), sizeof(float) * F.large_nnz);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host arrays above die with this scope
        F.scr_k = h->params.k;
        const int64_t kp_max = (F.scr_k + 3) & ~3;
        if (e == cudaSuccess)
            e = dev_alloc(h, reinterpret_cast<void **>(&F.scr), sizeof(float) * (MS + 1) * nl * kp_max);
        // the padding columns of the basis stay zero
        if (e == cudaSuccess) e = cudaMemsetAsync(F.scr, 0, sizeof(float) * (MS + 1) * nl * kp_max, s);
        // 64-row segments inside each large tile
        std::vector<int64_t> seg_p0;
        std::vector<int32_t> seg_n, seg_t;
        for (int64_t q = 0; q < F.n_large; ++q)
            for (int64_t off = 0; off < l_m[q]; off += SEG) {
                seg_p0.push_back(l_base[q] + off);
                seg_n.push_back(static_cast<int32_t>(std::min<int64_t>(SEG, l_m[q] - off)));
                seg_t.push_back(static_cast<int32_t>(q));
            }
        F.n_seg = static_cast<int64_t>(seg_p0.size());
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.seg_p0), seg_p0.data(), sizeof(int64_t) * F.n_seg);
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.seg_n), seg_n.data(), sizeof(int32_t) * F.n_seg);
        if (e == cudaSuccess) e = up_(reinterpret_cast<void **>(&F.seg_t), seg_t.data(), sizeof(int32_t) * F.n_seg);
        if (e == cudaSuccess)
            e = dev_alloc(h, reinterpret_cast<void **>(&F.acc), sizeof(float) * (MS * 2 + 1) * F.n_large * NV * 32);
        if (e != cudaSuccess) return e;
    }
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) F.ready = true;
    return e;
}

template <int L, typename T>
cudaError_t fom_launch(const lobpcg_ctx *h, int k, int steps, const T *R, const double *theta, T *W, cudaStream_t s) {
    const FomTiles &F = h->fom;
    if (F.n_small) {
        const size_t smem = sizeof(float) * ((BS + L) * PITCH + 2 * 8 * NV * 32);
        cudaError_t e = cudaFuncSetAttribute(k_fom_small<L, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_fom_small<L, T><<<static_cast<unsigned>(F.n_small), 256, smem, s>>>(k, steps, F.s_t0, F.s_m, F.A, R, theta,
                                                                             W);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (F.n_large) {
        if (k > F.scr_k) return cudaErrorInvalidValue;
        LargeArgs a{};
        a.k = k;
        a.kp = (k + 3) & ~3;
        a.steps = steps;
        a.nl = F.large_rows;
        a.nlt = F.n_large;
        a.seg_p0 = F.seg_p0;
        a.seg_n = F.seg_n;
        a.seg_t = F.seg_t;
        a.l_t0 = F.l_t0;
        a.l_base = F.l_base;
        a.rp = F.rp;
        a.lcol = F.col;
        a.lval = F.val;
        a.V = F.scr;
        a.acc = F.acc;
        a.accb = F.acc + static_cast<int64_t>(MS) * 2 * F.n_large * NV * 32;
        // sums of this call: the steps' slots and the norms
        cudaError_t e = cudaMemsetAsync(a.acc, 0, sizeof(float) * steps * 2 * F.n_large * NV * 32, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(a.accb, 0, sizeof(float) * F.n_large * 32, s);
        if (e != cudaSuccess) return e;
        constexpr int G = L / 4;
        const unsigned g = static_cast<unsigned>(F.n_seg);
        k_fl_norm<G, T><<<g, 64 * G, 0, s>>>(a, R);
        k_fl_start<G, T><<<g, 64 * G, 0, s>>>(a, R);
        for (int st = 0; st < steps; ++st) {
            k_fl_matvec<G><<<g, 64 * G, 0, s>>>(a, st, theta);
            k_fl_dots1<G><<<g, 64 * G, 0, s>>>(a, st);
            k_fl_dots2<G><<<g, 64 * G, 0, s>>>(a, st);
            if (st + 1 < steps) k_fl_next<G><<<g, 64 * G, 0, s>>>(a, st);
        }
        k_fl_finish<G, T><<<g, 64 * G, 0, s>>>(a, theta, W);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t fom_setup(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const void *val, bool val_fp64,
                      const int64_t *tile_ptr, int64_t ntiles) {
    if (val_fp64)
        return fom_setup_impl<double>(h, row_ptr, col, static_cast<const double *>(val), tile_ptr, ntiles);
    return fom_setup_impl<float>(h, row_ptr, col, static_cast<const float *>(val), tile_ptr, ntiles);
}

template <typename T>
cudaError_t fom_apply(const lobpcg_ctx *h, int k, const T *R, const double *theta, T *W, cudaStream_t s) {
    if (!h->fom.ready || k < 1 || k > 32) return cudaErrorInvalidValue;
    const int steps = h->params.fom_steps > 0 ? h->params.fom_steps : FOM_DEFAULT_STEPS;
    if (k <= 8) return fom_launch<8, T>(h, k, steps, R, theta, W, s);
    if (k <= 16) return fom_launch<16, T>(h, k, steps, R, theta, W, s);
    return fom_launch<32, T>(h, k, steps, R, theta, W, s);
}

template cudaError_t fom_apply<float>(const lobpcg_ctx *, int, const float *, const double *, float *, cudaStream_t);
template cudaError_t fom_apply<double>(const lobpcg_ctx *, int, const double *, const double *, double *,
                                       cudaStream_t);

}  // namespace lobpcg
