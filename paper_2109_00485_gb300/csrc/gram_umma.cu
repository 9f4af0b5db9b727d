// Gram matrices M = A^T B (Section 3.4 Gram blocks; Cholesky-QR's W^T W and
// X^T W) on the fifth-generation tensor cores: tcgen05.mma with TF32
// operands from shared memory and FP32 accumulators in tensor memory.
//
// A = [A_0 .. A_{na-1}] (n x ma), B = [B_0 .. B_{nb-1}] (n x mb), every block
// float32 n x k row-major.  The product is formed as D = B^T A (the MMA's M
// dimension runs over B's columns, padded to 128; N over A's columns, padded
// to a multiple of 16; K over rows), so M = D^T.  FP32-level products come
// from the split x = hi + lo with hi = x truncated to TF32 and lo = x - hi
// (exact): a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, three MMAs per K-step.
// The tensor core reads an FP32 bit pattern as TF32 by ignoring its low 13
// bits, so the hi operand is the value itself.
//
// One CTA per SM walks 32-row tiles (tile = blockIdx.x + i gridDim.x):
//   warp 0      bulk-copies the tile of every distinct block into a raw
//               stage (6 stages), completing on an mbarrier;
//   warps 1-8   copy each raw tile into the K-major operand layout of the
//               MMA (128-byte swizzle: 8-row x 128-byte atoms, the 16-byte
//               chunk c of row r at chunk c ^ (r % 8)), as hi and lo, and
//               drain each tensor-memory accumulator, one accumulation
//               period (two tiles) after its last MMA was issued, into
//               Kahan-compensated FP32 sums (64-row partial sums, as in the
//               CUDA-core Gram); warp w reads tensor-memory lanes
//               32 (w % 4) .. + 31, warps 1-4 the first half of the
//               accumulator columns and warps 5-8 the second;
//   warp 9      allocates tensor memory and one lane issues the MMAs, twelve
//               per tile, alternating between two accumulators so that a
//               drain overlaps the following tiles.
// At the end each thread adds its sums (FP64) to M with atomics.  Every wait
// is bounded; on a timeout the kernel records DEV_TIMEOUT, lets its copies
// and MMAs finish, frees its tensor memory and returns.
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"

namespace lobpcg {

namespace {

constexpr int UG_KT = 32;        // rows per tile (four K-steps of 8; one 128-byte swizzle atom along K)
constexpr int UG_RAW = 12;       // most raw stages (fitted to shared memory)
constexpr int UG_OPS = 3;        // operand stages
constexpr int UG_DRAIN = 2;      // tiles per accumulation period
constexpr int UG_MU = 128;       // MMA M (B's columns, padded)
constexpr int UG_MAXNU = 64;     // largest N (A's columns, padded to 16)
constexpr int UG_CONV = 8;                        // converter warps (1..8)
constexpr int UG_THREADS = 32 * (UG_CONV + 2);
constexpr int UG_TMEM_COLS = 128;                 // two accumulators of up to 64 columns
constexpr int UG_SBO = 1024;                      // bytes between the 8-row groups of an operand tile

struct UgArgs {
    int64_t n;
    int k;
    int nuq;                 // distinct blocks staged per tile
    int nraw;                // raw stages (<= UG_RAW, fitted to shared memory)
    const float *blk[12];    // their pointers
    int ma, mb, nu;          // nu = ma rounded up to 16
    int mapA[UG_MU];         // column m of B: raw offset (floats) in a stage, or -1 past mb
    int mapB[UG_MAXNU];      // column n of A: raw offset, or -1 past ma
    double *M;               // ma x mb, row-major, accumulated into
    int *err;
};

struct UgSmem {
    uint32_t off_opA, off_opB, off_raw, bytes;   // bytes in dynamic shared memory
};

__host__ __device__ inline UgSmem ug_layout(int nuq, int k, int nu, int nraw) {
    UgSmem L;
    const uint32_t opA = UG_OPS * 2u * UG_MU * UG_KT * 4u;
    const uint32_t opB = UG_OPS * 2u * static_cast<uint32_t>(nu) * UG_KT * 4u;
    const uint32_t raw = static_cast<uint32_t>(nraw * nuq) * UG_KT * static_cast<uint32_t>(k) * 4u;
    L.off_opA = 0;
    L.off_opB = opA;
    L.off_raw = opA + opB;
    L.bytes = opA + opB + raw;
    return L;
}

// Byte offset of element (row r, k-index kk) in a K-major operand tile with
// the 128-byte swizzle: row r's 128 bytes (its 32 k-values) at
// (r / 8) 1024 + (r % 8) 128, 16-byte chunk kk / 4 stored at chunk
// (kk / 4) ^ (r % 8).  Tiles start on 1024-byte boundaries.
__device__ __forceinline__ uint32_t op_off(int r, int kk) {
    return static_cast<uint32_t>((r >> 3) * UG_SBO + (r & 7) * 128 + ((((kk >> 2) ^ (r & 7)) & 7) << 4) + (kk & 3) * 4);
}

// Shared-memory matrix descriptor: start address, stride byte offset (next
// 8-row group) 1024, descriptor version 1 (bits 46-47), 128-byte swizzle
// (bits 61-63 = 2); the leading byte offset is unused with this swizzle
// along K.  A K-step starts 32 bytes further into the atom.
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr) {
    uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(1) << 16;
    d |= static_cast<uint64_t>((static_cast<uint32_t>(UG_SBO) >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;
    d |= static_cast<uint64_t>(2) << 61;
    return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator (bits 4-5 = 1), TF32
// A and B (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4
// at bits 24-28.
__device__ __forceinline__ uint32_t mma_idesc(int nu) {
    return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(nu >> 3) << 17) |
           (static_cast<uint32_t>(UG_MU >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive accumulator columns of this warp's 32 tensor-memory lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int lds_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// Bounded wait; on a timeout records the error and sets `bad`.
__device__ __forceinline__ bool wait_ok(uint64_t *bar, uint32_t parity, int *err, bool &bad) {
    if (bad) return false;
    if (mbar_wait_bounded(bar, parity)) return true;
    atomicExch(err, DEV_TIMEOUT);
    bad = true;
    return false;
}

__global__ void __launch_bounds__(UG_THREADS, 1) k_gram_umma(const __grid_constant__ UgArgs a) {
    extern __shared__ __align__(1024) unsigned char ug_smem[];
    __shared__ __align__(8) uint64_t raw_full[UG_RAW], raw_empty[UG_RAW], op_full[UG_OPS], op_empty[UG_OPS],
        acc_full[2], acc_empty[2], fin_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int mapA[UG_MU], mapB[UG_MAXNU];
    const UgSmem L = ug_layout(a.nuq, a.k, a.nu, a.nraw);
    const int NR = a.nraw;
    // swizzled operand tiles start on 1024-byte boundaries (1 KB of slack is allocated)
    unsigned char *base = ug_smem + ((1024u - (smem_addr(ug_smem) & 1023u)) & 1023u);
    unsigned char *opA = base + L.off_opA;   // [stage][hi, lo][MU x KT] K-major
    unsigned char *opB = base + L.off_opB;   // [stage][hi, lo][nu x KT]
    float *raw = reinterpret_cast<float *>(base + L.off_raw);   // [stage][block][KT][k]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = a.k, KTk = UG_KT * k;
    const uint32_t opA_bytes = UG_MU * UG_KT * 4u, opB_bytes = static_cast<uint32_t>(a.nu) * UG_KT * 4u;
    const int64_t ntile = (a.n + UG_KT - 1) / UG_KT;
    const int my_tiles = (blockIdx.x < ntile) ? static_cast<int>((ntile - 1 - blockIdx.x) / gridDim.x + 1) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NR; ++s) { mbar_init(&raw_full[s], 1); mbar_init(&raw_empty[s], UG_CONV); }
        for (int s = 0; s < UG_OPS; ++s) { mbar_init(&op_full[s], UG_CONV); mbar_init(&op_empty[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], UG_CONV); }
        mbar_init(&fin_bar, 1);
        abort_flag = 0;
        fence_proxy_async();
    }
    for (int m = threadIdx.x; m < UG_MU; m += blockDim.x) mapA[m] = a.mapA[m];
    for (int m = threadIdx.x; m < UG_MAXNU; m += blockDim.x) mapB[m] = a.mapB[m];
    // operand tiles start zeroed: rows past mb (A) and ma (B) are never written
    for (uint32_t e = threadIdx.x; e < L.off_raw / 16; e += blockDim.x)
        reinterpret_cast<float4 *>(base)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    fence_proxy_async();
    if (warp == UG_CONV + 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(UG_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    bool bad = false;

    if (warp == 0) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            int issued = 0;
            for (int i = 0; i < my_tiles; ++i) {
                const int rs = i % NR;
                if (i >= NR && !wait_ok(&raw_empty[rs], ((i / NR) - 1) & 1, a.err, bad)) break;
                if (abort_flag) break;
                const int64_t tile = blockIdx.x + static_cast<int64_t>(i) * gridDim.x;
                const int64_t r0 = tile * UG_KT;
                const int rows = static_cast<int>(a.n - r0 < UG_KT ? a.n - r0 : UG_KT);
                const uint32_t bytes = static_cast<uint32_t>(rows * k) * 4u;
                mbar_arrive_expect_tx(&raw_full[rs], bytes * static_cast<uint32_t>(a.nuq));
                for (int q = 0; q < a.nuq; ++q)
                    bulk_g2s(raw + (rs * a.nuq + q) * KTk, a.blk[q] + r0 * k, bytes, &raw_full[rs], pol);
                issued = i + 1;
            }
            // copies still landing must finish before the CTA's shared memory goes
            for (int i = (issued > NR ? issued - NR : 0); i < issued; ++i)
                mbar_wait_bounded(&raw_full[i % NR], (i / NR) & 1);
        }
    } else if (warp == UG_CONV + 1) {
        // ---------------------------------------------------------------- MMA issue
        if (lane == 0) {
            const uint32_t idesc = mma_idesc(a.nu);
            const uint32_t sA = smem_addr(opA), sB = smem_addr(opB);
            for (int i = 0; i < my_tiles; ++i) {
                const int os = i % UG_OPS;
                if (!wait_ok(&op_full[os], (i / UG_OPS) & 1, a.err, bad)) break;
                const int p = i / UG_DRAIN, b = p & 1;
                const bool first = (i % UG_DRAIN) == 0;
                if (first && p >= 2 && !wait_ok(&acc_empty[b], ((p >> 1) - 1) & 1, a.err, bad)) break;
                tc_fence_after();
                const uint32_t d = tmem + static_cast<uint32_t>(b * (UG_TMEM_COLS / 2));
                const uint32_t aHi = sA + os * 2 * opA_bytes, aLo = aHi + opA_bytes;
                const uint32_t bHi = sB + os * 2 * opB_bytes, bLo = bHi + opB_bytes;
#pragma unroll
                for (int ks = 0; ks < UG_KT / 8; ++ks) {
                    const uint32_t o = ks * 32;    // 8 tf32 values along K
                    umma_tf32(d, op_desc(aLo + o), op_desc(bHi + o), idesc, (first && ks == 0) ? 0u : 1u);
                    umma_tf32(d, op_desc(aHi + o), op_desc(bLo + o), idesc, 1u);
                    umma_tf32(d, op_desc(aHi + o), op_desc(bHi + o), idesc, 1u);
                }
                umma_commit(&op_empty[os]);
                if ((i % UG_DRAIN) == UG_DRAIN - 1 || i == my_tiles - 1) umma_commit(&acc_full[b]);
            }
            // every MMA issued has completed before tensor memory is released
            umma_commit(&fin_bar);
            mbar_wait_bounded(&fin_bar, 0);
        }
    } else {
        // ---------------------------------------------------------------- convert + drain (warps 1-8)
        const int cw = warp - 1;                       // converter index 0..7
        const int q4 = warp & 3;                       // tensor-memory lane quadrant of this warp
        const int half = cw >> 2;                      // accumulator column half drained by this warp
        const int mi = lane >> 2, ki = lane & 3;       // position in a core matrix
        const int ncoreA = (a.mb + 7) >> 3, ncoreB = (a.ma + 7) >> 3;
        const int items = (ncoreA + ncoreB) * (UG_KT / 4);
        const int hc = a.nu >> 1;                      // columns per half (a multiple of 8)
        constexpr int HMAX = UG_MAXNU / 2;
        float sum[HMAX], cmp[HMAX];
#pragma unroll
        for (int c = 0; c < HMAX; ++c) sum[c] = cmp[c] = 0.f;
        auto drain = [&](int p) {
            const int b = p & 1;
            wait_ok(&acc_full[b], (p >> 1) & 1, a.err, bad);
            bad = __any_sync(0xffffffffu, bad);   // tcgen05.ld needs the whole warp
            if (bad) return;
            tc_fence_after();
            const uint32_t base_t = tmem + (static_cast<uint32_t>(32 * q4) << 16) +
                                    static_cast<uint32_t>(b * (UG_TMEM_COLS / 2) + half * hc);
#pragma unroll
            for (int c0 = 0; c0 < HMAX; c0 += 8) {
                if (c0 < hc) {
                    float v[8];
                    tmem_ld8(base_t + c0, v);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float y = v[q] - cmp[c0 + q];
                        const float t = sum[c0 + q] + y;
                        cmp[c0 + q] = (t - sum[c0 + q]) - y;
                        sum[c0 + q] = t;
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        };
        int drained = 0;   // accumulation periods drained
        for (int i = 0; i < my_tiles && !bad; ++i) {
            const int rs = i % NR, os = i % UG_OPS;
            wait_ok(&raw_full[rs], (i / NR) & 1, a.err, bad);
            if (i >= UG_OPS) wait_ok(&op_empty[os], ((i / UG_OPS) - 1) & 1, a.err, bad);
            bad = __any_sync(0xffffffffu, bad);   // the warp leaves together
            if (bad) break;
            const int64_t tile = blockIdx.x + static_cast<int64_t>(i) * gridDim.x;
            const int rows = static_cast<int>(a.n - tile * UG_KT < UG_KT ? a.n - tile * UG_KT : UG_KT);
            // shared-memory (32-bit) addresses: explicit ld/st.shared
            const uint32_t rst = smem_addr(raw) + static_cast<uint32_t>(rs * a.nuq * KTk) * 4u;
            const uint32_t aHi = smem_addr(opA) + os * 2 * opA_bytes;
            const uint32_t bHi = smem_addr(opB) + os * 2 * opB_bytes;
            const uint32_t mA = smem_addr(mapA), mB = smem_addr(mapB);
            // items it = cw + 8 j: four at a time, loads first
            for (int it0 = cw; it0 < items; it0 += 4 * UG_CONV) {
                float x[4];
                uint32_t dst[4], lo[4];
                bool ok[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int it = it0 + u * UG_CONV;
                    const int kc = it & (UG_KT / 4 - 1), g = it / (UG_KT / 4);
                    const bool isA = g < ncoreA;
                    const int r = 8 * (isA ? g : g - ncoreA) + mi, kk = 4 * kc + ki;
                    ok[u] = it < items;
                    const int src = ok[u] ? lds_s32((isA ? mA : mB) + 4u * static_cast<uint32_t>(r)) : -1;
                    x[u] = (src >= 0 && kk < rows) ? lds_f32(rst + 4u * static_cast<uint32_t>(src + kk * k)) : 0.f;
                    dst[u] = (isA ? aHi : bHi) + op_off(r, kk);
                    lo[u] = isA ? opA_bytes : opB_bytes;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (ok[u]) {
                        const float hi = __uint_as_float(__float_as_uint(x[u]) & 0xFFFFE000u);
                        sts_f32(dst[u], x[u]);
                        sts_f32(dst[u] + lo[u], x[u] - hi);
                    }
                }
            }
            fence_proxy_async();   // operand writes visible to the tensor core
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&raw_empty[rs]);
                mbar_arrive(&op_full[os]);
            }
            // drain a period once the next period's tiles are converted too
            // (its MMAs have had a whole period to finish)
            if ((i + 1) % UG_DRAIN == 0 && (i + 1) / UG_DRAIN >= 2) drain(drained++);
        }
        while (!bad && drained * UG_DRAIN < my_tiles) drain(drained++);
        if (bad) abort_flag = 1;
        // M[n][m] += sum over this CTA, m = tensor-memory lane, n = column
        const int m = 32 * q4 + lane;
        if (!bad && m < a.mb) {
            for (int c = 0; c < HMAX; ++c) {
                const int col = half * hc + c;
                if (c < hc && col < a.ma)
                    atomicAdd(&a.M[col * a.mb + m], static_cast<double>(sum[c]) - static_cast<double>(cmp[c]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == UG_CONV + 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UG_TMEM_COLS) : "memory");
}

}  // namespace

// Eligible: float32, k % 4 == 0, 16-byte aligned blocks, ma <= 64, mb <= 128.
bool gram_umma_ok(int k, int na, const float *const *ap, int nb, const float *const *bp) {
    const int ma = na * k, mb = nb * k;
    if (k % 4 != 0 || ma > UG_MAXNU || mb > UG_MU || na + nb > 12) return false;
    for (int q = 0; q < na; ++q)
        if (reinterpret_cast<uintptr_t>(ap[q]) & 15u) return false;
    for (int q = 0; q < nb; ++q)
        if (reinterpret_cast<uintptr_t>(bp[q]) & 15u) return false;
    return true;
}

cudaError_t launch_gram_umma(int64_t n, int k, int na, const float *const *ap, int nb, const float *const *bp,
                             double *M, int *err, int num_sms, cudaStream_t s) {
    UgArgs a{};
    a.n = n;
    a.k = k;
    a.ma = na * k;
    a.mb = nb * k;
    a.nu = (a.ma + 15) / 16 * 16;
    a.M = M;
    a.err = err;
    // distinct blocks (A and B often share S)
    int nuq = 0;
    auto uq = [&](const float *p) {
        for (int q = 0; q < nuq; ++q)
            if (a.blk[q] == p) return q;
        a.blk[nuq] = p;
        return nuq++;
    };
    const int KTk = UG_KT * k;
    for (int m = 0; m < UG_MU; ++m) a.mapA[m] = -1;
    for (int m = 0; m < UG_MAXNU; ++m) a.mapB[m] = -1;
    for (int q = 0; q < nb; ++q) {
        const int u = uq(bp[q]);
        for (int c = 0; c < k; ++c) a.mapA[q * k + c] = u * KTk + c;
    }
    for (int q = 0; q < na; ++q) {
        const int u = uq(ap[q]);
        for (int c = 0; c < k; ++c) a.mapB[q * k + c] = u * KTk + c;
    }
    a.nuq = nuq;
    a.nraw = UG_RAW;
    while (a.nraw > 2 && ug_layout(nuq, k, a.nu, a.nraw).bytes > 200u * 1024u) --a.nraw;
    const UgSmem L = ug_layout(nuq, k, a.nu, a.nraw);
    if (L.bytes > 200u * 1024u) return cudaErrorInvalidValue;   // (not reached for ma <= 64, mb <= 128, k <= 128)
    cudaError_t e = cudaMemsetAsync(M, 0, sizeof(double) * a.ma * a.mb, s);
    if (e != cudaSuccess) return e;
    const uint32_t smem = L.bytes + 1024u;   // slack for the 1024-byte alignment
    e = cudaFuncSetAttribute(k_gram_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    const int64_t ntile = (n + UG_KT - 1) / UG_KT;
    const int blocks = static_cast<int>(ntile < num_sms ? ntile : num_sms);
    k_gram_umma<<<blocks > 0 ? blocks : 1, UG_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lobpcg
