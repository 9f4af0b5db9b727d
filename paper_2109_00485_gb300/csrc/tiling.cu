// Conversion of the caller's lower-triangle CSR into the tiled layout the
// SpMM streams (see internal.h), plus the per-matrix facts the solver needs:
// the diagonal d_i and the Gershgorin bound ||H||_G = max_i sum_j |h_ij|.
//
// All passes run on the device.  The row pointers are validated first, so
// no later kernel reads outside the arrays.
#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "internal.h"

namespace lobpcg {

// Thread per row: row_ptr monotone and in range; columns strictly
// increasing, 0 <= col <= row.  Records the first bad row.
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col, int *bad,
                           unsigned long long *bad_row) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t a = row_ptr[i], b = row_ptr[i + 1];
    bool ok = (a >= 0 && b >= a && b <= nnz);
    if (i == 0 && a != 0) ok = false;
    if (i == n - 1 && b != nnz) ok = false;
    if (ok) {
        int64_t prev = -1;
        for (int64_t e = a; e < b; ++e) {
            const int64_t c = col[e];
            if (c <= prev || c > i) { ok = false; break; }
            prev = c;
        }
    }
    if (!ok) {
        atomicExch(bad, 1);
        atomicMin(bad_row, static_cast<unsigned long long>(i));
    }
}

// Warp per row block (lanes 0..15 own its rows).  COUNT pass: number of
// chunks, padded entries, data words and full chunks per row block.  FILL
// pass: writes the entries and the chunk table at the offsets (chunks,
// words) from the COUNT pass.  vonly: complete tiles and complete diagonal
// triangles keep value words only.
template <bool FILL, typename VT>
__global__ void k_tile_rows(int64_t n, int64_t R, const int64_t *row_ptr, const int32_t *col, const VT *val,
                            int vonly, int64_t *cnt_chunks, int64_t *cnt_npad, int64_t *cnt_full,
                            int64_t *cnt_words, const int64_t *rb_chunk, const int64_t *rb_words, uint32_t *data,
                            ChunkRec *chunk) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    for (int64_t rb = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); rb < R;
         rb += nwarps) {
        const int64_t i = rb * TILE + lane;
        const bool valid = lane < TILE && i < n;
        int64_t p = valid ? row_ptr[i] : 0, e = valid ? row_ptr[i + 1] : 0;
        const int64_t dlo = rb * TILE;
        int64_t q = e;
        while (q > p && col[q - 1] >= dlo) --q;
        // diagonal chunk
        const int dcnt = static_cast<int>(e - q);
        const int dtot = warp_sum_i32(dcnt);
        const int dpad = (dtot + 3) & ~3;
        const bool dvo = vonly && dtot == TILE * (TILE + 1) / 2;   // complete triangle (only in a full row block)
        int64_t base = 0, cidx = 0, nch = 1, npad = dpad, nfull = 0, nwords = dvo ? dpad : 2 * dpad;
        if (FILL) {
            base = rb_words[rb];
            cidx = rb_chunk[rb];
            // words [base, base + dpad): indices (none when value-only); then dpad values
            uint32_t *ci = data + base, *cv = dvo ? ci : ci + dpad;
            const int o = warp_excl_scan_i32(dcnt);
            for (int t = 0; t < dcnt; ++t) {
                if (!dvo) ci[o + t] = static_cast<uint32_t>(col[q + t]) | (static_cast<uint32_t>(lane) << 28);
                cv[o + t] = __float_as_uint(static_cast<float>(val[q + t]));
            }
            if (lane < dpad - dtot) {
                if (!dvo) ci[dtot + lane] = IDX_PAD;
                cv[dtot + lane] = 0u;
            }
            if (lane == 0) {
                ChunkRec r;
                r.off = base; r.ct = static_cast<int32_t>(rb);
                r.info = dtot | DIAG_FLAG | (dvo ? VONLY_FLAG : 0) | (dpad << NPAD_SHIFT);
                chunk[cidx] = r;
            }
            base += dvo ? dpad : 2 * dpad;
            ++cidx;
        }
        // off-diagonal chunks: merge the 16 rows by column tile
        while (true) {
            const int ct_l = (p < q) ? (col[p] >> 4) : INT_MAX;
            const int m = warp_min_i32(ct_l);
            if (m == INT_MAX) break;
            int c_l = 0;
            while (p + c_l < q && (col[p + c_l] >> 4) == m) ++c_l;
            const int tot = warp_sum_i32(c_l);
            const int tpad = (tot + 3) & ~3;
            const bool tvo = vonly && tot == 256;
            if (FILL) {
                uint32_t *ci = data + base, *cv = tvo ? ci : ci + tpad;
                const int o = warp_excl_scan_i32(c_l);
                // a full chunk (all 256 entries of its tile) keeps its rows in
                // order, but stores column c of a row at position
                // 4 (c mod 4) + c / 4, so that the four columns c, c + 4,
                // c + 8, c + 12 one lane of the SpMM's tile products reads
                // are one 16-byte word
                const bool full = (tot == 256);
                for (int t = 0; t < c_l; ++t) {
                    const int pos = full ? 4 * (t & 3) + (t >> 2) : t;
                    if (!tvo) ci[o + pos] = static_cast<uint32_t>(col[p + t]) | (static_cast<uint32_t>(lane) << 28);
                    cv[o + pos] = __float_as_uint(static_cast<float>(val[p + t]));
                }
                if (lane < tpad - tot) { ci[tot + lane] = IDX_PAD; cv[tot + lane] = 0u; }
                if (lane == 0) {
                    ChunkRec r;
                    r.off = base; r.ct = m; r.info = tot | (tvo ? VONLY_FLAG : 0) | (tpad << NPAD_SHIFT);
                    chunk[cidx] = r;
                }
                base += tvo ? tpad : 2 * tpad;
                ++cidx;
            } else {
                ++nch;
                npad += tpad;
                nwords += tvo ? tpad : 2 * tpad;
                nfull += (tot == 256);
            }
            p += c_l;
        }
        if (!FILL && lane == 0) {
            cnt_chunks[rb] = nch;
            cnt_npad[rb] = npad;
            cnt_full[rb] = nfull;
            cnt_words[rb] = nwords;
        }
    }
}

// d_i = h_ii (last entry of row i when it is on the diagonal).
template <typename VT>
__global__ void k_diag(int64_t n, const int64_t *row_ptr, const int32_t *col, const VT *val, float *d) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t b = row_ptr[i + 1];
    d[i] = (b > row_ptr[i] && col[b - 1] == i) ? static_cast<float>(val[b - 1]) : 0.f;
}

// Row sums of |H| over full rows: own entries, then transposed ones.
template <typename VT>
__global__ void k_abs_rowsum(int64_t n, const int64_t *row_ptr, const int32_t *col, const VT *val, double *s) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        const double a = fabs(static_cast<double>(static_cast<float>(val[e])));
        acc += a;
        if (col[e] != i) atomicAdd(s + col[e], a);
    }
    atomicAdd(s + i, acc);
}

__global__ void k_max_nonneg(int64_t n, const double *s, unsigned long long *out) {
    double m = 0.0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        m = fmax(m, s[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(m)));
}

#define TRY(x)                                   \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return e_;        \
    } while (0)

template <typename VT>
static cudaError_t build_impl(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const VT *val,
                              std::string &err, lobpcg_status &st) {
    cudaStream_t s = h->stream;
    Tiled &T = h->T;
    const int64_t n = T.n, nnz = T.nnz, R = (n + TILE - 1) / TILE;
    T.R = R;
    const int tpb = 256;
    const int64_t gblocks = (n + tpb - 1) / tpb;

    // 1. validate
    int *d_bad = nullptr;
    unsigned long long *d_bad_row = nullptr, *d_gmax = nullptr;
    TRY(cudaMallocAsync(&d_bad, 32, s));  // flag at 0, bad row at 8, Gershgorin bits at 16
    d_bad_row = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(d_bad) + 8);
    d_gmax = d_bad_row + 1;
    // zero flag, set bad_row to max, zero gmax
    unsigned char init[24];
    std::memset(init, 0, sizeof(init));
    unsigned long long big = ~0ull;
    std::memcpy(init + 8, &big, 8);
    TRY(cudaMemcpyAsync(d_bad, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_validate<<<static_cast<unsigned>(gblocks), tpb, 0, s>>>(n, nnz, row_ptr, col, d_bad, d_bad_row);
    TRY(cudaGetLastError());
    int h_bad = 0;
    unsigned long long h_bad_row = 0;
    TRY(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRY(cudaMemcpyAsync(&h_bad_row, d_bad_row, sizeof(h_bad_row), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    if (h_bad) {
        cudaFreeAsync(d_bad, s);
        err = "matrix structure invalid at row " + std::to_string(h_bad_row) +
              " (row_ptr must be monotone with row_ptr[0]=0, row_ptr[n]=nnz; columns strictly increasing, 0<=col<=row)";
        st = LOBPCG_ERR_BOUNDS;
        return cudaSuccess;
    }

    // 2. count chunks per row block
    int64_t *d_cnt = nullptr;
    TRY(cudaMallocAsync(&d_cnt, sizeof(int64_t) * 4 * R, s));
    const int wpb = 8;
    const int64_t tblocks = std::min<int64_t>((R + wpb - 1) / wpb, 65535LL * 16);
    k_tile_rows<false, VT><<<static_cast<unsigned>(tblocks), wpb * 32, 0, s>>>(
        n, R, row_ptr, col, val, T.vonly, d_cnt, d_cnt + R, d_cnt + 2 * R, d_cnt + 3 * R, nullptr, nullptr,
        nullptr, nullptr);
    TRY(cudaGetLastError());
    std::vector<int64_t> cnt(4 * R);
    TRY(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int64_t) * 4 * R, cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    std::vector<int64_t> rb_chunk(R + 1), rb_words(R + 1);
    rb_chunk[0] = rb_words[0] = 0;
    int64_t full = 0, npad = 0;
    for (int64_t r = 0; r < R; ++r) {
        rb_chunk[r + 1] = rb_chunk[r] + cnt[r];
        rb_words[r + 1] = rb_words[r] + cnt[3 * R + r];
        npad += cnt[R + r];
        full += cnt[2 * R + r];
    }
    T.nchunks = rb_chunk[R];
    T.npad = npad;
    T.words = rb_words[R];
    T.full_chunks = full;

    // 3. allocate the tiled arrays and fill them
    TRY(dev_alloc(h, reinterpret_cast<void **>(&T.data), sizeof(uint32_t) * std::max<int64_t>(T.words, 8)));
    TRY(dev_alloc(h, reinterpret_cast<void **>(&T.chunk), sizeof(ChunkRec) * T.nchunks));
    TRY(dev_alloc(h, reinterpret_cast<void **>(&T.rb_chunk), sizeof(int64_t) * (R + 1)));
    // padded to a multiple of 4 entries plus 4 (zeros): kernels stage rows of
    // d by 16-byte bulk copies that may round a ragged last tile up
    const int64_t n_diag = (n + 3) / 4 * 4 + 4;
    TRY(dev_alloc(h, reinterpret_cast<void **>(&T.diag), sizeof(float) * n_diag));
    TRY(cudaMemsetAsync(T.diag, 0, sizeof(float) * n_diag, s));
    int64_t *d_rb_words = nullptr;
    TRY(cudaMallocAsync(&d_rb_words, sizeof(int64_t) * (R + 1), s));
    TRY(cudaMemcpyAsync(T.rb_chunk, rb_chunk.data(), sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, s));
    TRY(cudaMemcpyAsync(d_rb_words, rb_words.data(), sizeof(int64_t) * (R + 1), cudaMemcpyHostToDevice, s));
    k_tile_rows<true, VT><<<static_cast<unsigned>(tblocks), wpb * 32, 0, s>>>(
        n, R, row_ptr, col, val, T.vonly, nullptr, nullptr, nullptr, nullptr, T.rb_chunk, d_rb_words, T.data,
        T.chunk);
    TRY(cudaGetLastError());
    k_diag<VT><<<static_cast<unsigned>(gblocks), tpb, 0, s>>>(n, row_ptr, col, val, T.diag);
    TRY(cudaGetLastError());

    // 4. Gershgorin bound
    double *d_rowsum = nullptr;
    TRY(cudaMallocAsync(&d_rowsum, sizeof(double) * n, s));
    TRY(cudaMemsetAsync(d_rowsum, 0, sizeof(double) * n, s));
    k_abs_rowsum<VT><<<static_cast<unsigned>(gblocks), tpb, 0, s>>>(n, row_ptr, col, val, d_rowsum);
    TRY(cudaGetLastError());
    k_max_nonneg<<<std::max(1, std::min(h->num_sms * 4, static_cast<int>(gblocks))), tpb, 0, s>>>(n, d_rowsum, d_gmax);
    TRY(cudaGetLastError());
    unsigned long long gbits = 0;
    TRY(cudaMemcpyAsync(&gbits, d_gmax, sizeof(gbits), cudaMemcpyDeviceToHost, s));
    TRY(cudaStreamSynchronize(s));
    std::memcpy(&h->gershgorin, &gbits, sizeof(double));

    // 5. SpMM residency (warps hand out row-block groups among themselves
    //    through the work counter) and the counter itself
#ifndef SPMM_WARPS_PER_SM
#define SPMM_WARPS_PER_SM 16
#endif
    const int64_t want = static_cast<int64_t>(h->num_sms) * SPMM_WARPS_PER_SM;
    T.warps = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, R)));
    TRY(dev_alloc(h, reinterpret_cast<void **>(&T.sched), sizeof(int) * 4));

    TRY(cudaFreeAsync(d_rowsum, s));
    TRY(cudaFreeAsync(d_rb_words, s));
    TRY(cudaFreeAsync(d_cnt, s));
    TRY(cudaFreeAsync(d_bad, s));
    TRY(cudaStreamSynchronize(s));
    st = LOBPCG_OK;
    return cudaSuccess;
}

cudaError_t build_tiled(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const void *val, bool val_fp64,
                        std::string &err, lobpcg_status &st) {
    if (val_fp64) return build_impl<double>(h, row_ptr, col, static_cast<const double *>(val), err, st);
    return build_impl<float>(h, row_ptr, col, static_cast<const float *>(val), err, st);
}

}  // namespace lobpcg
