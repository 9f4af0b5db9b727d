// Internal state of a lobpcg handle and the launchers the C ABI calls.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include "lobpcg.h"
#include "mlp.h"

namespace lobpcg {

struct SolverState;
struct DavState;

// One 16-byte record per chunk (see Tiled).
struct __align__(16) ChunkRec {
    int64_t off;
    int32_t ct;
    int32_t info;
};
constexpr int NPAD_SHIFT = 20;
constexpr int VONLY_FLAG = 1 << 17;   // chunk info bit: value words only (a complete tile or diagonal triangle)

// Tiled copy of the stored lower triangle.
//
// Rows are grouped in row blocks of 16.  Within a row block the entries are
// grouped by 16-column tile ("chunks"); the diagonal chunk comes first, then
// the off-diagonal chunks in ascending tile order.  Inside a chunk entries
// keep CSR order (by row, then column), except in a chunk holding all 256
// entries of its tile: that one is the tile row by row, with column c of a
// row at position 4 (c mod 4) + c / 4 of the row.  Each chunk is padded to
// a multiple of 4 entries (16 bytes) and stored as one contiguous run of
// 2 npad words -- its npad index words, then its npad value words -- so one
// bulk copy moves a whole chunk.  With tile_format 1 a chunk holding all
// 256 entries of its tile, or the complete lower triangle (136 entries) of
// a diagonal tile, keeps only its npad value words (VONLY_FLAG): the
// positions of its entries are implied.
//   index word = col | (row_in_block << 28), or IDX_PAD for padding
//   value word = float32 bits (0 for padding)
//   chunk[c].off   first word of chunk c in data[]
//   chunk[c].ct    column tile of chunk c (col >> 4)
//   chunk[c].info  real entry count | DIAG_FLAG (diagonal chunk) |
//                  VONLY_FLAG (value words only) | npad << 20
//   rb_chunk[rb]   first chunk of row block rb (rb_chunk[R] = nchunks)
struct Tiled {
    int64_t n = 0, nnz = 0, R = 0, nchunks = 0, npad = 0, full_chunks = 0;
    int64_t words = 0;        // 32-bit words in data[]
    int vonly = 0;            // tile_format 1: complete tiles store value words only
    uint32_t *data = nullptr;
    struct ChunkRec *chunk = nullptr;
    int64_t *rb_chunk = nullptr;
    int32_t warps = 0;        // SpMM warps launched
    int *sched = nullptr;     // SpMM work counter (row-block groups handed out)
    float *diag = nullptr;   // d_i = h_ii (float32)
};

// Float64-vector SpMM (spmm_df.cu): the off-diagonal chunks listed by
// column tile (col_list[col_ptr[ct] .. col_ptr[ct + 1]): (chunk, row block),
// in row-block order), built on first use; x_hi, x_lo of the last call
// (x_lo at xs + xs_stride), allocated for up to xs_k columns.
struct DfIndex {
    int64_t *col_ptr = nullptr;
    int2 *col_list = nullptr;
    float *xs = nullptr;
    int xs_k = 0;
    int64_t xs_stride = 0;
};

// Diagonal tiles of the FOM preconditioner (fom.cu).  Small tiles (<= 64
// rows): dense FP32 64 x 64 blocks, both triangles, zero outside the m x m
// corner, one per small tile in s_t0 order.  Large tiles (> 64 rows), in
// decreasing size: each tile as a CSR of both triangles over the rows of
// the large tiles packed one after another (tile q starts at packed row
// l_base[q]), local column indices, cut into segments of <= 64 rows inside
// one tile; scr holds the Krylov basis and work vector of every large-tile
// row (7 blocks of large_rows x scr_k floats), acc the per-tile sums.
struct FomTiles {
    int64_t n_small = 0, n_large = 0, large_rows = 0, large_nnz = 0;
    int32_t max_large = 0;
    int64_t *s_t0 = nullptr;
    int32_t *s_m = nullptr;
    float *A = nullptr;
    int64_t *l_t0 = nullptr;
    int32_t *l_m = nullptr;
    int64_t *l_base = nullptr;
    int64_t *rp = nullptr;        // [large_rows + 1]
    int32_t *col = nullptr;
    float *val = nullptr;
    float *scr = nullptr;
    int32_t scr_k = 0;
    int64_t n_seg = 0;
    int64_t *seg_p0 = nullptr;
    int32_t *seg_n = nullptr;
    int32_t *seg_t = nullptr;
    float *acc = nullptr;
    bool ready = false;
};

}  // namespace lobpcg

struct lobpcg_ctx {
    lobpcg::Tiled T;
    lobpcg_params params{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    double gershgorin = 0.0;
    int *d_err = nullptr;        // device error word (DevErr)
    int *h_err = nullptr;        // pinned mirror
    int64_t device_bytes = 0;
    std::vector<void *> allocs;  // every device allocation, freed at destroy
    float *stage_x = nullptr;    // device staging of host X / Y blocks (spmm_sym with host pointers)
    float *stage_y = nullptr;
    size_t stage_k = 0;
    float *bj_Q = nullptr;       // block-Jacobi: per 64-row tile eigenvectors (64 x 64) and eigenvalues
    float *bj_lam = nullptr;
    lobpcg::FomTiles fom;        // FOM preconditioner tiles (fom.cu)
    lobpcg::DfIndex df;          // float64-vector SpMM (spmm_df.cu)
    lobpcg::SolverState *solver = nullptr;  // workspaces of lobpcg_solve (solver.cu)
    lobpcg::DavState *dav = nullptr;        // workspaces of lobpcg_davidson (solver.cu), made on first use
    lobpcg::Mlp mlp;                         // learned tile preconditioner (mlp.cu)
    std::string last_error;
};

namespace lobpcg {

// Every buffer, stream and graph of a handle belongs to the device that was
// current at create, so every call that touches the device must run with
// that device current.  Returns false (with the reason in last_error) when
// another device is current or the current device cannot be read.
inline bool device_ok(lobpcg_ctx *h) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->last_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return false;
    }
    if (cur != h->device) {
        h->last_error = "the handle was created on device " + std::to_string(h->device) + " but device " +
                        std::to_string(cur) + " is current; make the handle's device current first";
        return false;
    }
    return true;
}

// tiling.cu
cudaError_t build_tiled(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const void *val,
                        bool val_fp64, std::string &err, lobpcg_status &st);

// spmm_sym.cu
cudaError_t launch_spmm_sym_f32(const lobpcg_ctx *h, const float *X, float *Y, int k, cudaStream_t s);
cudaError_t launch_spmm_sym_f64(lobpcg_ctx *h, const double *X, double *Y, int k, cudaStream_t s);
// spmm_df.cu: the float64-vector product in compensated float32 (even k <= 32)
bool spmm_df_ok(int k, const double *X, const double *Y);
cudaError_t launch_spmm_sym_df(lobpcg_ctx *h, const double *X, double *Y, int k, cudaStream_t s);

// helpers in api.cu
cudaError_t dev_alloc(lobpcg_ctx *h, void **p, size_t bytes);

// solver.cu
cudaError_t solver_setup(lobpcg_ctx *h);
void solver_release(lobpcg_ctx *h);
lobpcg_status solve(lobpcg_ctx *h, float *X, bool x_on_host, double *evals, double *resid, lobpcg_stats *st,
                    std::string &err);
cudaError_t copy_x_f64(lobpcg_ctx *h, double *out);
lobpcg_status davidson(lobpcg_ctx *h, float *X, bool x_on_host, int max_blocks, double *evals, double *resid,
                       lobpcg_stats *st, std::string &err);
lobpcg_status iterate(lobpcg_ctx *h, const float *X0, bool x_on_host, int steps, double *theta_out,
                      lobpcg_stats *st, std::string &err, int harvest = 0);

}  // namespace lobpcg
