// Preconditioner launchers (precond.cu, mlp.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct lobpcg_ctx;

namespace lobpcg {

// Eigendecompositions of the 64-row diagonal tiles, from the caller's CSR
// (device pointers) at create.
cudaError_t bjacobi_setup(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const void *val, bool val_fp64);

// FOM form (mode 4, fom.cu): the diagonal tiles of the row partition
// tile_ptr (host, ntiles + 1 boundaries; NULL: 64-row tiles) -- tiles of at
// most 64 rows as dense FP32 blocks, larger ones as a local CSR of their
// lower triangle -- and the scratch the larger ones iterate in.
cudaError_t fom_setup(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const void *val, bool val_fp64,
                      const int64_t *tile_ptr, int64_t ntiles);
template <typename T>
cudaError_t fom_apply(const lobpcg_ctx *h, int k, const T *R, const double *theta, T *W, cudaStream_t s);
constexpr int FOM_DEFAULT_STEPS = 4;   // FOM iterations when params.fom_steps is 0
constexpr int FOM_MAX_STEPS = 6;
constexpr int FOM_SMALL = 64;          // tiles of at most this many rows run from shared memory

// W = K^{-1} R for mode 0 (identity), 1 (diagonal), 2 (block-Jacobi 64),
// 3 (learned tile network), 4 (FOM on the shifted 64-row tiles);
// R and W are n x k device blocks (may alias), theta k FP64 shifts (device).
template <typename T>
cudaError_t precond_apply(const lobpcg_ctx *h, int mode, int k, const T *R, const double *theta, T *W,
                          cudaStream_t s);

}  // namespace lobpcg
