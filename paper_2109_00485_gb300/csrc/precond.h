// Preconditioner launchers (precond.cu, mlp.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct lobpcg_ctx;

namespace lobpcg {

// Eigendecompositions of the 64-row diagonal tiles, from the caller's CSR
// (device pointers) at create.
cudaError_t bjacobi_setup(lobpcg_ctx *h, const int64_t *row_ptr, const int32_t *col, const void *val, bool val_fp64);

// W = K^{-1} R for mode 0 (identity), 1 (diagonal), 2 (block-Jacobi 64);
// R and W are n x k device blocks (may alias), theta k FP64 shifts (device).
template <typename T>
cudaError_t precond_apply(const lobpcg_ctx *h, int mode, int k, const T *R, const double *theta, T *W,
                          cudaStream_t s);

}  // namespace lobpcg
