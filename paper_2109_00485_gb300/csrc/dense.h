// Launchers for the dense LOBPCG steps (dense.cu) and the preconditioners.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

namespace lobpcg {

// Up to six n x k blocks addressed as one n x (nb k) matrix [B_0 .. B_5].
template <typename T>
struct GemmBlocks {
    const T *p[6];
};

// Up to two outputs of k_combine: z[o] = A[:, c0[o]:] C[o]; C[o] is
// (na k - c0[o]) x k FP64 row-major.  norm_of: output whose squared column
// norms are accumulated (or -1).
template <typename T>
struct CombineOut {
    T *z[2];
    const double *C[2];
    int c0[2];
    int norm_of;
    float *Cf = nullptr;   // device scratch (>= 2 * 96 * 32 floats) for float32 coefficient copies
    int *err = nullptr;    // device error word: single float32 outputs may take the bulk-copy kernel
};

template <typename T>
cudaError_t launch_resid(int64_t n, int k, const T *X, const T *HX, const double *theta, const float *d, T *W,
                         int mode, double *norms, int num_sms, cudaStream_t s);
// Mixed-precision refinement: float64 residual into a float32 W, and the
// float64 X / HX update Z <- Z C + A (A float32) with a float32 copy of Z.
cudaError_t launch_resid_mixed(int64_t n, int k, const double *X, const double *HX, const double *theta,
                               const float *d, float *W, float *R32, int mode, double *norms, int num_sms,
                               cudaStream_t s);
cudaError_t launch_xupdate(int64_t n, int k, double *Z, const double *C, const float *A, float *Z32, int num_sms,
                           cudaStream_t s);
// M (ma x mb, FP64) = A^T B.  With LOBPCG_GRAM=umma in the environment,
// float32 blocks go to the tensor-memory kernel (gram_umma.cu) when it takes
// the shape and err (device error word for its bounded waits) is given;
// otherwise to the mma.sync kernel k_gram_tc.
template <typename T>
cudaError_t launch_gram(int64_t n, int k, int na, GemmBlocks<T> a, int nb, GemmBlocks<T> b, double *M, int num_sms,
                        cudaStream_t s, int *err = nullptr);
bool gram_umma_ok(int k, int na, const float *const *ap, int nb, const float *const *bp);
cudaError_t launch_gram_umma(int64_t n, int k, int na, const float *const *ap, int nb, const float *const *bp,
                             double *M, int *err, int num_sms, cudaStream_t s);
// One k x k output block of a Gram pair list (gram_ff.cu): M block at block
// row ro, block column co (units of k) = blk[a]^T blk[b].  GRAM_SYM: a
// symmetric block (only its lower half is computed, the upper half written
// as its transpose inside the same block); GRAM_MIRROR: the block is also
// written transposed at block (mro, mco).
constexpr int GRAM_SYM = 1;
constexpr int GRAM_MIRROR = 2;
struct GramPair {
    int a, b, ro, co, flags, mro, mco;
};
bool gram_pairs_ok(int k, int nblk, const float *const *blk, int npairs);
// gram_pairs_ok and the pairs' sub-tile units (k/4 squared per pair, fewer
// for GRAM_SYM) within what one CTA of the kernel holds.
bool gram_pairs_fit(int k, int nblk, const float *const *blk, int npairs, int units);
// M (ldm_rows x ldm, FP64, row-major; zeroed first when `zero`) += the
// listed blocks.  float32 blocks n x k, 16-byte aligned, k % 4 == 0,
// k <= 32, at most 8 distinct blocks and 16 pairs.  err: device error word
// for the bounded waits.
cudaError_t launch_gram_pairs(int64_t n, int k, int nblk, const float *const *blk, int npairs, const GramPair *pairs,
                              double *M, int ldm, int ldm_rows, bool zero, int *err, int num_sms, cudaStream_t s);
// update.cu: X <- S C, HX <- HS C, P <- S[:, k:] C[k:], HP <- HS[:, k:] C[k:]
// and W = R or D_theta^{-1} R (mode 0 / 1) with R = HX - X Theta, in place,
// plus norms = [||r_j||^2, ||x_j||^2] and colsq = ||p_j||^2 (zeroed here).
// S, HS: na (2 or 3) float32 n x k blocks, 16-byte aligned; k in {8, 16, 20}.
// update.cu: Z = [A_0 .. A_{na-1}] C (one float32 output, in place allowed),
// C (na k) x k FP64; k in {8, 16, 20}, na <= 3, 16-byte aligned blocks.
// The float64 refinement's dense steps in compensated float32 (mixed_df.cu,
// k <= 32): G = X^T [HX X] (k x 2k, zeroed first) from float64 X and HX,
// and the fused update below.
bool mixed_df_ok(int k);
cudaError_t launch_gram_x_df(int64_t n, int k, const double *X, const double *HX, double *G, int num_sms,
                             cudaStream_t s);
// Both updates and the next residual in one pass (mixed_df.cu): X <- X C + P,
// HX <- HX C + HP (float64; X32, HX32 float32 copies), then R32 = HX - X
// Theta, W = R32 (mode 0) or the diagonal-preconditioned R32 (mode 1), and
// norms (zeroed first) = (||r_j||^2, ||x_j||^2), as launch_resid_mixed.
// With C23 (float64 nz k x k: the W and P rows of the Ritz coefficients),
// Wb, HWb (the basis blocks W, HW) and colsq: P <- [W P] C23 and HP <- [HW HP]
// C23 in place first (float32; nz = 1 leaves the P block out), colsq =
// ||p_j||^2 (zeroed first); the X and HX updates then add these.
cudaError_t launch_xupdate2_df(int64_t n, int k, double *X, double *HX, const double *C, float *P, float *HP,
                               float *X32, float *HX32, const double *theta, const float *d, float *W, float *R32,
                               int mode, double *norms, int num_sms, cudaStream_t s, const float *Wb = nullptr,
                               const float *HWb = nullptr, const double *C23 = nullptr, int nz = 0,
                               double *colsq = nullptr);
bool combine_ff_ok(int k, int na, const float *const *blocks, const float *Z);
cudaError_t launch_combine_ff(int64_t n, int k, int na, const float *const *A, const double *C, float *Z, int *err,
                              int num_sms, cudaStream_t s);
bool update_post_ok(int k, int na, const float *const *blocks);
cudaError_t launch_update_post(int64_t n, int k, int na, const float *const *S, const float *const *HS,
                               float *X, float *P, float *HX, float *HP, float *W, const double *C,
                               const double *theta, const float *d, int mode, double *norms, double *colsq,
                               int *err, int num_sms, cudaStream_t s);
template <typename T>
cudaError_t launch_combine(int64_t n, int k, int na, GemmBlocks<T> a, int nout, CombineOut<T> out, double *colsq,
                           int num_sms, cudaStream_t s);
// G, O: m x m blocks with row stride ld (they may be the two halves of one
// m x 2m Gram matrix).
cudaError_t launch_rayleigh_ritz(int m, int k, int p0, const double *G, const double *O, int ld, const double *pscale,
                                 double *C, double *theta, int *status, cudaStream_t s);
cudaError_t launch_orth_factor(int k, const double *B, double *T, int *status, cudaStream_t s);

}  // namespace lobpcg
