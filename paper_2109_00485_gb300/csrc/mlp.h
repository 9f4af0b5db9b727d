// Learned tile preconditioner (mlp.cu): sizes, packed layout, launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct lobpcg_ctx;

namespace lobpcg {

constexpr int MLP_TILE = 64;     // rows per diagonal tile
constexpr int MLP_KIN = 144;     // 129 inputs padded to a multiple of 16
constexpr int MLP_NHID = 256;
constexpr int MLP_NOUT = 64;
constexpr float MLP_CLIP = 1e3f;
constexpr int MLP_BATCH = 4096;
// packed parameters on the device: W1 [256][144] | b1 [256] | W2 [64][256] | b2 [64]
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_NHID * MLP_KIN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_NHID;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_NOUT * MLP_NHID;
constexpr int MLP_NPARAM = MLP_OFF_B2 + MLP_NOUT;
// the caller's layout: W1 [256][129] | b1 | W2 [64][256] | b2
constexpr int MLP_NPARAM_CALLER = MLP_NHID * 129 + MLP_NHID + MLP_NOUT * MLP_NHID + MLP_NOUT;

struct Mlp {
    float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;   // params, grads, Adam moments
    int64_t cap_apply = 0;        // (tile, column) pairs of one apply on the handle's block size
    float *Xp = nullptr, *Tp = nullptr;   // harvested pairs (inputs, targets)
    unsigned long long *d_count = nullptr;
    int64_t cap_pairs = 0;
    uint64_t keep = 0;            // harvest keep threshold (of 2^32)
    int step = 0;                 // Adam step count
    bool ready = false;           // parameters set or trained
};

cudaError_t mlp_setup(lobpcg_ctx *h);
void mlp_release(lobpcg_ctx *h);
cudaError_t mlp_set_params(lobpcg_ctx *h, const float *src, bool on_host);
cudaError_t mlp_get_params(lobpcg_ctx *h, float *dst, bool on_host, bool grads);
cudaError_t mlp_forward_rows(lobpcg_ctx *h, const float *X129, int64_t B, float *Y);
cudaError_t mlp_grad_rows(lobpcg_ctx *h, const float *X129, const float *T, int64_t B, double *loss_host);
cudaError_t mlp_adam(lobpcg_ctx *h, float lr);
cudaError_t mlp_init(lobpcg_ctx *h, uint64_t seed);
cudaError_t mlp_apply(lobpcg_ctx *h, int k, const float *R, const double *theta, float *W, cudaStream_t s);
cudaError_t mlp_alloc_pairs(lobpcg_ctx *h, int64_t cap, int harvest_iters);
cudaError_t mlp_harvest(lobpcg_ctx *h, int k, const float *R, const float *Wt, const double *theta, int iter);
cudaError_t mlp_train(lobpcg_ctx *h, int epochs, float lr, double *loss_hist, int64_t *npairs_out);

}  // namespace lobpcg
