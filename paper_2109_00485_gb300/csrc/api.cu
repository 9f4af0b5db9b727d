// C ABI: handle lifetime, argument checks and dispatch to the kernels.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"
#include "internal.h"
#include "lobpcg.h"
#include "precond.h"
#include "mlp.h"

using namespace lobpcg;

namespace {
thread_local std::string g_create_error;

lobpcg_status fail(lobpcg_ctx *h, lobpcg_status st, const std::string &msg) {
    if (h) h->last_error = msg; else g_create_error = msg;
    return st;
}

lobpcg_status cuda_fail(lobpcg_ctx *h, cudaError_t e, const char *where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? LOBPCG_ERR_OOM : LOBPCG_ERR_CUDA, msg);
}

void release(lobpcg_ctx *h) {
    if (!h) return;
    for (void *p : h->allocs) cudaFree(p);
    h->allocs.clear();
    solver_release(h);
    mlp_release(h);
    if (h->stage_x) cudaFree(h->stage_x);
    if (h->stage_y) cudaFree(h->stage_y);
    h->stage_x = h->stage_y = nullptr;
    if (h->h_err) cudaFreeHost(h->h_err);
    h->h_err = nullptr;
}

bool is_host_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}
}  // namespace

namespace lobpcg {
cudaError_t dev_alloc(lobpcg_ctx *h, void **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(*p);
    h->device_bytes += static_cast<int64_t>(bytes);
    return cudaSuccess;
}
}  // namespace lobpcg

extern "C" {

lobpcg_status lobpcg_create(lobpcg_t *out, const lobpcg_matrix *A, const lobpcg_params *params, void *stream) {
    if (!out) return fail(nullptr, LOBPCG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!A || !params) return fail(nullptr, LOBPCG_ERR_ARG, "matrix or params is NULL");
    if (A->n < 1 || A->n >= (int64_t(1) << 28)) return fail(nullptr, LOBPCG_ERR_ARG, "n must be in [1, 2^28)");
    if (A->nnz < 0 || A->nnz >= (int64_t(1) << 40)) return fail(nullptr, LOBPCG_ERR_ARG, "nnz out of range");
    if (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
        return fail(nullptr, LOBPCG_ERR_ARG, "row_ptr/col/val is NULL");
    if (A->mem != LOBPCG_MEM_DEVICE && A->mem != LOBPCG_MEM_HOST)
        return fail(nullptr, LOBPCG_ERR_ARG, "mem must be LOBPCG_MEM_DEVICE or LOBPCG_MEM_HOST");
    const lobpcg_params &P = *params;
    if (P.k < 1 || P.k > 32) return fail(nullptr, LOBPCG_ERR_ARG, "k must be in [1, 32]");
    if (P.nev < 1 || P.nev > P.k) return fail(nullptr, LOBPCG_ERR_ARG, "nev must be in [1, k]");
    if (P.tile_format != 0 && P.tile_format != 1) return fail(nullptr, LOBPCG_ERR_ARG, "tile_format must be 0 or 1");
    if (P.precond < 0 || P.precond > 4) return fail(nullptr, LOBPCG_ERR_ARG, "precond must be 0..4");
    if (P.fom_steps < 0 || P.fom_steps > 6) return fail(nullptr, LOBPCG_ERR_ARG, "fom_steps must be 0..6");
    if (P.reserved != 0) return fail(nullptr, LOBPCG_ERR_ARG, "reserved must be 0");
    if (P.precond == 4 && P.fom_tile_ptr) {
        const int64_t *tp = P.fom_tile_ptr;
        if (P.fom_ntiles < 1 || P.fom_ntiles > A->n) return fail(nullptr, LOBPCG_ERR_ARG, "fom_ntiles must be in [1, n]");
        if (tp[0] != 0 || tp[P.fom_ntiles] != A->n)
            return fail(nullptr, LOBPCG_ERR_ARG, "fom_tile_ptr must start at 0 and end at n");
        for (int64_t t = 0; t < P.fom_ntiles; ++t)
            if (tp[t + 1] <= tp[t]) return fail(nullptr, LOBPCG_ERR_ARG, "fom_tile_ptr must be strictly increasing");
    }

    lobpcg_ctx *h = new (std::nothrow) lobpcg_ctx();
    if (!h) return fail(nullptr, LOBPCG_ERR_OOM, "host allocation failed");
    h->params = P;
    h->stream = static_cast<cudaStream_t>(stream);
    h->T.n = A->n;
    h->T.nnz = A->nnz;
    h->T.vonly = P.tile_format;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        lobpcg_status st = cuda_fail(nullptr, e, "device query");
        delete h;
        return st;
    }
    auto bail = [&](lobpcg_status st, const std::string &msg) {
        g_create_error = msg;
        release(h);
        delete h;
        return st;
    };
    e = dev_alloc(h, reinterpret_cast<void **>(&h->d_err), sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int) * 4, h->stream);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h->h_err), sizeof(int) * 4);
    if (e != cudaSuccess) return bail(LOBPCG_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(e));

    // Bring the CSR onto the device if it is on the host.
    const size_t vsz = A->val_is_fp64 ? 8 : 4;
    const int64_t *rp = A->row_ptr;
    const int32_t *cl = A->col;
    const void *vl = A->val;
    void *tmp = nullptr;
    if (A->mem == LOBPCG_MEM_HOST) {
        const size_t b_rp = sizeof(int64_t) * (A->n + 1), b_cl = sizeof(int32_t) * A->nnz, b_vl = vsz * A->nnz;
        const size_t o_cl = (b_rp + 255) & ~size_t(255), o_vl = (o_cl + b_cl + 255) & ~size_t(255);
        e = cudaMallocAsync(&tmp, o_vl + b_vl + 16, h->stream);
        if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? LOBPCG_ERR_OOM : LOBPCG_ERR_CUDA,
                                          std::string("staging: ") + cudaGetErrorString(e));
        char *base = static_cast<char *>(tmp);
        e = cudaMemcpyAsync(base, A->row_ptr, b_rp, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && b_cl) e = cudaMemcpyAsync(base + o_cl, A->col, b_cl, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && b_vl) e = cudaMemcpyAsync(base + o_vl, A->val, b_vl, cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(tmp, h->stream);
            return bail(LOBPCG_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
        }
        rp = reinterpret_cast<const int64_t *>(base);
        cl = reinterpret_cast<const int32_t *>(base + o_cl);
        vl = base + o_vl;
    }
    std::string err;
    lobpcg_status st = LOBPCG_ERR_CUDA;
    e = build_tiled(h, rp, cl, vl, A->val_is_fp64 != 0, err, st);
    if (e == cudaSuccess && st == LOBPCG_OK && (P.precond == 2 || P.precond == 3))
        e = bjacobi_setup(h, rp, cl, vl, A->val_is_fp64 != 0);   // the learned form trains on exact tile solves
    if (e == cudaSuccess && st == LOBPCG_OK && P.precond == 3) e = mlp_setup(h);
    if (e == cudaSuccess && st == LOBPCG_OK && P.precond == 4) e = fom_setup(h, rp, cl, vl, A->val_is_fp64 != 0, P.fom_tile_ptr, P.fom_ntiles);
    if (e == cudaSuccess && st == LOBPCG_OK) e = solver_setup(h);
    if (e == cudaSuccess && st == LOBPCG_OK) e = cudaStreamSynchronize(h->stream);
    if (tmp) {
        cudaFreeAsync(tmp, h->stream);
        cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess)
        return bail(e == cudaErrorMemoryAllocation ? LOBPCG_ERR_OOM : LOBPCG_ERR_CUDA,
                    std::string("tiling: ") + cudaGetErrorString(e));
    if (st != LOBPCG_OK) return bail(st, err);
    *out = h;
    return LOBPCG_OK;
}

lobpcg_status lobpcg_destroy(lobpcg_t h) {
    if (!h) return LOBPCG_OK;
    // free on the handle's device whatever device the caller has current
    int cur = -1;
    bool switched = false;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != h->device) {
        switched = cudaSetDevice(h->device) == cudaSuccess;
        if (!switched) cudaGetLastError();
    }
    if (h->stream) cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
    if (switched) cudaSetDevice(cur);
    return LOBPCG_OK;
}

lobpcg_status lobpcg_test_set_device_ordinal(lobpcg_t h, int32_t device) {
    if (!h) return LOBPCG_ERR_ARG;
    h->device = device;
    return LOBPCG_OK;
}

const char *lobpcg_last_error(lobpcg_t h) {
    return h ? h->last_error.c_str() : g_create_error.c_str();
}

lobpcg_status lobpcg_matrix_info(lobpcg_t h, lobpcg_info *info) {
    if (!h || !info) return LOBPCG_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n = h->T.n;
    info->nnz = h->T.nnz;
    info->row_blocks = h->T.R;
    info->chunks = h->T.nchunks;
    info->padded_nnz = h->T.npad;
    info->full_chunks = h->T.full_chunks;
    info->device_bytes = h->device_bytes;
    info->gershgorin = h->gershgorin;
    info->num_sms = h->num_sms;
    info->warps = h->T.warps;
    info->tile_format = h->T.vonly;
    info->stream_bytes = h->T.words * 4;
    return LOBPCG_OK;
}

lobpcg_status lobpcg_sync(lobpcg_t h) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(h->h_err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    if (*h->h_err == DEV_TIMEOUT) {
        cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
        return fail(h, LOBPCG_ERR_TIMEOUT, "a device-side wait gave up (bulk copy did not complete)");
    }
    return LOBPCG_OK;
}

lobpcg_status lobpcg_spmm_sym(lobpcg_t h, const float *X, float *Y, int32_t k) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!X || !Y) return fail(h, LOBPCG_ERR_ARG, "X or Y is NULL");
    if (k < 1 || k > 32) return fail(h, LOBPCG_ERR_ARG, "k must be in [1, 32]");
    const size_t bytes = sizeof(float) * static_cast<size_t>(h->T.n) * k;
    if (ranges_overlap(X, bytes, Y, bytes)) return fail(h, LOBPCG_ERR_ARG, "X and Y overlap");
    const bool xh = is_host_ptr(X), yh = is_host_ptr(Y);
    if (xh != yh) return fail(h, LOBPCG_ERR_ARG, "X and Y must both be host or both be device pointers");
    cudaError_t e;
    if (xh) {
        // host buffers: stage through the handle's device blocks
        if (static_cast<size_t>(k) > h->stage_k) {
            for (float **b : {&h->stage_x, &h->stage_y}) {
                if (*b) { cudaFree(*b); h->device_bytes -= sizeof(float) * h->T.n * h->stage_k; }
                *b = nullptr;
            }
            e = cudaMalloc(&h->stage_x, bytes);
            if (e == cudaSuccess) e = cudaMalloc(&h->stage_y, bytes);
            if (e != cudaSuccess) return cuda_fail(h, e, "staging");
            h->stage_k = k;
            h->device_bytes += 2 * static_cast<int64_t>(bytes);
        }
        e = cudaMemcpyAsync(h->stage_x, X, bytes, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_spmm_sym_f32(h, h->stage_x, h->stage_y, k, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(Y, h->stage_y, bytes, cudaMemcpyDeviceToHost, h->stream);
    } else {
        e = launch_spmm_sym_f32(h, X, Y, k, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "spmm_sym");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_spmm_sym_f64(lobpcg_t h, const double *X, double *Y, int32_t k) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!X || !Y) return fail(h, LOBPCG_ERR_ARG, "X or Y is NULL");
    if (k < 1 || k > 32) return fail(h, LOBPCG_ERR_ARG, "k must be in [1, 32]");
    const size_t bytes = sizeof(double) * static_cast<size_t>(h->T.n) * k;
    if (ranges_overlap(X, bytes, Y, bytes)) return fail(h, LOBPCG_ERR_ARG, "X and Y overlap");
    cudaError_t e = launch_spmm_sym_f64(h, X, Y, k, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "spmm_sym_f64");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_precond_apply(lobpcg_t h, const float *R, const double *theta, float *W, int32_t k,
                                   int32_t mode) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!R || !W || !theta) return fail(h, LOBPCG_ERR_ARG, "R, W or theta is NULL");
    if (k < 1 || k > 32) return fail(h, LOBPCG_ERR_ARG, "k must be in [1, 32]");
    if (mode < 0 || mode > 4) return fail(h, LOBPCG_ERR_ARG, "mode must be 0..4");
    if (mode == 4 && !h->fom.ready) return fail(h, LOBPCG_ERR_UNSUPPORTED, "FOM needs params.precond = 4 at create");
    if (mode == 4 && h->fom.n_large && k > h->fom.scr_k)
        return fail(h, LOBPCG_ERR_ARG, "FOM with tiles over 64 rows: k must be <= params.k");
    if (mode == 2 && !h->bj_Q) return fail(h, LOBPCG_ERR_UNSUPPORTED, "block-Jacobi needs params.precond = 2 at create");
    if (mode == 3 && !h->mlp.P) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned form needs params.precond = 3 at create");
    if (mode == 3 && !h->mlp.ready) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned preconditioner has no weights");
    if (mode == 3 && k > h->params.k) return fail(h, LOBPCG_ERR_ARG, "learned form: k must be <= params.k");
    cudaError_t e = precond_apply<float>(h, mode, k, R, theta, W, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "precond_apply");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_rayleigh_ritz(lobpcg_t h, const float *S, const float *HS, int32_t m, int32_t k, double *C,
                                   double *theta) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!S || !HS || !C || !theta) return fail(h, LOBPCG_ERR_ARG, "S, HS, C or theta is NULL");
    if (m < 1 || m > 96 || k < 1 || k > m) return fail(h, LOBPCG_ERR_ARG, "need 1 <= k <= m <= 96");
    double *G = nullptr, *O = nullptr;
    int *status = nullptr;
    cudaError_t e = cudaMallocAsync(&G, sizeof(double) * (2 * m * m + 1), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "rayleigh_ritz");
    O = G + m * m;
    status = reinterpret_cast<int *>(O + m * m);
    GemmBlocks<float> a{}, b{};
    a.p[0] = S;
    b.p[0] = HS;
    e = launch_gram<float>(h->T.n, m, 1, a, 1, b, G, h->num_sms, h->stream, h->d_err);
    if (e == cudaSuccess) e = launch_gram<float>(h->T.n, m, 1, a, 1, a, O, h->num_sms, h->stream, h->d_err);
    if (e == cudaSuccess) e = launch_rayleigh_ritz(m, k, m, G, O, m, nullptr, C, theta, status, h->stream);
    int hs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFreeAsync(G, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "rayleigh_ritz");
    if (hs == 2) return fail(h, LOBPCG_ERR_BREAKDOWN, "fewer than k directions in span(S)");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_solve(lobpcg_t h, float *X, double *evals, double *resid, lobpcg_stats *st) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!X) return fail(h, LOBPCG_ERR_ARG, "X is NULL");
    if (!h->solver) return fail(h, LOBPCG_ERR_UNSUPPORTED, "solver workspace missing");
    if (h->params.precond == 3 && !h->mlp.ready)
        return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned preconditioner has no weights (train or set them first)");
    std::string err;
    lobpcg_status s = solve(h, X, is_host_ptr(X), evals, resid, st, err);
    if (s != LOBPCG_OK) return fail(h, s, err);
    return LOBPCG_OK;
}

lobpcg_status lobpcg_davidson(lobpcg_t h, float *X, int32_t max_blocks, double *evals, double *resid,
                              lobpcg_stats *st) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!X) return fail(h, LOBPCG_ERR_ARG, "X is NULL");
    if (!h->solver) return fail(h, LOBPCG_ERR_UNSUPPORTED, "solver workspace missing");
    if (max_blocks < 2 || max_blocks > 6 || max_blocks * h->params.k > 96)
        return fail(h, LOBPCG_ERR_ARG, "max_blocks must be in [2, min(6, 96 / k)]");
    if (h->params.precond == 3 && !h->mlp.ready)
        return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned preconditioner has no weights (train or set them first)");
    std::string err;
    lobpcg_status s = davidson(h, X, is_host_ptr(X), max_blocks, evals, resid, st, err);
    if (s != LOBPCG_OK) return fail(h, s, err);
    return LOBPCG_OK;
}

lobpcg_status lobpcg_iterate(lobpcg_t h, const float *X0, int32_t steps, double *theta, lobpcg_stats *st) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (steps < 0) return fail(h, LOBPCG_ERR_ARG, "steps must be >= 0");
    if (!h->solver) return fail(h, LOBPCG_ERR_UNSUPPORTED, "solver workspace missing");
    if (h->params.precond == 3 && !h->mlp.ready)
        return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned preconditioner has no weights (train or set them first)");
    std::string err;
    lobpcg_status s = iterate(h, X0, X0 ? is_host_ptr(X0) : false, steps, theta, st, err);
    if (s != LOBPCG_OK) return fail(h, s, err);
    return LOBPCG_OK;
}

lobpcg_status lobpcg_get_x_f64(lobpcg_t h, double *X) {
    if (!h || !X) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    cudaError_t e = copy_x_f64(h, X);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_x_f64");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_mlp_set_params(lobpcg_t h, const float *params, int64_t count) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!h->mlp.P) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned form needs params.precond = 3 at create");
    if (!params || count != MLP_NPARAM_CALLER) return fail(h, LOBPCG_ERR_ARG, "params NULL or count != 49728");
    cudaError_t e = mlp_set_params(h, params, is_host_ptr(params));
    if (e != cudaSuccess) return cuda_fail(h, e, "mlp_set_params");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_mlp_get_params(lobpcg_t h, float *out, int64_t count, int32_t which) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!h->mlp.P) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned form needs params.precond = 3 at create");
    if (!out || count != MLP_NPARAM_CALLER) return fail(h, LOBPCG_ERR_ARG, "out NULL or count != 49728");
    if (which != 0 && which != 1) return fail(h, LOBPCG_ERR_ARG, "which must be 0 (weights) or 1 (gradients)");
    cudaError_t e = mlp_get_params(h, out, is_host_ptr(out), which == 1);
    if (e != cudaSuccess) return cuda_fail(h, e, "mlp_get_params");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_mlp_forward(lobpcg_t h, const float *Xin, int64_t B, float *Y) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!h->mlp.P) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned form needs params.precond = 3 at create");
    if (!Xin || !Y || B < 1 || B > (int64_t(1) << 30)) return fail(h, LOBPCG_ERR_ARG, "Xin/Y NULL or B out of range");
    cudaError_t e = mlp_forward_rows(h, Xin, B, Y);
    if (e != cudaSuccess) return cuda_fail(h, e, "mlp_forward");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_mlp_grad(lobpcg_t h, const float *Xin, const float *T, int64_t B, double *loss) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!h->mlp.P) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned form needs params.precond = 3 at create");
    if (!Xin || !T || B < 1 || B > (int64_t(1) << 30)) return fail(h, LOBPCG_ERR_ARG, "Xin/T NULL or B out of range");
    double l = 0.0;
    cudaError_t e = mlp_grad_rows(h, Xin, T, B, &l);
    if (e != cudaSuccess) return cuda_fail(h, e, "mlp_grad");
    if (loss) *loss = l;
    return LOBPCG_OK;
}

lobpcg_status lobpcg_mlp_adam(lobpcg_t h, float lr) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!h->mlp.P) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned form needs params.precond = 3 at create");
    if (!(lr > 0.f)) return fail(h, LOBPCG_ERR_ARG, "lr must be > 0");
    cudaError_t e = mlp_adam(h, lr);
    if (e != cudaSuccess) return cuda_fail(h, e, "mlp_adam");
    return LOBPCG_OK;
}

lobpcg_status lobpcg_precond_train(lobpcg_t h, int32_t harvest_iters, int64_t n_pairs, int32_t epochs,
                                   const float *X0, float lr, double *loss_hist, int64_t *pairs_used) {
    if (!h) return LOBPCG_ERR_ARG;
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!h->mlp.P) return fail(h, LOBPCG_ERR_UNSUPPORTED, "learned form needs params.precond = 3 at create");
    if (!X0) return fail(h, LOBPCG_ERR_ARG, "X0 is NULL");
    if (harvest_iters < 1 || epochs < 0 || n_pairs < MLP_BATCH || n_pairs > (int64_t(1) << 32) || !(lr > 0.f))
        return fail(h, LOBPCG_ERR_ARG, "need harvest_iters >= 1, epochs >= 0, 4096 <= n_pairs <= 2^32, lr > 0");
    cudaError_t e = mlp_alloc_pairs(h, n_pairs, harvest_iters);
    if (e != cudaSuccess) {
        mlp_release(h);
        return cuda_fail(h, e, "pair buffer");
    }
    std::string err;
    lobpcg_status s = iterate(h, X0, is_host_ptr(X0), harvest_iters, nullptr, nullptr, err, 1);
    if (s != LOBPCG_OK) {
        mlp_release(h);
        return fail(h, s, "harvest: " + err);
    }
    if (!h->mlp.ready) e = mlp_init(h, h->params.seed);
    int64_t np = 0;
    if (e == cudaSuccess) e = mlp_train(h, epochs, lr, loss_hist, &np);
    mlp_release(h);
    if (pairs_used) *pairs_used = np;
    if (e == cudaErrorInvalidValue) return fail(h, LOBPCG_ERR_ARG, "fewer than 4096 pairs harvested");
    if (e != cudaSuccess) return cuda_fail(h, e, "precond_train");
    return LOBPCG_OK;
}

}  // extern "C"
