// Rayleigh-Ritz step with a fixed, statically reserved scratch area.
//
// lobpcg_rayleigh_ritz takes its G and O workspaces from the stream-ordered
// pool on every call.  Some callers cannot let a library call allocate: a
// host loop that has reserved all device memory up front and must not grow
// the pool, a program that runs with a hard memory budget, or a loop where an
// allocator call could block on other work of the device.  This variant does
// the same computation with its workspace in a file-scope __device__ array
// whose size is fixed when the library is built, so it allocates nothing on
// the device or in pinned host memory.
//
// The array is shared by every call on a device: two calls that overlap in
// time (different streams, threads or handles on the same device) race on it
// and both results are then undefined.  After a call the array keeps that
// call's last contents; nothing reads it before the next call overwrites it.
#include <cstdint>
#include <mutex>
#include <string>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"
#include "internal.h"
#include "lobpcg.h"

namespace {

// G (m x m) | O (m x m) | status word, for m up to RR_STATIC_MAX_M.
constexpr int RR_STATIC_MAX_M = 96;
constexpr size_t RR_STATIC_DOUBLES = 2 * RR_STATIC_MAX_M * RR_STATIC_MAX_M + 2;
__device__ __align__(256) double g_rr_scratch[RR_STATIC_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_addr[MAX_DEVICES] = {};

// Device address of the scratch array on `device`, resolved once per device.
cudaError_t scratch_address(int device, double **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rr_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<double *>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace

using namespace lobpcg;

extern "C" lobpcg_status lobpcg_rayleigh_ritz_noalloc(lobpcg_t h, const float *S, const float *HS, int32_t m,
                                                      int32_t k, double *C, double *theta) {
    if (!h) return LOBPCG_ERR_ARG;
    // the address lookup below resolves the array on the current device and
    // caches it under h->device: both must be the same device
    if (!device_ok(h)) return LOBPCG_ERR_ARG;
    if (!S || !HS || !C || !theta) {
        h->last_error = "S, HS, C or theta is NULL";
        return LOBPCG_ERR_ARG;
    }
    if (m < 1 || k < 1 || k > m) {
        h->last_error = "need 1 <= k <= m";
        return LOBPCG_ERR_ARG;
    }
    if (m > RR_STATIC_MAX_M) {
        h->last_error = "rayleigh_ritz_noalloc: m = " + std::to_string(m) + " needs " +
                        std::to_string(16 * m * m + 16) + " bytes of scratch; the static area holds " +
                        std::to_string(sizeof(double) * RR_STATIC_DOUBLES) + " (m <= 96)";
        return LOBPCG_ERR_ARG;
    }
    if (h->device < 0 || h->device >= MAX_DEVICES) {
        h->last_error = "device ordinal out of range";
        return LOBPCG_ERR_ARG;
    }
    double *G = nullptr;
    cudaError_t e = scratch_address(h->device, &G);
    if (e != cudaSuccess) {
        h->last_error = std::string("rayleigh_ritz_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return LOBPCG_ERR_CUDA;
    }
    double *O = G + m * m;
    int *status = reinterpret_cast<int *>(O + m * m);
    GemmBlocks<float> a{}, b{};
    a.p[0] = S;
    b.p[0] = HS;
    // launch_gram clears its output before accumulating; the status word is
    // always written by the Rayleigh-Ritz kernel.
    e = launch_gram<float>(h->T.n, m, 1, a, 1, b, G, h->num_sms, h->stream, h->d_err);
    if (e == cudaSuccess) e = launch_gram<float>(h->T.n, m, 1, a, 1, a, O, h->num_sms, h->stream, h->d_err);
    if (e == cudaSuccess) e = launch_rayleigh_ritz(m, k, m, G, O, m, nullptr, C, theta, status, h->stream);
    int hs = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->last_error = std::string("rayleigh_ritz_noalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? LOBPCG_ERR_OOM : LOBPCG_ERR_CUDA;
    }
    if (hs == 2) {
        h->last_error = "fewer than k directions in span(S)";
        return LOBPCG_ERR_BREAKDOWN;
    }
    return LOBPCG_OK;
}
