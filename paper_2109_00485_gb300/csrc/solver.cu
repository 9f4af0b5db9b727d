// lobpcg_solve: block LOBPCG (Algorithm 1) driven from the host, every step
// on the device, one stream, one small device->host read per iteration (the
// residual norms for the convergence test).
//
// Per iteration (in the paper's order):
//   R = HX - X Theta, column norms; W = K^{-1} R               (lines 6, 10-11)
//   W <- W - X (X^T W); Cholesky-QR (SVQB on breakdown); twice  (Section 3.4)
//   HW = H W  (the one SpMM per iteration)                      (eqs. upd1-upd2)
//   G = S^T HS, O = S^T S for S = [X W P], HS = [HX HW HP]      (eq. go)
//   Rayleigh-Ritz on (G, O), P columns scaled to unit norm      (eq. rreig)
//   X = S C, HX = HS C, P = [W P] C_23, HP = [HW HP] C_23       (eqs. xupd, pupd, upd1, upd2)
// The iteration runs with float32 vectors and SpMM; when the float32
// residual stops improving above the tolerance (its rounding floor), the
// solve continues from the current X with float64 vectors, the float64
// SpMM and the same steps.  On exit HX is recomputed by an explicit SpMM and
// the test repeated.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>
#include <cuda_runtime.h>
#include "common.cuh"
#include "dense.h"
#include "internal.h"
#include "lobpcg.h"
#include "precond.h"
#include "mlp.h"

namespace lobpcg {

template <typename T>
struct Blocks {
    T *X = nullptr, *HX = nullptr, *W = nullptr, *HW = nullptr, *P = nullptr, *HP = nullptr;
};

struct SolverState {
    int k = 0;
    Blocks<float> f;
    Blocks<double> d;
    double *G = nullptr, *O = nullptr, *C = nullptr, *theta = nullptr, *norms = nullptr, *colsqP = nullptr;
    double *pscale = nullptr, *B = nullptr, *Tm = nullptr, *Cproj = nullptr;
    double *B2 = nullptr;        // 2k x k: [X^T W ; W^T W] (second orthonormalisation pass)
    double *Gx = nullptr;        // k x 2k: [X^T HX | X^T X] in float64 (mixed refinement)
    double *Rt = nullptr;        // k x 2k: R^T [W P] (mixed refinement)
    float *Cf = nullptr;         // float copies of combine coefficients
    int *status = nullptr;       // [0] RR status, [1] orthonormalisation status
    double *h_buf = nullptr;     // pinned: norms (2k), theta (k), status (2 as doubles)
    bool hasP32 = false;         // lobpcg_iterate: P holds a search direction
    bool ready32 = false;        // lobpcg_iterate: state initialised
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the SpMM of an iteration
    bool ev_pending = false;
    cudaGraphExec_t gpre = nullptr, gpost = nullptr;   // float32 iteration with P, before / after the SpMM
    int graph_pmode = -1;                              // preconditioner the graphs were captured with
    bool graph_failed = false;                         // capture failed once: launch directly
};

// Block Davidson workspace (lobpcg_davidson): up to nbmax blocks of the
// basis V and of HV, float32 and (for the float64 phase) float64.
struct DavState {
    int k = 0, nbmax = 0;
    float *V32[6] = {}, *HV32[6] = {};
    double *V64[6] = {}, *HV64[6] = {};
    double *G = nullptr;    // [V^T HV] then [V^T V], two m x m blocks (m <= 96)
    double *C = nullptr;    // m x k Ritz coefficients
    double *B = nullptr;    // m x k: V^T W
    double *Cp = nullptr;   // (k + m) x k: [I; -B]
};

// Zero the entries of G and O (both ld x ld, O right after G) in rows or
// columns c0.. that lie inside the leading m x m: the blocks a Gram of the
// basis's new blocks then fills.
__global__ void k_dav_zero(double *G, int ld, int m, int c0) {
    for (int e = threadIdx.x; e < 2 * ld * ld; e += blockDim.x) {
        const int i = (e / ld) % ld, j = e % ld;
        if (i < m && j < m && (i >= c0 || j >= c0)) G[e] = 0.0;
    }
}

// Cp = [I; -B] ((k + m) x k): W - V B = [W V] Cp
__global__ void k_proj_coef_m(int k, int m, const double *B, double *Cp) {
    for (int e = threadIdx.x; e < (k + m) * k; e += blockDim.x) {
        const int r = e / k, j = e % k;
        Cp[e] = (r < k) ? (r == j ? 1.0 : 0.0) : -B[(r - k) * k + j];
    }
}

__global__ void k_proj_coef(int k, const double *B, double *Cp) {
    // Cp = [I; -B]  (2k x k): W - X B = [W X] Cp
    for (int e = threadIdx.x; e < 2 * k * k; e += blockDim.x) {
        const int r = e / k, j = e % k;
        Cp[e] = (r < k) ? (r == j ? 1.0 : 0.0) : -B[(r - k) * k + j];
    }
}

// Omega = W^T W - S^T S with S = X^T W: B2 = [S ; W^T W] (2k x k).  The
// Gram of W - X S when X has orthonormal columns (the Pythagorean form of
// block Gram-Schmidt: Carson, Lund, Rozloznik, Thomas 2022).
__global__ void k_pip_omega(int k, const double *B2, double *Om) {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        double v = B2[(k + i) * k + j];
        for (int l = 0; l < k; ++l) v -= B2[l * k + i] * B2[l * k + j];
        Om[e] = v;
    }
}

// C = [T ; -S T] (2k x k): (W - X S) T = [W X] C.
__global__ void k_pip_coef(int k, const double *B2, const double *Tm, double *C) {
    for (int e = threadIdx.x; e < 2 * k * k; e += blockDim.x) {
        const int r = e / k, j = e % k;
        if (r < k) {
            C[e] = Tm[r * k + j];
        } else {
            double v = 0.0;
            for (int l = 0; l < k; ++l) v -= B2[(r - k) * k + l] * Tm[l * k + j];
            C[e] = v;
        }
    }
}

__global__ void k_pscale(int k, const double *colsq, double *ps) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) ps[j] = colsq[j] > 0.0 ? 1.0 / sqrt(colsq[j]) : 1.0;
}

template <typename A, typename B>
__global__ void k_convert(int64_t m, const A *in, B *out) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[e] = static_cast<B>(in[e]);
}

}  // namespace lobpcg

using namespace lobpcg;

namespace {

#define CK(x)                                        \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

template <typename T>
cudaError_t spmm_T(lobpcg_ctx *h, const T *X, T *Y, int k);
template <>
cudaError_t spmm_T<float>(lobpcg_ctx *h, const float *X, float *Y, int k) {
    return launch_spmm_sym_f32(h, X, Y, k, h->stream);
}
template <>
cudaError_t spmm_T<double>(lobpcg_ctx *h, const double *X, double *Y, int k) {
    return launch_spmm_sym_f64(h, X, Y, k, h->stream);
}

// H W with CUDA events around it on the handle's stream; the elapsed time is
// collected at the next synchronisation (read_progress).
template <typename T>
cudaError_t timed_spmm(lobpcg_ctx *h, SolverState *s, const T *W, T *HW, int k) {
    CK(cudaEventRecord(s->ev0, h->stream));
    CK(spmm_T<T>(h, W, HW, k));
    CK(cudaEventRecord(s->ev1, h->stream));
    s->ev_pending = true;
    return cudaSuccess;
}

template <typename T>
Blocks<T> &blocks_of(SolverState *s);
template <>
Blocks<float> &blocks_of<float>(SolverState *s) { return s->f; }
template <>
Blocks<double> &blocks_of<double>(SolverState *s) { return s->d; }

// LOBPCG_TRACE=1 in the environment prints one line per iteration to
// stderr: phase, iteration, worst residual of the nev columns, theta_0.
bool trace_on() {
    static const bool on = [] {
        const char *v = std::getenv("LOBPCG_TRACE");
        return v && v[0] == '1';
    }();
    return on;
}

void trace(const char *phase, int it, const std::vector<double> &rho, const std::vector<double> &theta, int nev,
           int rr_st) {
    if (!trace_on()) return;
    double worst = 0.0;
    for (int j = 0; j < nev && j < static_cast<int>(rho.size()); ++j) worst = std::max(worst, rho[j]);
    std::fprintf(stderr, "lobpcg %s it %d worst_rho %.3e theta0 %.15g rr %d\n", phase, it, worst,
                 theta.empty() ? 0.0 : theta[0], rr_st);
}

struct PhaseResult {
    int iters = 0;
    bool converged = false;
    bool stagnated = false;
    bool hasP = false;           // P holds a search direction at exit
    std::vector<double> rho;
    std::vector<double> theta;
};

// Read norms + theta + statuses (one sync); compute rho on the host.
template <typename T>
cudaError_t read_progress(lobpcg_ctx *h, SolverState *s, std::vector<double> &rho, std::vector<double> &theta,
                          int *rr_status, int *orth_status, lobpcg_stats *st) {
    const int k = s->k;
    CK(cudaMemcpyAsync(s->h_buf, s->norms, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(s->h_buf + 2 * k, s->theta, sizeof(double) * k, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(reinterpret_cast<int *>(s->h_buf + 3 * k), s->status, sizeof(int) * 2, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (s->ev_pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
        if (st) {
            st->spmm_ms += ms;
            st->spmm_calls += 1;
        }
        s->ev_pending = false;
    }
    rho.resize(k);
    theta.resize(k);
    const double G = h->gershgorin;
    for (int j = 0; j < k; ++j) {
        const double rn = std::sqrt(std::max(0.0, s->h_buf[j])), xn = std::sqrt(std::max(0.0, s->h_buf[k + j]));
        const double th = s->h_buf[2 * k + j];
        theta[j] = th;
        const double den = (h->params.resid_mode == 0) ? std::max(std::fabs(th), 1e-12 * G) * xn : G * xn;
        rho[j] = den > 0 ? rn / den : INFINITY;
    }
    const int *sts = reinterpret_cast<const int *>(s->h_buf + 3 * k);
    *rr_status = sts[0];
    *orth_status = sts[1];
    return cudaSuccess;
}

// One orthonormalisation pass: W <- W - X (X^T W), then W <- W T with the
// Cholesky-QR (or SVQB) factor T of W^T W.
template <typename T>
cudaError_t orth_pass(lobpcg_ctx *h, SolverState *s, Blocks<T> &b) {
    const int k = s->k;
    const int64_t n = h->T.n;
    GemmBlocks<T> ax{}, aw{};
    ax.p[0] = b.X;
    aw.p[0] = b.W;
    CK(launch_gram<T>(n, k, 1, ax, 1, aw, s->B, h->num_sms, h->stream, h->d_err));          // B = X^T W
    k_proj_coef<<<1, 256, 0, h->stream>>>(k, s->B, s->Cproj);
    CK(cudaGetLastError());
    GemmBlocks<T> awx{};
    awx.p[0] = b.W;
    awx.p[1] = b.X;
    CombineOut<T> o1{};
    o1.z[0] = b.W; o1.C[0] = s->Cproj; o1.c0[0] = 0; o1.norm_of = -1; o1.Cf = s->Cf; o1.err = h->d_err;
    CK(launch_combine<T>(n, k, 2, awx, 1, o1, nullptr, h->num_sms, h->stream));   // W -= X B
    CK(launch_gram<T>(n, k, 1, aw, 1, aw, s->B, h->num_sms, h->stream, h->d_err));          // B = W^T W
    CK(launch_orth_factor(k, s->B, s->Tm, s->status, h->stream));
    CombineOut<T> o2{};
    o2.z[0] = b.W; o2.C[0] = s->Tm; o2.c0[0] = 0; o2.norm_of = -1; o2.Cf = s->Cf; o2.err = h->d_err;
    return launch_combine<T>(n, k, 1, aw, 1, o2, nullptr, h->num_sms, h->stream);  // W <- W T
}

// The second orthonormalisation pass in one read of X and W and one combine
// (float32 blocks the Gram pair kernel takes): [X^T W ; W^T W] by one Gram
// launch, Omega = W^T W - S^T S (S = X^T W) is the Gram of W - X S, its
// Cholesky-QR (or SVQB) factor T, and W <- (W - X S) T = [W X] [T ; -S T].
// After the first pass W is orthogonal to X to working precision, so the
// subtraction in Omega loses nothing (the first pass, where W may lie
// nearly in span(X), forms W - X S explicitly).  Other cases: orth_pass.
template <typename T>
cudaError_t orth_pass_pip(lobpcg_ctx *h, SolverState *s, Blocks<T> &b) {
    const int k = s->k;
    const int64_t n = h->T.n;
    if constexpr (std::is_same<T, float>::value) {
        const float *blk[2] = {b.X, b.W};
        const GramPair pr[2] = {GramPair{0, 1, 0, 0, 0, 0, 0}, GramPair{1, 1, 1, 0, 0, 0, 0}};
        if (gram_pairs_fit(k, 2, blk, 2, 2 * (k / 4) * (k / 4))) {
            CK(launch_gram_pairs(n, k, 2, blk, 2, pr, s->B2, k, 2 * k, true, h->d_err, h->num_sms, h->stream));
            k_pip_omega<<<1, 256, 0, h->stream>>>(k, s->B2, s->B);
            CK(cudaGetLastError());
            CK(launch_orth_factor(k, s->B, s->Tm, s->status, h->stream));
            k_pip_coef<<<1, 256, 0, h->stream>>>(k, s->B2, s->Tm, s->Cproj);
            CK(cudaGetLastError());
            GemmBlocks<T> awx{};
            awx.p[0] = b.W;
            awx.p[1] = b.X;
            CombineOut<T> o{};
            o.z[0] = b.W; o.C[0] = s->Cproj; o.c0[0] = 0; o.norm_of = -1; o.Cf = s->Cf; o.err = h->d_err;
            return launch_combine<T>(n, k, 2, awx, 1, o, nullptr, h->num_sms, h->stream);
        }
    }
    return orth_pass<T>(h, s, b);
}

// Rayleigh-Ritz on X alone (Algorithm 1, lines 1-2): X <- X C, HX <- HX C.
template <typename T>
cudaError_t rr_on_x(lobpcg_ctx *h, SolverState *s, Blocks<T> &b) {
    const int k = s->k;
    const int64_t n = h->T.n;
    GemmBlocks<T> ax{}, ahx{};
    ax.p[0] = b.X;
    ahx.p[0] = b.HX;
    GemmBlocks<T> ab{};
    ab.p[0] = b.HX;
    ab.p[1] = b.X;
    CK(launch_gram<T>(n, k, 1, ax, 2, ab, s->G, h->num_sms, h->stream, h->d_err));   // [X^T HX | X^T X]
    CK(launch_rayleigh_ritz(k, k, k, s->G, s->G + k, 2 * k, nullptr, s->C, s->theta, s->status, h->stream));
    CombineOut<T> ox{}, oh{};
    ox.z[0] = b.X; ox.C[0] = s->C; ox.c0[0] = 0; ox.norm_of = -1; ox.Cf = s->Cf;
    oh.z[0] = b.HX; oh.C[0] = s->C; oh.c0[0] = 0; oh.norm_of = -1; oh.Cf = s->Cf;
    CK(launch_combine<T>(n, k, 1, ax, 1, ox, nullptr, h->num_sms, h->stream));
    return launch_combine<T>(n, k, 1, ahx, 1, oh, nullptr, h->num_sms, h->stream);
}

// Everything of one iteration after the residual (W = K^{-1} R in b.W):
// preconditioner, orthonormalisation, H W, Gram, Rayleigh-Ritz, update.
// Preconditioner used by a phase: the float64 refinement applies the
// diagonal form in place of the learned one.
template <typename T>
int effective_precond(const lobpcg_ctx *h) {
    const int p = h->params.precond;
    return (std::is_same<T, double>::value && p == 3) ? 1 : p;
}

// Before the SpMM: preconditioner (the diagonal one was applied inside the
// residual kernel) and the two orthonormalisation passes of W.
template <typename T>
cudaError_t body_pre(lobpcg_ctx *h, SolverState *s, Blocks<T> &b, int pmode, int harvest_iter) {
    const int k = s->k;
    const int64_t n = h->T.n;
    if (pmode == 2) {
        if constexpr (std::is_same<T, float>::value) {
            if (harvest_iter >= 0) {   // exact tile solves into HW, harvest (R, solve) pairs, then W = HW
                CK(precond_apply<T>(h, 2, k, b.W, s->theta, b.HW, h->stream));
                CK(mlp_harvest(h, k, b.W, b.HW, s->theta, harvest_iter));
                CK(cudaMemcpyAsync(b.W, b.HW, sizeof(T) * n * k, cudaMemcpyDeviceToDevice, h->stream));
            } else {
                CK(precond_apply<T>(h, 2, k, b.W, s->theta, b.W, h->stream));
            }
        } else {
            CK(precond_apply<T>(h, 2, k, b.W, s->theta, b.W, h->stream));
        }
    }
    if (pmode == 3 || pmode == 4) CK(precond_apply<T>(h, pmode, k, b.W, s->theta, b.W, h->stream));
    // orthonormalise W against X and itself
    CK(orth_pass<T>(h, s, b));
    CK(orth_pass_pip<T>(h, s, b));
    return cudaSuccess;
}

// LOBPCG_GRAM_POST=full computes every block of the post-SpMM Gram
// (for comparison with the lower-block form).
bool gram_post_forced_full() {
    static const bool on = [] {
        const char *v = std::getenv("LOBPCG_GRAM_POST");
        return v && std::strcmp(v, "full") == 0;
    }();
    return on;
}

// [S^T HS | S^T S] (m x 2m, FP64, m = na k) for S = [X W P] (na = 3) or
// [X W] (na = 2), HS = [HX HW HP].  float32 blocks go to the CUDA-core pair
// kernel with the diagonal and lower blocks only: the Rayleigh-Ritz step
// averages G[i][j] and G[j][i], so each upper block is written as the
// transpose of its lower partner.  Of the two products of an off-diagonal G block the
// one with HW, this iteration's explicit SpMM, is taken (X^T HW, P^T HW);
// the (X, P) block is P^T HX.  Other shapes: all blocks by launch_gram.
template <typename T>
cudaError_t gram_post(lobpcg_ctx *h, SolverState *s, Blocks<T> &b, int na) {
    const int k = s->k;
    const int64_t n = h->T.n;
    const int m = na * k;
    if constexpr (std::is_same<T, float>::value) {
        const float *blk[6] = {b.X, b.W, b.P, b.HX, b.HW, b.HP};
        if (na == 2) {
            blk[2] = b.HX;
            blk[3] = b.HW;
        }
        const int X = 0, W = 1, P = 2, HX = na, HW = na + 1;
        GramPair pr[12];
        int np = 0;
        // diagonal blocks in full: a warp then holds exactly one pair (k = 16)
        // and reads one 128-byte line per load (packed lower halves put two
        // pairs in many warps and doubled the shared-memory wavefronts)
        for (int i = 0; i < na; ++i) {
            pr[np++] = GramPair{i, na + i, i, i, 0, 0, 0};                    // S_i^T HS_i
            pr[np++] = GramPair{i, i, i, na + i, 0, 0, 0};                    // S_i^T S_i
        }
        pr[np++] = GramPair{X, HW, 0, 1, GRAM_MIRROR, 1, 0};                 // X^T HW
        pr[np++] = GramPair{W, X, 1, na + 0, GRAM_MIRROR, 0, na + 1};        // W^T X
        if (na == 3) {
            pr[np++] = GramPair{P, HW, 2, 1, GRAM_MIRROR, 1, 2};             // P^T HW
            pr[np++] = GramPair{P, HX, 2, 0, GRAM_MIRROR, 0, 2};             // P^T HX
            pr[np++] = GramPair{P, X, 2, na + 0, GRAM_MIRROR, 0, na + 2};    // P^T X
            pr[np++] = GramPair{P, W, 2, na + 1, GRAM_MIRROR, 1, na + 2};    // P^T W
        }
        const int T4 = k / 4;
        const int units = np * T4 * T4;
        if (!gram_post_forced_full() && gram_pairs_fit(k, 2 * na, blk, np, units))
            return launch_gram_pairs(n, k, 2 * na, blk, np, pr, s->G, 2 * m, m, true, h->d_err, h->num_sms,
                                     h->stream);
    }
    GemmBlocks<T> aS{}, aB{};
    aS.p[0] = b.X; aS.p[1] = b.W; aS.p[2] = b.P;
    const T *hs[3] = {b.HX, b.HW, b.HP};
    for (int q = 0; q < na; ++q) {
        aB.p[q] = hs[q];
        aB.p[na + q] = aS.p[q];
    }
    return launch_gram<T>(n, k, na, aS, 2 * na, aB, s->G, h->num_sms, h->stream, h->d_err);
}

// LOBPCG_FUSED_UPDATE=0 keeps the update on the combine kernels and the
// residual on its own kernel (for comparison).
bool fused_update_on() {
    static const bool on = [] {
        const char *v = std::getenv("LOBPCG_FUSED_UPDATE");
        return !(v && v[0] == '0');
    }();
    return on;
}

// Whether body_post forms the next iteration's residual (and W) itself: the
// fused update kernel (update.cu) takes float32 blocks with k = 8, 16, 20.
template <typename T>
bool post_fused(const lobpcg_ctx *h, const SolverState *s, const Blocks<T> &b, bool hasP) {
    if constexpr (std::is_same<T, float>::value) {
        if (!fused_update_on()) return false;
        const int na = hasP ? 3 : 2;
        const float *S[3] = {b.X, b.W, b.P}, *HS[3] = {b.HX, b.HW, b.HP};
        const float *blk[6];
        for (int q = 0; q < na; ++q) {
            blk[q] = S[q];
            blk[na + q] = HS[q];
        }
        return update_post_ok(s->k, na, blk);
    } else {
        (void)h; (void)s; (void)b; (void)hasP;
        return false;
    }
}

// After the SpMM: Gram matrices of S = [X W P], HS = [HX HW HP],
// Rayleigh-Ritz and the updates X = S C, P = [W P] C_23 (with ||p_j||^2),
// HX = HS C, HP = [HW HP] C_23.
template <typename T>
cudaError_t body_post(lobpcg_ctx *h, SolverState *s, Blocks<T> &b, bool hasP, int pmode) {
    const int k = s->k;
    const int64_t n = h->T.n;
    const int na = hasP ? 3 : 2;
    const int m = na * k;
    GemmBlocks<T> aS{}, aHS{};
    aS.p[0] = b.X; aS.p[1] = b.W; aS.p[2] = b.P;
    aHS.p[0] = b.HX; aHS.p[1] = b.HW; aHS.p[2] = b.HP;
    CK(gram_post<T>(h, s, b, na));   // [S^T HS | S^T S]
    if (hasP) {
        k_pscale<<<1, 64, 0, h->stream>>>(k, s->colsqP, s->pscale);
        CK(cudaGetLastError());
    }
    CK(launch_rayleigh_ritz(m, k, 2 * k, s->G, s->G + m, 2 * m, hasP ? s->pscale : nullptr, s->C, s->theta,
                            s->status, h->stream));
    if constexpr (std::is_same<T, float>::value) {
        if (post_fused<T>(h, s, b, hasP)) {
            // updates and the next residual W = K^{-1} R (diagonal K) in one pass
            const float *S[3] = {b.X, b.W, b.P}, *HS[3] = {b.HX, b.HW, b.HP};
            return launch_update_post(n, k, na, S, HS, b.X, b.P, b.HX, b.HP, b.W, s->C, s->theta, h->T.diag,
                                      pmode == 1 ? 1 : 0, s->norms, s->colsqP, h->d_err, h->num_sms, h->stream);
        }
    }
    CombineOut<T> ox{}, oh{};
    ox.Cf = s->Cf;
    oh.Cf = s->Cf;
    ox.z[0] = b.X; ox.C[0] = s->C; ox.c0[0] = 0;
    ox.z[1] = b.P; ox.C[1] = s->C + static_cast<int64_t>(k) * k; ox.c0[1] = k; ox.norm_of = 1;
    oh.z[0] = b.HX; oh.C[0] = s->C; oh.c0[0] = 0;
    oh.z[1] = b.HP; oh.C[1] = s->C + static_cast<int64_t>(k) * k; oh.c0[1] = k; oh.norm_of = -1;
    CK(launch_combine<T>(n, k, na, aS, 2, ox, s->colsqP, h->num_sms, h->stream));
    CK(launch_combine<T>(n, k, na, aHS, 2, oh, nullptr, h->num_sms, h->stream));
    return cudaSuccess;
}

// LOBPCG_GRAPH=0 in the environment turns the graph replay off.
bool graphs_on() {
    static const bool on = [] {
        const char *v = std::getenv("LOBPCG_GRAPH");
        return !(v && v[0] == '0');
    }();
    return on;
}

// Capture fn's launches on the handle's stream into an executable graph.
// Returns false (and leaves the stream out of capture) if anything fails.
template <typename F>
bool capture(lobpcg_ctx *h, cudaGraphExec_t *out, F fn) {
    if (h->stream == nullptr || h->stream == cudaStreamLegacy) return false;   // no capture on the legacy stream
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();   // leave no error behind for the direct launches that follow
        return false;
    }
    const cudaError_t e = fn();
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    bool ok = e == cudaSuccess && e2 == cudaSuccess && g;
    if (ok) ok = cudaGraphInstantiate(out, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return ok;
}

// One iteration after the residual.  The float32 iteration with P (every
// iteration but the first of a run) replays two CUDA graphs captured on
// first use -- the launches before the SpMM and those after it -- with the
// timed SpMM launched between them; the first iteration, float64, the
// learned form, harvesting and handles on the legacy default stream (which
// cannot be captured) launch directly.
template <typename T>
cudaError_t iteration_body(lobpcg_ctx *h, SolverState *s, Blocks<T> &b, bool hasP, int pmode, int harvest_iter = -1) {
    const int k = s->k;
    if constexpr (std::is_same<T, float>::value) {
        if (hasP && harvest_iter < 0 && pmode != 3 && graphs_on() && !s->graph_failed) {
            if (s->graph_pmode != pmode) {
                if (s->gpre) cudaGraphExecDestroy(s->gpre);
                if (s->gpost) cudaGraphExecDestroy(s->gpost);
                s->gpre = s->gpost = nullptr;
                const bool ok = capture(h, &s->gpre, [&] { return body_pre<T>(h, s, b, pmode, -1); }) &&
                                capture(h, &s->gpost, [&] { return body_post<T>(h, s, b, true, pmode); });
                if (!ok) {
                    s->graph_failed = true;
                    if (s->gpre) cudaGraphExecDestroy(s->gpre);
                    if (s->gpost) cudaGraphExecDestroy(s->gpost);
                    s->gpre = s->gpost = nullptr;
                } else {
                    s->graph_pmode = pmode;
                }
            }
            if (!s->graph_failed) {
                CK(cudaGraphLaunch(s->gpre, h->stream));
                CK(timed_spmm<T>(h, s, b.W, b.HW, k));   // the one SpMM per iteration
                return cudaGraphLaunch(s->gpost, h->stream);
            }
        }
    }
    CK(body_pre<T>(h, s, b, pmode, harvest_iter));
    CK(timed_spmm<T>(h, s, b.W, b.HW, k));   // the one SpMM per iteration
    return body_post<T>(h, s, b, hasP, pmode);
}

template <typename T>
cudaError_t run_phase(lobpcg_ctx *h, SolverState *s, int max_iters, bool stop_on_stagnation, PhaseResult &res,
                      lobpcg_stats *st, lobpcg_status &status) {
    const int k = s->k, nev = h->params.nev;
    const int64_t n = h->T.n;
    const double tol = h->params.tol;
    Blocks<T> &b = blocks_of<T>(s);
    const int pmode = effective_precond<T>(h);
    // snapshot of the best X of a float32 phase that a refinement may
    // continue (the float64 W block is free during that phase)
    T *snap = (std::is_same<T, float>::value && s->d.W) ? reinterpret_cast<T *>(s->d.W) : nullptr;
    status = LOBPCG_OK;

    CK(spmm_T<T>(h, b.X, b.HX, k));
    CK(rr_on_x<T>(h, s, b));
    bool hasP = false;
    double best = INFINITY, floor_best = INFINITY;
    int since_best = 0, since_floor = 0;
    int restarts = 0;
    std::vector<double> rho, theta;
    bool resid_ready = false;   // the last iteration's fused update formed R (and W)
    while (true) {
        // R = HX - X Theta and norms; W = K^{-1} R
        if (!resid_ready)
            CK(launch_resid<T>(n, k, b.X, b.HX, s->theta, h->T.diag, b.W, pmode == 1 ? 1 : 0, s->norms,
                               h->num_sms, h->stream));
        resid_ready = false;
        int rr_st = 0, orth_st = 0;
        CK(read_progress<T>(h, s, rho, theta, &rr_st, &orth_st, st));
        trace(std::is_same<T, float>::value ? "fp32" : "fp64", res.iters, rho, theta, nev, rr_st);
        if (rr_st == 2) {
            status = LOBPCG_ERR_BREAKDOWN;
            break;
        }
        if (rr_st == 1 && st) st->p_dropped++;
        if (orth_st == 1 && st) st->svqb_used++;
        bool finite = true;
        for (int j = 0; j < k; ++j) finite = finite && std::isfinite(rho[j]) && std::isfinite(theta[j]);
        if (!finite) {
            status = LOBPCG_ERR_NONFINITE;
            break;
        }
        double worst = 0.0;
        for (int j = 0; j < nev; ++j) worst = std::max(worst, rho[j]);
        if (worst <= tol) {
            // explicit re-check: HX from a fresh SpMM (into HW as scratch)
            CK(spmm_T<T>(h, b.X, b.HW, k));
            CK(launch_resid<T>(n, k, b.X, b.HW, s->theta, h->T.diag, b.W, pmode == 1 ? 1 : 0, s->norms,
                               h->num_sms, h->stream));
            CK(read_progress<T>(h, s, rho, theta, &rr_st, &orth_st, st));
            double worst_e = 0.0;
            for (int j = 0; j < nev; ++j) worst_e = std::max(worst_e, rho[j]);
            if (worst_e <= tol || restarts >= 5) {
                res.converged = worst_e <= tol;
                break;
            }
            ++restarts;
            if (st) st->explicit_restarts++;
            CK(cudaMemcpyAsync(b.HX, b.HW, sizeof(T) * n * k, cudaMemcpyDeviceToDevice, h->stream));
            continue;
        }
        // Stagnation (15 iterations without a 0.7x improvement, with a best
        // below 1e-2: far above the float32 rounding floor more precision
        // does not help a stalled run), growth
        // (4x above a best below 1e-3: at the float32 rounding floor the
        // HX/HP recurrences lose consistency and the residual grows
        // geometrically) or a floor (below 1e-2, no new minimum by 5 % in 3
        // iterations: the residual only fluctuates around the rounding
        // level, while a slow but converging run still gains 5 % an
        // iteration) ends a phase that can be continued in higher
        // precision; it then hands over the X of the lowest residual seen.
        if (worst < 0.95 * floor_best) {
            floor_best = worst;
            since_floor = 0;
            if (stop_on_stagnation && snap)
                CK(cudaMemcpyAsync(snap, b.X, sizeof(T) * n * k, cudaMemcpyDeviceToDevice, h->stream));
        } else {
            ++since_floor;
        }
        if (worst < 0.7 * best) {
            best = worst;
            since_best = 0;
        } else if (stop_on_stagnation && ((++since_best >= 15 && best < 1e-2) || (best < 1e-3 && worst > 4.0 * best) ||
                                          (floor_best < 1e-2 && since_floor >= 3))) {
            res.stagnated = true;
            if (snap) CK(cudaMemcpyAsync(b.X, snap, sizeof(T) * n * k, cudaMemcpyDeviceToDevice, h->stream));
            break;
        }
        if (res.iters >= max_iters) break;
        ++res.iters;
        CK(iteration_body<T>(h, s, b, hasP, pmode));
        resid_ready = post_fused<T>(h, s, b, hasP);
        hasP = true;
    }
    res.rho = rho;
    res.theta = theta;
    res.hasP = hasP;
    return cudaSuccess;
}

// The blocks of G = [S^T HS | S^T S] (m x 2m) that couple X with the
// corrections are taken from float64 or residual-based values:
//   X^T H X, X^T X                  float64 products (Gx, k x 2k)
//   X^T H Z = Theta X^T Z + R^T Z   for Z = W, P  (H X = X Theta + R exactly,
//                                   by the definition of R), so that the
//                                   coupling is as accurate as R itself;
//                                   X^T Z is the float32 Gram's S^T S block.
// Both triangles are written (the Rayleigh-Ritz step reads full blocks).
__global__ void k_patch_mixed(int k, int m, const double *theta, const double *Gx, const double *Rt, double *G) {
    const int ld = 2 * m, nz = m - k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int i = e / k, j = e % k;
        G[i * ld + j] = Gx[i * 2 * k + j];
        G[i * ld + m + j] = Gx[i * 2 * k + k + j];
    }
    for (int e = threadIdx.x; e < k * nz; e += blockDim.x) {
        const int i = e / nz, c = k + e % nz;
        const double v = theta[i] * G[i * ld + m + c] + Rt[i * nz + (c - k)];   // Rt: k x (m - k)
        G[i * ld + c] = v;
        G[c * ld + i] = v;
    }
}

// Mixed-precision refinement (after the float32 phase has reached its
// rounding floor).  X and HX are float64; W, P, HW, HP and the one SpMM per
// iteration stay float32.  HX starts from an explicit float64 SpMM and is then
// updated by the recurrence HX <- HX C_x + [HW HP] C_23, whose float32 part
// only carries the (shrinking) correction, so its rounding error shrinks with
// the step.  The X-X blocks of the Gram matrices (the Ritz values) are formed
// from the float64 X and HX; the other blocks from float32 copies.
cudaError_t run_phase_mixed(lobpcg_ctx *h, SolverState *s, int max_iters, PhaseResult &res, lobpcg_stats *st,
                            lobpcg_status &status) {
    const int k = s->k, nev = h->params.nev;
    const int64_t n = h->T.n;
    const double tol = h->params.tol;
    Blocks<float> &f = s->f;
    Blocks<double> &d = s->d;
    const int pmode = h->params.precond;
    const int nb = std::max(1, std::min<int>(h->num_sms * 8, static_cast<int>((n * k + 255) / 256)));
    float *R32 = reinterpret_cast<float *>(d.W);   // float32 residual (d.W is free until the explicit check)
    bool hasP = false;   // the float32 phase's P and HP are not carried over: HP has drifted from H P
    status = LOBPCG_OK;
    auto refresh32 = [&]() -> cudaError_t {   // float32 copies of X and HX
        k_convert<double, float><<<nb, 256, 0, h->stream>>>(n * k, d.X, f.X);
        k_convert<double, float><<<nb, 256, 0, h->stream>>>(n * k, d.HX, f.HX);
        return cudaGetLastError();
    };
    k_convert<float, double><<<nb, 256, 0, h->stream>>>(n * k, f.X, d.X);
    CK(cudaGetLastError());
    CK(spmm_T<double>(h, d.X, d.HX, k));
    CK(rr_on_x<double>(h, s, d));
    CK(refresh32());
    std::vector<double> rho, theta;
    int restarts = 0, refreshes = 0, since_best = 0;
    double best = INFINITY;
    bool resid_ready = false;   // the previous iteration's update formed this residual
    while (true) {
        if (!resid_ready)
            CK(launch_resid_mixed(n, k, d.X, d.HX, s->theta, h->T.diag, f.W, R32, pmode == 1 ? 1 : 0, s->norms,
                                  h->num_sms, h->stream));
        resid_ready = false;
        int rr_st = 0, orth_st = 0;
        CK(read_progress<float>(h, s, rho, theta, &rr_st, &orth_st, st));
        trace("mixed", res.iters, rho, theta, nev, rr_st);
        if (rr_st == 2) {
            status = LOBPCG_ERR_BREAKDOWN;
            break;
        }
        if (rr_st == 1 && st) st->p_dropped++;
        if (orth_st == 1 && st) st->svqb_used++;
        bool finite = true;
        for (int j = 0; j < k; ++j) finite = finite && std::isfinite(rho[j]) && std::isfinite(theta[j]);
        if (!finite) {
            status = LOBPCG_ERR_NONFINITE;
            break;
        }
        double worst = 0.0;
        for (int j = 0; j < nev; ++j) worst = std::max(worst, rho[j]);
        if (worst <= tol) {
            // explicit float64 re-check: HX from a fresh SpMM (into d.HW)
            CK(spmm_T<double>(h, d.X, d.HW, k));
            CK(launch_resid<double>(n, k, d.X, d.HW, s->theta, h->T.diag, d.W, 0, s->norms, h->num_sms, h->stream));
            CK(read_progress<float>(h, s, rho, theta, &rr_st, &orth_st, st));
            double worst_e = 0.0;
            for (int j = 0; j < nev; ++j) worst_e = std::max(worst_e, rho[j]);
            trace("check", res.iters, rho, theta, nev, 0);
            if (worst_e <= tol || restarts >= 5) {
                res.converged = worst_e <= tol;
                break;
            }
            ++restarts;
            if (st) st->explicit_restarts++;
            CK(cudaMemcpyAsync(d.HX, d.HW, sizeof(double) * n * k, cudaMemcpyDeviceToDevice, h->stream));
            CK(refresh32());
            continue;
        }
        // Growth (4x above the best) or no 0.7x improvement in 50 iterations:
        // the recurrence HX <- HX C_x + HP may have accumulated float32 error
        // from many small steps; restart from an explicit float64 HX without
        // P (at most 20 times).
        if (worst < 0.7 * best) {
            best = worst;
            since_best = 0;
        } else if ((++since_best >= 50 || worst > 4.0 * best) && refreshes < 20) {
            ++refreshes;
            if (st) st->explicit_restarts++;
            CK(spmm_T<double>(h, d.X, d.HX, k));
            CK(rr_on_x<double>(h, s, d));
            CK(refresh32());
            hasP = false;
            best = INFINITY;
            since_best = 0;
            continue;
        }
        if (res.iters >= max_iters) break;
        ++res.iters;
        // preconditioner (the diagonal one was applied in the residual)
        if (pmode >= 2) CK(precond_apply<float>(h, pmode, k, f.W, s->theta, f.W, h->stream));
        CK(orth_pass<float>(h, s, f));
        CK(orth_pass_pip<float>(h, s, f));
        CK(timed_spmm<float>(h, s, f.W, f.HW, k));
        const int na = hasP ? 3 : 2;
        const int m = na * k;
        CK(gram_post<float>(h, s, f, na));   // [S^T HS | S^T S]; the X blocks are patched below
        if (mixed_df_ok(k)) {
            CK(launch_gram_x_df(n, k, d.X, d.HX, s->Gx, h->num_sms, h->stream));   // [X^T HX | X^T X]
        } else {
            GemmBlocks<double> ax{}, axx{};
            ax.p[0] = d.X;
            axx.p[0] = d.HX;
            axx.p[1] = d.X;
            CK(launch_gram<double>(n, k, 1, ax, 2, axx, s->Gx, h->num_sms, h->stream, h->d_err));
        }
        GemmBlocks<float> ar{}, awp{};
        ar.p[0] = R32;
        awp.p[0] = f.W;
        awp.p[1] = f.P;
        CK(launch_gram<float>(n, k, 1, ar, na - 1, awp, s->Rt, h->num_sms, h->stream, h->d_err));
        k_patch_mixed<<<1, 256, 0, h->stream>>>(k, m, s->theta, s->Gx, s->Rt, s->G);
        CK(cudaGetLastError());
        if (hasP) {
            k_pscale<<<1, 64, 0, h->stream>>>(k, s->colsqP, s->pscale);
            CK(cudaGetLastError());
        }
        CK(launch_rayleigh_ritz(m, k, 2 * k, s->G, s->G + m, 2 * m, hasP ? s->pscale : nullptr, s->C, s->theta,
                                s->status, h->stream));
        // P = [W P] C_23 (with ||p_j||^2), HP = [HW HP] C_23, then
        // X = X C_x + P, HX = HX C_x + HP in float64
        const double *C23 = s->C + static_cast<int64_t>(k) * k;
        if (mixed_df_ok(k)) {
            // the directions, both updates and the next iteration's residual
            // in one pass
            CK(launch_xupdate2_df(n, k, d.X, d.HX, s->C, f.P, f.HP, f.X, f.HX, s->theta, h->T.diag, f.W, R32,
                                  pmode == 1 ? 1 : 0, s->norms, h->num_sms, h->stream, f.W, f.HW, C23, na - 1,
                                  s->colsqP));
            resid_ready = true;
        } else {
            GemmBlocks<float> aWP{}, aHWP{};
            aWP.p[0] = f.W; aWP.p[1] = f.P;
            aHWP.p[0] = f.HW; aHWP.p[1] = f.HP;
            CombineOut<float> op{}, ohp{};
            op.Cf = s->Cf;
            ohp.Cf = s->Cf;
            op.z[0] = f.P; op.C[0] = C23; op.c0[0] = 0; op.norm_of = 0;
            ohp.z[0] = f.HP; ohp.C[0] = C23; ohp.c0[0] = 0; ohp.norm_of = -1;
            CK(launch_combine<float>(n, k, na - 1, aWP, 1, op, s->colsqP, h->num_sms, h->stream));
            CK(launch_combine<float>(n, k, na - 1, aHWP, 1, ohp, nullptr, h->num_sms, h->stream));
            CK(launch_xupdate(n, k, d.X, s->C, f.P, f.X, h->num_sms, h->stream));
            CK(launch_xupdate(n, k, d.HX, s->C, f.HP, f.HX, h->num_sms, h->stream));
        }
        hasP = true;
    }
    res.rho = rho;
    res.theta = theta;
    res.hasP = hasP;
    return cudaSuccess;
}

template <typename T>
cudaError_t alloc_blocks(lobpcg_ctx *h, Blocks<T> &b, int k) {
    const size_t bytes = sizeof(T) * static_cast<size_t>(h->T.n) * k;
    for (T **p : {&b.X, &b.HX, &b.W, &b.HW, &b.P, &b.HP}) CK(dev_alloc(h, reinterpret_cast<void **>(p), bytes));
    return cudaSuccess;
}

}  // namespace

namespace lobpcg {

cudaError_t solver_setup(lobpcg_ctx *h) {
    const int k = h->params.k;
    SolverState *s = new SolverState();
    h->solver = s;
    s->k = k;
    CK(alloc_blocks<float>(h, s->f, k));
    if (h->params.polish_fp64) CK(alloc_blocks<double>(h, s->d, k));
    const int m = 3 * k;
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->G), sizeof(double) * 2 * m * m));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->O), sizeof(double) * m * m));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->C), sizeof(double) * m * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->theta), sizeof(double) * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->norms), sizeof(double) * 2 * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->colsqP), sizeof(double) * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->pscale), sizeof(double) * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->B), sizeof(double) * k * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->Tm), sizeof(double) * k * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->Cproj), sizeof(double) * 2 * k * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->B2), sizeof(double) * 2 * k * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->Gx), sizeof(double) * 2 * k * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->Rt), sizeof(double) * 2 * k * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->status), sizeof(int) * 4));
    CK(dev_alloc(h, reinterpret_cast<void **>(&s->Cf), sizeof(float) * 2 * 96 * 32));
    CK(cudaMemsetAsync(s->status, 0, sizeof(int) * 4, h->stream));
    CK(cudaMallocHost(reinterpret_cast<void **>(&s->h_buf), sizeof(double) * (4 * k + 4)));
    CK(cudaEventCreate(&s->ev0));
    CK(cudaEventCreate(&s->ev1));
    return cudaSuccess;
}

void solver_release(lobpcg_ctx *h) {
    delete h->dav;
    h->dav = nullptr;
    if (!h->solver) return;
    if (h->solver->h_buf) cudaFreeHost(h->solver->h_buf);
    if (h->solver->ev0) cudaEventDestroy(h->solver->ev0);
    if (h->solver->gpre) cudaGraphExecDestroy(h->solver->gpre);
    if (h->solver->gpost) cudaGraphExecDestroy(h->solver->gpost);
    if (h->solver->ev1) cudaEventDestroy(h->solver->ev1);
    delete h->solver;
    h->solver = nullptr;
}

// The full solve (see the file comment).  X: n x k float32 (device or host),
// in: initial guess, out: Ritz vectors.
lobpcg_status solve(lobpcg_ctx *h, float *Xio, bool x_on_host, double *evals, double *resid, lobpcg_stats *st,
                    std::string &err) {
    SolverState *s = h->solver;
    const int k = s->k, nev = h->params.nev;
    const int64_t n = h->T.n;
    const size_t bytes32 = sizeof(float) * n * k;
    auto t0 = std::chrono::steady_clock::now();
    if (st) std::memset(st, 0, sizeof(*st));
    cudaError_t e = cudaMemcpyAsync(s->f.X, Xio, bytes32, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e != cudaSuccess) { err = std::string("solve: ") + cudaGetErrorString(e); return LOBPCG_ERR_CUDA; }
    PhaseResult r32;
    lobpcg_status status = LOBPCG_OK;
    e = run_phase<float>(h, s, h->params.maxiter, h->params.polish_fp64 != 0, r32, st, status);
    if (e != cudaSuccess) { err = std::string("solve (fp32): ") + cudaGetErrorString(e); return LOBPCG_ERR_CUDA; }
    PhaseResult final = r32;
    int iters64 = 0;
    bool used64 = false;
    if (status == LOBPCG_OK && !r32.converged && h->params.polish_fp64 && s->d.X) {
        // continue from the current X with float64 X and HX (mixed refinement)
        PhaseResult r64;
        e = run_phase_mixed(h, s, std::max(0, h->params.maxiter - r32.iters), r64, st, status);
        if (e != cudaSuccess) { err = std::string("solve (fp64): ") + cudaGetErrorString(e); return LOBPCG_ERR_CUDA; }
        iters64 = r64.iters;
        final = r64;
        used64 = true;   // f.X holds float32(X) of the refinement
    }
    if (!used64 && s->d.X) {   // keep a float64 copy for lobpcg_get_x_f64
        const int64_t mm = n * k;
        k_convert<float, double><<<std::max(1, std::min<int>(h->num_sms * 8, static_cast<int>((mm + 255) / 256))), 256,
                                   0, h->stream>>>(mm, s->f.X, s->d.X);
    }
    e = cudaMemcpyAsync(Xio, s->f.X, bytes32, x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { err = std::string("solve: ") + cudaGetErrorString(e); return LOBPCG_ERR_CUDA; }
    for (int j = 0; j < nev && j < static_cast<int>(final.theta.size()); ++j) {
        if (evals) evals[j] = final.theta[j];
        if (resid) resid[j] = final.rho[j];
    }
    if (st) {
        st->iters = r32.iters + iters64;
        st->iters_fp64 = iters64;
        st->used_fp64 = used64 ? 1 : 0;
        st->converged = final.converged ? 1 : 0;
        st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status != LOBPCG_OK) {
        err = status == LOBPCG_ERR_BREAKDOWN ? "Rayleigh-Ritz breakdown" : "non-finite residual";
        return status;
    }
    if (!final.converged) {
        err = "maxiter reached before the residual tolerance";
        return LOBPCG_ERR_NOT_CONVERGED;
    }
    return LOBPCG_OK;
}

// A fixed number of float32 iterations with no exit test (the residual
// norms are still formed and read each iteration, as in the solve).  X0 (n x k,
// device or host) starts a new run; NULL continues the previous one.
lobpcg_status iterate(lobpcg_ctx *h, const float *X0, bool x_on_host, int steps, double *theta_out,
                      lobpcg_stats *st, std::string &err, int harvest) {
    SolverState *s = h->solver;
    const int k = s->k;
    const int64_t n = h->T.n;
    Blocks<float> &b = s->f;
    auto fail = [&](cudaError_t e) {
        err = std::string("iterate: ") + cudaGetErrorString(e);
        return LOBPCG_ERR_CUDA;
    };
    auto t0 = std::chrono::steady_clock::now();
    if (st) std::memset(st, 0, sizeof(*st));
    cudaError_t e = cudaSuccess;
    if (X0) {
        e = cudaMemcpyAsync(b.X, X0, sizeof(float) * n * k, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                            h->stream);
        if (e == cudaSuccess) e = spmm_T<float>(h, b.X, b.HX, k);
        if (e == cudaSuccess) e = rr_on_x<float>(h, s, b);
        if (e != cudaSuccess) return fail(e);
        s->hasP32 = false;
        s->ready32 = true;
    }
    if (!s->ready32) {
        err = "iterate: no state to continue (pass X0)";
        return LOBPCG_ERR_ARG;
    }
    std::vector<double> rho, theta;
    const int pmode = harvest ? 2 : h->params.precond;   // harvesting runs the exact tile solves
    bool resid_ready = false;   // the last iteration's fused update formed R (and W)
    for (int it = 0; it < steps; ++it) {
        if (!resid_ready)
            e = launch_resid<float>(n, k, b.X, b.HX, s->theta, h->T.diag, b.W, pmode == 1 ? 1 : 0, s->norms,
                                    h->num_sms, h->stream);
        int rr_st = 0, orth_st = 0;
        if (e == cudaSuccess) e = read_progress<float>(h, s, rho, theta, &rr_st, &orth_st, st);
        if (e == cudaSuccess) e = iteration_body<float>(h, s, b, s->hasP32, pmode, harvest ? it : -1);
        if (e != cudaSuccess) return fail(e);
        resid_ready = post_fused<float>(h, s, b, s->hasP32);
        s->hasP32 = true;
        if (st) st->iters++;
    }
    std::vector<double> r2, t2;
    int a1, a2;
    e = read_progress<float>(h, s, r2, t2, &a1, &a2, st);   // collects the last SpMM time
    if (e != cudaSuccess) return fail(e);
    if (theta_out)
        for (int j = 0; j < k && j < static_cast<int>(t2.size()); ++j) theta_out[j] = t2[j];
    if (st) st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return LOBPCG_OK;
}

cudaError_t copy_x_f64(lobpcg_ctx *h, double *out) {
    SolverState *s = h->solver;
    if (!s || !s->d.X) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(out, s->d.X, sizeof(double) * h->T.n * s->k, cudaMemcpyDefault, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e;
}

}  // namespace lobpcg

// ---------------------------------------------------------------- block Davidson
// The same SpMM, preconditioners, Gram, combine and Rayleigh-Ritz kernels
// inside block (generalised) Davidson: a growing orthonormal basis V of at
// most nbmax blocks, the k leftmost Ritz pairs of (V^T H V, V^T V) each
// iteration, the preconditioned residuals orthonormalised against V and
// appended (one SpMM per iteration), and a restart to the Ritz vectors when
// V is full.  float32 first; when its residual stalls above tol and
// params.polish_fp64 is set, the same iteration continues in float64.

namespace {

// W <- W - V (V^T W), then Cholesky-QR (SVQB on failure); twice.
template <typename T>
cudaError_t dav_orth(lobpcg_ctx *h, SolverState *s, DavState *D, T *const *V, int nb, T *W) {
    const int k = s->k, m = nb * k;
    const int64_t n = h->T.n;
    GemmBlocks<T> av{}, aw{}, awv{};
    for (int q = 0; q < nb; ++q) {
        av.p[q] = V[q];
        awv.p[q + 1] = V[q];
    }
    aw.p[0] = W;
    awv.p[0] = W;
    for (int pass = 0; pass < 2; ++pass) {
        if (nb > 0) {
            CK(launch_gram<T>(n, k, nb, av, 1, aw, D->B, h->num_sms, h->stream, h->d_err));   // B = V^T W
            k_proj_coef_m<<<1, 256, 0, h->stream>>>(k, m, D->B, D->Cp);
            CK(cudaGetLastError());
            CombineOut<T> o1{};
            o1.z[0] = W; o1.C[0] = D->Cp; o1.c0[0] = 0; o1.norm_of = -1; o1.Cf = s->Cf;
            CK(launch_combine<T>(n, k, nb + 1, awv, 1, o1, nullptr, h->num_sms, h->stream));   // W -= V B
        }
        CK(launch_gram<T>(n, k, 1, aw, 1, aw, s->B, h->num_sms, h->stream, h->d_err));         // W^T W
        CK(launch_orth_factor(k, s->B, s->Tm, s->status, h->stream));
        CombineOut<T> o2{};
        o2.z[0] = W; o2.C[0] = s->Tm; o2.c0[0] = 0; o2.norm_of = -1; o2.Cf = s->Cf;
        CK(launch_combine<T>(n, k, 1, aw, 1, o2, nullptr, h->num_sms, h->stream));              // W <- W T
    }
    return cudaSuccess;
}

template <typename T>
T **dav_v(DavState *D);
template <>
float **dav_v<float>(DavState *D) { return D->V32; }
template <>
double **dav_v<double>(DavState *D) { return D->V64; }
template <typename T>
T **dav_hv(DavState *D);
template <>
float **dav_hv<float>(DavState *D) { return D->HV32; }
template <>
double **dav_hv<double>(DavState *D) { return D->HV64; }

template <typename T>
cudaError_t dav_phase(lobpcg_ctx *h, SolverState *s, DavState *D, int max_iters, bool stop_on_stagnation,
                      PhaseResult &res, lobpcg_stats *st, lobpcg_status &status) {
    const int k = s->k, nev = h->params.nev;
    const int64_t n = h->T.n;
    const double tol = h->params.tol;
    const size_t blk = sizeof(T) * n * k;
    Blocks<T> &b = blocks_of<T>(s);
    T **V = dav_v<T>(D), **HV = dav_hv<T>(D);
    const int pmode = effective_precond<T>(h);
    const char *tag = std::is_same<T, float>::value ? "dav32" : "dav64";
    status = LOBPCG_OK;
    // V_0: an orthonormal basis of X
    CK(cudaMemcpyAsync(V[0], b.X, blk, cudaMemcpyDeviceToDevice, h->stream));
    CK(dav_orth<T>(h, s, D, V, 0, V[0]));
    CK(spmm_T<T>(h, V[0], HV[0], k));
    int nb = 1, restarts = 0, since_best = 0, since_floor = 0;
    int fresh = 0;   // leading blocks of the basis whose rows of G and O are current (float32 runs)
    double best = INFINITY, floor_best = INFINITY;
    std::vector<double> rho, theta;
    const int ldg = D->nbmax * k;   // float32 runs keep G and O at this leading dimension
    while (true) {
        const int m = nb * k;
        GemmBlocks<T> av{}, ahv{};
        for (int q = 0; q < nb; ++q) {
            av.p[q] = V[q];
            ahv.p[q] = HV[q];
        }
        bool incremental = false;
        if constexpr (std::is_same<T, float>::value) {
            // Only the blocks added since the last Rayleigh-Ritz step are new:
            // for each, V_q^T HV_b and V_q^T V_b (q <= b) by one pair-Gram
            // launch, mirrored into row b (the older blocks are unchanged).
            const float *probe[2] = {V[0], HV[0]};
            incremental = gram_pairs_fit(k, 2, probe, 2 * D->nbmax, 2 * D->nbmax * (k / 4) * (k / 4));
            if (incremental) {
                k_dav_zero<<<1, 256, 0, h->stream>>>(D->G, ldg, m, fresh * k);
                CK(cudaGetLastError());
                for (int b = fresh; b < nb; ++b) {
                    const float *gb[8];   // V_0 .. V_b, HV_b
                    for (int q = 0; q <= b; ++q) gb[q] = V[q];
                    gb[b + 1] = HV[b];
                    GramPair pr[12];
                    int np = 0;
                    for (int q = 0; q <= b; ++q) {
                        const int fl = q < b ? GRAM_MIRROR : 0;
                        pr[np++] = GramPair{q, b + 1, q, b, fl, b, q};                                // V_q^T HV_b
                        pr[np++] = GramPair{q, b, D->nbmax + q, b, fl, D->nbmax + b, q};              // V_q^T V_b
                    }
                    CK(launch_gram_pairs(n, k, b + 2, gb, np, pr, D->G, ldg, 2 * ldg, false, h->d_err,
                                         h->num_sms, h->stream));
                }
                fresh = nb;
                CK(launch_rayleigh_ritz(m, k, m, D->G, D->G + ldg * ldg, ldg, nullptr, D->C, s->theta, s->status,
                                        h->stream));
            }
        }
        if (!incremental) {
            CK(launch_gram<T>(n, k, nb, av, nb, ahv, D->G, h->num_sms, h->stream, h->d_err));           // V^T HV
            CK(launch_gram<T>(n, k, nb, av, nb, av, D->G + m * m, h->num_sms, h->stream, h->d_err));    // V^T V
            CK(launch_rayleigh_ritz(m, k, m, D->G, D->G + m * m, m, nullptr, D->C, s->theta, s->status, h->stream));
        }
        CombineOut<T> ox{}, oh{};
        ox.z[0] = b.X; ox.C[0] = D->C; ox.c0[0] = 0; ox.norm_of = -1; ox.Cf = s->Cf;
        oh.z[0] = b.HX; oh.C[0] = D->C; oh.c0[0] = 0; oh.norm_of = -1; oh.Cf = s->Cf;
        CK(launch_combine<T>(n, k, nb, av, 1, ox, nullptr, h->num_sms, h->stream));     // X = V C
        CK(launch_combine<T>(n, k, nb, ahv, 1, oh, nullptr, h->num_sms, h->stream));    // HX = HV C
        CK(launch_resid<T>(n, k, b.X, b.HX, s->theta, h->T.diag, b.W, pmode == 1 ? 1 : 0, s->norms, h->num_sms,
                           h->stream));
        int rr_st = 0, orth_st = 0;
        CK(read_progress<T>(h, s, rho, theta, &rr_st, &orth_st, st));
        trace(tag, res.iters, rho, theta, nev, rr_st);
        if (rr_st == 2) {
            status = LOBPCG_ERR_BREAKDOWN;
            break;
        }
        if (orth_st == 1 && st) st->svqb_used++;
        bool finite = true;
        for (int j = 0; j < k; ++j) finite = finite && std::isfinite(rho[j]) && std::isfinite(theta[j]);
        if (!finite) {
            status = LOBPCG_ERR_NONFINITE;
            break;
        }
        double worst = 0.0;
        for (int j = 0; j < nev; ++j) worst = std::max(worst, rho[j]);
        if (worst <= tol) {
            // explicit re-check: H X from a fresh SpMM (into HW as scratch)
            CK(spmm_T<T>(h, b.X, b.HW, k));
            CK(launch_resid<T>(n, k, b.X, b.HW, s->theta, h->T.diag, b.W, pmode == 1 ? 1 : 0, s->norms,
                               h->num_sms, h->stream));
            CK(read_progress<T>(h, s, rho, theta, &rr_st, &orth_st, st));
            double worst_e = 0.0;
            for (int j = 0; j < nev; ++j) worst_e = std::max(worst_e, rho[j]);
            trace("check", res.iters, rho, theta, nev, 0);
            if (worst_e <= tol || restarts >= 5) {
                res.converged = worst_e <= tol;
                break;
            }
            ++restarts;
            if (st) st->explicit_restarts++;
            // continue from the Ritz vectors and their explicit product
            CK(cudaMemcpyAsync(V[0], b.X, blk, cudaMemcpyDeviceToDevice, h->stream));
            CK(cudaMemcpyAsync(HV[0], b.HW, blk, cudaMemcpyDeviceToDevice, h->stream));
            nb = 1;
            fresh = 0;
            continue;
        }
        // a float32 run hands over once its residual stalls (15 iterations
        // without a 0.7x gain, best below 1e-2), grows 4x above a best below
        // 1e-3 or sits at a floor (below 1e-2, no new 5 % minimum in 3
        // iterations)
        if (worst < 0.95 * floor_best) {
            floor_best = worst;
            since_floor = 0;
        } else {
            ++since_floor;
        }
        if (worst < 0.7 * best) {
            best = worst;
            since_best = 0;
        } else if (stop_on_stagnation && ((++since_best >= 15 && best < 1e-2) || (best < 1e-3 && worst > 4.0 * best) ||
                                          (floor_best < 1e-2 && since_floor >= 3))) {
            res.stagnated = true;
            break;
        }
        if (res.iters >= max_iters) break;
        ++res.iters;
        if (pmode >= 2) CK(precond_apply<T>(h, pmode, k, b.W, s->theta, b.W, h->stream));
        if (nb == D->nbmax) {   // restart with the Ritz vectors
            CK(cudaMemcpyAsync(V[0], b.X, blk, cudaMemcpyDeviceToDevice, h->stream));
            CK(cudaMemcpyAsync(HV[0], b.HX, blk, cudaMemcpyDeviceToDevice, h->stream));
            nb = 1;
            fresh = 0;
        }
        CK(cudaMemcpyAsync(V[nb], b.W, blk, cudaMemcpyDeviceToDevice, h->stream));
        CK(dav_orth<T>(h, s, D, V, nb, V[nb]));
        CK(timed_spmm<T>(h, s, V[nb], HV[nb], k));   // the one SpMM per iteration
        ++nb;
    }
    res.rho = rho;
    res.theta = theta;
    return cudaSuccess;
}

cudaError_t dav_setup(lobpcg_ctx *h, int nbmax) {
    DavState *D = new DavState();
    h->dav = D;
    const int k = h->params.k;
    const int64_t n = h->T.n;
    D->k = k;
    D->nbmax = nbmax;
    const int mmax = nbmax * k;
    for (int q = 0; q < nbmax; ++q) {
        CK(dev_alloc(h, reinterpret_cast<void **>(&D->V32[q]), sizeof(float) * n * k));
        CK(dev_alloc(h, reinterpret_cast<void **>(&D->HV32[q]), sizeof(float) * n * k));
        if (h->params.polish_fp64) {
            CK(dev_alloc(h, reinterpret_cast<void **>(&D->V64[q]), sizeof(double) * n * k));
            CK(dev_alloc(h, reinterpret_cast<void **>(&D->HV64[q]), sizeof(double) * n * k));
        }
    }
    CK(dev_alloc(h, reinterpret_cast<void **>(&D->G), sizeof(double) * 2 * mmax * mmax));
    CK(dev_alloc(h, reinterpret_cast<void **>(&D->C), sizeof(double) * mmax * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&D->B), sizeof(double) * mmax * k));
    CK(dev_alloc(h, reinterpret_cast<void **>(&D->Cp), sizeof(double) * (mmax + k) * k));
    return cudaSuccess;
}

}  // namespace

namespace lobpcg {

lobpcg_status davidson(lobpcg_ctx *h, float *Xio, bool x_on_host, int max_blocks, double *evals, double *resid,
                       lobpcg_stats *st, std::string &err) {
    SolverState *s = h->solver;
    const int k = s->k, nev = h->params.nev;
    const int64_t n = h->T.n;
    const size_t bytes32 = sizeof(float) * n * k;
    auto t0 = std::chrono::steady_clock::now();
    if (st) std::memset(st, 0, sizeof(*st));
    auto cuda_err = [&](const char *where, cudaError_t e) {
        err = std::string(where) + ": " + cudaGetErrorString(e);
        return LOBPCG_ERR_CUDA;
    };
    if (!h->dav) {
        cudaError_t e = dav_setup(h, max_blocks);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LOBPCG_ERR_OOM : cuda_err("davidson setup", e);
    } else if (max_blocks > h->dav->nbmax) {
        err = "max_blocks larger than at the first lobpcg_davidson call on this handle";
        return LOBPCG_ERR_ARG;
    }
    DavState *D = h->dav;
    const int saved = D->nbmax;
    D->nbmax = max_blocks;
    cudaError_t e = cudaMemcpyAsync(s->f.X, Xio, bytes32, x_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                    h->stream);
    if (e != cudaSuccess) return cuda_err("davidson", e);
    PhaseResult r32;
    lobpcg_status status = LOBPCG_OK;
    const bool polish = h->params.polish_fp64 && s->d.X && D->V64[0];
    e = dav_phase<float>(h, s, D, h->params.maxiter, polish, r32, st, status);
    if (e != cudaSuccess) { D->nbmax = saved; return cuda_err("davidson (fp32)", e); }
    PhaseResult final = r32;
    int iters64 = 0;
    bool used64 = false;
    const int nb = std::max(1, std::min<int>(h->num_sms * 8, static_cast<int>((n * k + 255) / 256)));
    if (status == LOBPCG_OK && !r32.converged && polish) {
        k_convert<float, double><<<nb, 256, 0, h->stream>>>(n * k, s->f.X, s->d.X);
        PhaseResult r64;
        e = dav_phase<double>(h, s, D, std::max(0, h->params.maxiter - r32.iters), false, r64, st, status);
        if (e != cudaSuccess) { D->nbmax = saved; return cuda_err("davidson (fp64)", e); }
        iters64 = r64.iters;
        final = r64;
        used64 = true;
        k_convert<double, float><<<nb, 256, 0, h->stream>>>(n * k, s->d.X, s->f.X);
    } else if (s->d.X) {
        k_convert<float, double><<<nb, 256, 0, h->stream>>>(n * k, s->f.X, s->d.X);
    }
    D->nbmax = saved;
    e = cudaMemcpyAsync(Xio, s->f.X, bytes32, x_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_err("davidson", e);
    for (int j = 0; j < nev && j < static_cast<int>(final.theta.size()); ++j) {
        if (evals) evals[j] = final.theta[j];
        if (resid) resid[j] = final.rho[j];
    }
    if (st) {
        st->iters = r32.iters + iters64;
        st->iters_fp64 = iters64;
        st->used_fp64 = used64 ? 1 : 0;
        st->converged = final.converged ? 1 : 0;
        st->time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status != LOBPCG_OK) {
        err = status == LOBPCG_ERR_BREAKDOWN ? "Rayleigh-Ritz breakdown" : "non-finite residual";
        return status;
    }
    if (!final.converged) {
        err = "maxiter reached before the residual tolerance";
        return LOBPCG_ERR_NOT_CONVERGED;
    }
    return LOBPCG_OK;
}

}  // namespace lobpcg
