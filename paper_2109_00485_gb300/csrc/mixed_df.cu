// Dense steps of the float64 refinement in compensated float32 (df.cuh):
//
//   k_xupdate2_df  X <- X C + P and HX <- HX C + HP (float64 in place, C
//                  k x k float64, P and HP float32) with their float32
//                  copies, and the next residual HX - X Theta, its
//                  preconditioned copy and norms: the X and HX updates of
//                  the refinement fused with the following residual
//   k_gram_x_df    G = X^T [HX X] (k x 2k float64) from float64 X and HX:
//                  the Gram blocks the refinement keeps in float64
//
// Each float64 input is split into a float pair on its bit pattern, the
// products summed with error-free transformations in float32 (relative
// error of a few 2^-47 per term), and only the results touch the FP64
// pipe: one float64 addition per output of the update, and per Gram entry
// two every 64 rows (the fold of a float pair into a float64 sum).
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>
#include "df.cuh"
#include "dense.h"

namespace lobpcg {

namespace {

constexpr int XU_THREADS = 256;

// Both updates and the next residual in one pass (k <= 32):
//   X <- X C + P, HX <- HX C + HP (float64, X32 / HX32 their float32 copies)
//   R = HX - X Theta (float32 R32), W = R (mode 0) or R / g(d_i - theta_j)
//   (mode 1, the guarded diagonal preconditioner), norms += (||r_j||^2,
//   ||x_j||^2).  The updated X and HX enter the residual as float pairs, so
//   HX - X Theta is formed without cancellation loss: TwoSum of hx_hi and
//   -fl(x_hi theta_hi), the rest in the low word.
// With C23 (float64, nz k x k: the W and P rows of the Ritz coefficients)
// the new search directions are formed here too, in float32 from the staged
// rows: P <- [W P] C23, HP <- [HW HP] C23 (P and HP in place, the P block
// left out when nz = 1), colsq += ||p_j||^2; W, the basis block, is read
// before the new W is written over it.
__global__ void __launch_bounds__(XU_THREADS) k_xupdate2_df(int64_t n, int k, double *X, double *HX, const double *C,
                                                            float *P, float *HP, float *X32, float *HX32,
                                                            const double *theta, const float *d, float *W, float *R32,
                                                            int mode, double *norms, const float *Wb,
                                                            const float *HWb, const double *C23, int nz,
                                                            double *colsq) {
    // C's words as duplicated pairs (c, c), (-c, -c), (c_lo, c_lo) (k x k
    // each); a row element of X and HX as the pairs (x_hi, hx_hi), (x_lo,
    // hx_lo) (per x k each): one packed df_mac2 updates x and hx together
    extern __shared__ float2 xs2[];
    __shared__ double red[96];      // [3k]
    const int per = XU_THREADS / k;
    float2 *cp = xs2, *cn = xs2 + k * k, *cl = xs2 + 2 * k * k, *zh = xs2 + 3 * k * k, *zl = zh + per * k;
    // the fused directions: the pass's rows of W, P, HW, HP, and C23 in float32
    float *wr = reinterpret_cast<float *>(zl + per * k), *pr = wr + per * k, *hwr = pr + per * k,
          *hpr = hwr + per * k, *c23 = hpr + per * k;
    const bool fuse = C23 != nullptr;
    if (fuse)
        for (int q = threadIdx.x; q < nz * k * k; q += blockDim.x) c23[q] = __double2float_rn(C23[q]);
    for (int q = threadIdx.x; q < k * k; q += blockDim.x) {
        float a, b;
        df_split(C[q], a, b);
        cp[q] = make_float2(a, a);
        cn[q] = make_float2(-a, -a);
        cl[q] = make_float2(b, b);
    }
    for (int q = threadIdx.x; q < 3 * k; q += blockDim.x) red[q] = 0.0;
    const int r = threadIdx.x / k, j = threadIdx.x % k;
    const bool active = r < per;
    float th_h = 0.f, th_l = 0.f;
    if (active) df_split(theta[j], th_h, th_l);
    const float thf = __fadd_rn(th_h, th_l);
    const float delta = 1e-3f * fmaxf(1.f, fabsf(thf));
    // float32 sums of nonnegative terms over this thread's rows (a few
    // hundred at most: relative error below 1e-4, enough for the norms'
    // use in the convergence test), folded into float64 once at the end
    float rr = 0.f, xx = 0.f, pp = 0.f;
    // a pass's inputs are loaded during the pass before (thread r k + j
    // loads element (r, j) of X and HX, which it also updates)
    const int64_t step = static_cast<int64_t>(gridDim.x) * per;
    double fx = 0.0, fh = 0.0;
    float fp = 0.f, fhp = 0.f, fd = 0.f, fw = 0.f, fhw = 0.f;
    auto fetch = [&](int64_t i) {
        const int rws = static_cast<int>(n - i < per ? n - i : per);
        if (threadIdx.x < rws * k) {
            fx = X[i * k + threadIdx.x];
            fh = HX[i * k + threadIdx.x];
            if (!fuse || nz == 2) {
                fp = P[i * k + threadIdx.x];
                fhp = HP[i * k + threadIdx.x];
            }
            if (fuse) {
                fw = Wb[i * k + threadIdx.x];
                fhw = HWb[i * k + threadIdx.x];
            }
            if (mode == 1) fd = d[i + r];
        }
    };
    if (static_cast<int64_t>(blockIdx.x) * per < n) fetch(static_cast<int64_t>(blockIdx.x) * per);
    for (int64_t i0 = static_cast<int64_t>(blockIdx.x) * per; i0 < n; i0 += step) {
        const int rows = static_cast<int>(n - i0 < per ? n - i0 : per);
        const float pe = fp, hpe = fhp, de = fd;
        __syncthreads();
        if (threadIdx.x < rows * k) {
            float a, b, c, e;
            df_split(fx, a, b);
            df_split(fh, c, e);
            zh[threadIdx.x] = make_float2(a, c);
            zl[threadIdx.x] = make_float2(b, e);
            if (fuse) {
                wr[threadIdx.x] = fw;
                hwr[threadIdx.x] = fhw;
                pr[threadIdx.x] = fp;
                hpr[threadIdx.x] = fhp;
            }
        }
        __syncthreads();
        if (i0 + step < n) fetch(i0 + step);
        if (active && r < rows) {
            float2 s2 = make_float2(0.f, 0.f), c2 = s2;   // (x, hx) sums and compensations
            for (int l = 0; l < k; ++l)
                df_mac2(zh[r * k + l], zl[r * k + l], cp[l * k + j], cn[l * k + j], cl[l * k + j], s2, c2);
            const float sx = s2.x, cx = c2.x, sh = s2.y, chh = c2.y;
            const int64_t e = (i0 + r) * k + j;
            float pn = pe, hpn = hpe;
            if (fuse) {   // P = [W P] C23, HP = [HW HP] C23
                float a = 0.f, b = 0.f;
                for (int l = 0; l < k; ++l) {
                    const float c = c23[l * k + j];
                    a = __fmaf_rn(wr[r * k + l], c, a);
                    b = __fmaf_rn(hwr[r * k + l], c, b);
                }
                if (nz == 2)
                    for (int l = 0; l < k; ++l) {
                        const float c = c23[(k + l) * k + j];
                        a = __fmaf_rn(pr[r * k + l], c, a);
                        b = __fmaf_rn(hpr[r * k + l], c, b);
                    }
                pn = a;
                hpn = b;
                P[e] = a;
                HP[e] = b;
                pp = __fmaf_rn(a, a, pp);
            }
            // + P, + HP: TwoSum with the high word, the rest into the low word
            auto add = [](float s, float c, float a, float &u, float &v) {
                u = __fadd_rn(s, a);
                const float ba = __fsub_rn(u, s);
                v = __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(u, ba)), __fsub_rn(a, ba)), c);
            };
            float ux, vx, uh, vh;
            add(sx, cx, pn, ux, vx);
            add(sh, chh, hpn, uh, vh);
            X[e] = df_to_f64(ux) + df_to_f64(vx);
            HX[e] = df_to_f64(uh) + df_to_f64(vh);
            const float x32 = __fadd_rn(ux, vx);
            X32[e] = x32;
            HX32[e] = __fadd_rn(uh, vh);
            // r = hx - x theta: x theta = p + ep + cross (p = fl(ux th_h), exact with ep)
            const float p = __fmul_rn(ux, th_h);
            const float ep = __fmaf_rn(ux, th_h, -p);
            const float cross = __fmaf_rn(ux, th_l, __fmul_rn(vx, th_h));
            float a0, a1;
            add(uh, vh, -p, a0, a1);
            const float rf = __fadd_rn(a0, __fsub_rn(a1, __fadd_rn(ep, cross)));
            R32[e] = rf;
            float w = rf;
            if (mode == 1) {
                const float t = __fsub_rn(de, thf);
                const float g = (t >= 0.f) ? fmaxf(t, delta) : -fmaxf(-t, delta);
                w = w / g;
            }
            W[e] = w;
            rr = __fmaf_rn(rf, rf, rr);
            xx = __fmaf_rn(x32, x32, xx);
        }
    }
    if (active) {
        atomicAdd(&red[j], static_cast<double>(rr));
        atomicAdd(&red[k + j], static_cast<double>(xx));
        atomicAdd(&red[2 * k + j], static_cast<double>(pp));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * k; q += blockDim.x) atomicAdd(&norms[q], red[q]);
    if (fuse)
        for (int q = threadIdx.x; q < k; q += blockDim.x) atomicAdd(&colsq[q], red[2 * k + q]);
}

constexpr int GX_THREADS = 256;
constexpr int GX_ROWS = 128;    // rows staged per pass at most (and folded into float64 per pass)
constexpr int GX_PER = 8;       // values of X (and of HX) a thread loads per pass: rows x k <= 8 x 256

// G = X^T [HX X] (k x 2k) with both k x k blocks symmetric: only their lower
// triangles are summed (H is symmetric, so X^T HX is in exact arithmetic)
// and mirrored on output.  The k columns are padded to kp (even) and each
// block's lower triangle covered by 2 x 2 sub-blocks ("units": U = 2 T,
// T = nb (nb + 1) / 2, nb = kp / 2); thread L (of `groups` x U, UPT units a
// thread) owns unit L % U and takes the pass's rows g, g + groups, ...
// (g = L / U), four df_mac per row from two float2 loads of each operand.
template <int UPT>
__global__ void __launch_bounds__(GX_THREADS) k_gram_x_df(int64_t n, int k, const double *X, const double *HX,
                                                          double *G) {
    extern __shared__ float gs[];   // xh, xl, yh, yl: GX_ROWS x kp each (y = HX rows)
    const int kp = (k + 1) & ~1, nb = kp / 2, T = nb * (nb + 1) / 2, U = 2 * T;
    const int groups = U <= GX_THREADS ? GX_THREADS / U : 1;
    float *xh = gs, *xl = gs + GX_ROWS * kp, *yh = gs + 2 * GX_ROWS * kp, *yl = gs + 3 * GX_ROWS * kp;
    for (int q = threadIdx.x; q < 4 * GX_ROWS * kp; q += blockDim.x) gs[q] = 0.f;   // padding columns stay 0
    int grp[UPT], ia[UPT], ib[UPT];
    bool hxb[UPT], valid[UPT];
    double acc[UPT][4];
    float2 sv[UPT][2], cv[UPT][2];   // entries (0, 1) and (2, 3) of a unit as packed pairs
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
        const int L = threadIdx.x + GX_THREADS * q;
        grp[q] = L / U;
        valid[q] = grp[q] < groups;
        int t = L % U;
        hxb[q] = t < T;
        if (!hxb[q]) t -= T;
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        ia[q] = 2 * bi;
        ib[q] = 2 * (t - bi * (bi + 1) / 2);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[q][e] = 0.0;
        sv[q][0] = sv[q][1] = cv[q][0] = cv[q][1] = make_float2(0.f, 0.f);
    }
    const int64_t per_cta = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * per_cta;
    const int64_t r1 = std::min<int64_t>(n, r0 + per_cta);
    const int RP = GX_PER * GX_THREADS / k < GX_ROWS ? GX_PER * GX_THREADS / k : GX_ROWS;   // rows per pass
    // a pass's rows are loaded into registers during the pass before
    double px[GX_PER], ph[GX_PER];
    auto fetch = [&](int64_t a, int rows) {
#pragma unroll
        for (int t = 0; t < GX_PER; ++t) {
            const int q = threadIdx.x + GX_THREADS * t;
            if (q < rows * k) {
                px[t] = X[a * k + q];
                ph[t] = HX[a * k + q];
            }
        }
    };
    if (r0 < r1) fetch(r0, static_cast<int>(std::min<int64_t>(RP, r1 - r0)));
    for (int64_t a = r0; a < r1; a += RP) {
        const int rows = static_cast<int>(std::min<int64_t>(RP, r1 - a));
        __syncthreads();
#pragma unroll
        for (int t = 0; t < GX_PER; ++t) {
            const int q = threadIdx.x + GX_THREADS * t;
            if (q < rows * k) {
                const int r = q / k, c = q - r * k;
                df_split(px[t], xh[r * kp + c], xl[r * kp + c]);
                df_split(ph[t], yh[r * kp + c], yl[r * kp + c]);
            }
        }
        __syncthreads();
        if (a + RP < r1) fetch(a + RP, static_cast<int>(std::min<int64_t>(RP, r1 - a - RP)));
#pragma unroll
        for (int q = 0; q < UPT; ++q) {
            if (!valid[q]) continue;
            const float *bh = hxb[q] ? yh : xh, *bl = hxb[q] ? yl : xl;
            for (int r = grp[q]; r < rows; r += groups) {
                const float2 ah = *reinterpret_cast<const float2 *>(xh + r * kp + ia[q]);
                const float2 al = *reinterpret_cast<const float2 *>(xl + r * kp + ia[q]);
                const float2 h2 = *reinterpret_cast<const float2 *>(bh + r * kp + ib[q]);
                const float2 l2 = *reinterpret_cast<const float2 *>(bl + r * kp + ib[q]);
                const float2 nh2 = make_float2(-h2.x, -h2.y);
                df_mac2(make_float2(ah.x, ah.x), make_float2(al.x, al.x), h2, nh2, l2, sv[q][0], cv[q][0]);
                df_mac2(make_float2(ah.y, ah.y), make_float2(al.y, al.y), h2, nh2, l2, sv[q][1], cv[q][1]);
            }
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {
                acc[q][2 * e2] += df_to_f64(sv[q][e2].x) + df_to_f64(cv[q][e2].x);
                acc[q][2 * e2 + 1] += df_to_f64(sv[q][e2].y) + df_to_f64(cv[q][e2].y);
                sv[q][e2] = cv[q][e2] = make_float2(0.f, 0.f);
            }
        }
    }
    // sum the groups' partials in shared memory, then one atomic per entry
    // (and its mirror)
    __syncthreads();
    double *red = reinterpret_cast<double *>(gs);   // [groups][U][4]
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
        if (!valid[q]) continue;
        const int L = threadIdx.x + GX_THREADS * q;
#pragma unroll
        for (int e = 0; e < 4; ++e) red[L * 4 + e] = acc[q][e];
    }
    __syncthreads();
    if (r0 >= r1) return;
    for (int v = threadIdx.x; v < 4 * U; v += blockDim.x) {
        double sum = 0.0;
        for (int g = 0; g < groups; ++g) sum += red[g * 4 * U + v];
        const int u = v / 4, e = v % 4;
        int t = u;
        const bool hx = t < T;
        if (!hx) t -= T;
        int bi = 0;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        const int i = 2 * bi + (e >> 1), j = 2 * (t - bi * (bi + 1) / 2) + (e & 1);
        if (i >= k || j > i) continue;
        const int off = hx ? 0 : k;
        atomicAdd(&G[i * 2 * k + off + j], sum);
        if (j != i) atomicAdd(&G[j * 2 * k + off + i], sum);
    }
}

}  // namespace

bool mixed_df_ok(int k) { return k >= 1 && k <= 32; }

cudaError_t launch_xupdate2_df(int64_t n, int k, double *X, double *HX, const double *C, float *P, float *HP,
                               float *X32, float *HX32, const double *theta, const float *d, float *W, float *R32,
                               int mode, double *norms, int num_sms, cudaStream_t s, const float *Wb,
                               const float *HWb, const double *C23, int nz, double *colsq) {
    if (!mixed_df_ok(k) || (C23 && (nz < 1 || nz > 2 || !Wb || !HWb || !colsq))) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * k, s);
    if (e == cudaSuccess && C23) e = cudaMemsetAsync(colsq, 0, sizeof(double) * k, s);
    if (e != cudaSuccess) return e;
    const int per = XU_THREADS / k;
    const size_t smem = sizeof(float2) * (3 * k * k + 2 * per * k) + sizeof(float) * (4 * per * k + 2 * k * k);
    int blocks = static_cast<int>(std::min<int64_t>((n + per - 1) / per, static_cast<int64_t>(num_sms) * 8));
    if (blocks < 1) blocks = 1;
    k_xupdate2_df<<<blocks, XU_THREADS, smem, s>>>(n, k, X, HX, C, P, HP, X32, HX32, theta, d, W, R32, mode, norms,
                                                   Wb, HWb, C23, nz, colsq);
    return cudaGetLastError();
}

cudaError_t launch_gram_x_df(int64_t n, int k, const double *X, const double *HX, double *G, int num_sms,
                             cudaStream_t s) {
    if (!mixed_df_ok(k)) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * 2 * k * k, s);
    if (e != cudaSuccess) return e;
    const int kp = (k + 1) & ~1, nb = kp / 2, U = nb * (nb + 1);
    const int groups = U <= GX_THREADS ? GX_THREADS / U : 1;
    // the staged rows, later the [groups][U][4] float64 partials
    const size_t smem = std::max(sizeof(float) * 4 * GX_ROWS * kp, sizeof(double) * 4 * groups * U);
    int blocks = static_cast<int>(std::min<int64_t>((n + GX_ROWS - 1) / GX_ROWS, static_cast<int64_t>(num_sms) * 3));
    if (blocks < 1) blocks = 1;
    if (U <= GX_THREADS) {
        e = cudaFuncSetAttribute(k_gram_x_df<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        k_gram_x_df<1><<<blocks, GX_THREADS, smem, s>>>(n, k, X, HX, G);
    } else {
        e = cudaFuncSetAttribute(k_gram_x_df<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        k_gram_x_df<2><<<blocks, GX_THREADS, smem, s>>>(n, k, X, HX, G);
    }
    return cudaGetLastError();
}

}  // namespace lobpcg
