/*
 * lobpcg.h - C ABI of the GB300 (sm_103a) block LOBPCG eigensolver for a
 * sparse symmetric matrix H stored as one triangle.
 *
 * Method: Maris, Yang, Oryspayev, Cook, "Accelerating an Iterative
 * Eigensolver for Nuclear Structure Configuration Interaction Calculations
 * on GPUs using OpenACC" (arXiv 2109.00485).  Each entry point below names
 * the passage of the paper that defines the operation it performs.
 *
 * Conventions shared by every call
 *   - Blocks of vectors (X, Y, R, W, ...) are n x k, ROW-MAJOR: the k entries
 *     of one row are contiguous (Section 3.3: "multiple vectors are stored in
 *     row major order").  Row stride = k elements.
 *   - Pointers are DEVICE pointers unless a parameter says "host".  The
 *     library never frees caller memory; it copies what it keeps.
 *   - Every call is ordered on the handle's CUDA stream (given at create).
 *     Calls that return host results synchronise that stream first.
 *   - Errors are returned as lobpcg_status; no call aborts, traps or throws.
 *     lobpcg_last_error() gives a one-line description of the last failure
 *     on a handle.
 *   - One handle is not safe for concurrent use from several host threads.
 */
#ifndef LOBPCG_H
#define LOBPCG_H

#include <stdint.h>

#if defined(__GNUC__)
#define LOBPCG_API __attribute__((visibility("default")))
#else
#define LOBPCG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lobpcg_ctx *lobpcg_t;

typedef enum {
    LOBPCG_OK = 0,
    LOBPCG_ERR_ARG = 1,            /* invalid argument (size, pointer, alignment, k) */
    LOBPCG_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    LOBPCG_ERR_OOM = 3,            /* device or host allocation failed */
    LOBPCG_ERR_BREAKDOWN = 4,      /* orthonormalisation / Rayleigh-Ritz breakdown */
    LOBPCG_ERR_NONFINITE = 5,      /* NaN or Inf detected */
    LOBPCG_ERR_NOT_CONVERGED = 6,  /* maxiter reached; outputs still written */
    LOBPCG_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
    LOBPCG_ERR_BOUNDS = 8,         /* matrix structure invalid (unsorted, out of range, upper entry) */
    LOBPCG_ERR_UNSUPPORTED = 9     /* valid request this build does not handle */
} lobpcg_status;

typedef enum { LOBPCG_MEM_DEVICE = 0, LOBPCG_MEM_HOST = 1 } lobpcg_mem;

/*
 * The lower triangle L of H, diagonal included, in CSR (Section 3.1: only
 * half of the symmetric H is stored; H = L + L^T - diag(L)).
 *   row_ptr : int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz
 *   col     : int32[nnz], strictly increasing within a row, 0 <= col <= row
 *   val     : float64[nnz] if val_is_fp64, else float32[nnz]
 *   mem     : where the three arrays live (device or host)
 * Limits: 1 <= n < 2^28, nnz < 2^40.
 */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int64_t *row_ptr;
    const int32_t *col;
    const void *val;
    int32_t val_is_fp64;
    int32_t mem;
} lobpcg_matrix;

/* Solver parameters (Algorithm 1 inputs: tol, maxiter; block size k). */
typedef struct {
    int32_t k;           /* block size, 1..32 */
    int32_t nev;         /* wanted eigenpairs, 1..k */
    int32_t maxiter;     /* iteration limit */
    double tol;          /* relative residual tolerance */
    int32_t precond;     /* 0 none, 1 diagonal, 2 block-Jacobi (64-row tiles), 3 learned MLP,
                            4 FOM on the shifted 64-row tiles (Section 3.3) */
    int32_t resid_mode;  /* 0: ||r||/(max(|theta|,1e-12||H||_G)||x||), 1: ||r||/(||H||_G||x||) */
    int32_t polish_fp64; /* 1: finish with FP64 vectors once FP32 stagnates */
    int32_t tile_format; /* 0: every stored entry keeps its index word and value word (8 bytes,
                            as CSR's column index and value); 1: a 16x16 tile holding all 256
                            entries, or a diagonal tile with its complete lower triangle, keeps
                            its value words only (4 bytes per entry, the positions implied;
                            Section 3.3 keeps 2-byte local indices in its compressed sparse
                            blocks for the same reason: fewer index bytes per entry) */
    uint64_t seed;
    int32_t fom_steps;   /* FOM iterations per tile for precond 4: 1..6, 0 = 4 (Section 3.3:
                            three to five are enough) */
    int32_t reserved;    /* must be 0 */
    const int64_t *fom_tile_ptr; /* precond 4: row partition into diagonal tiles, HOST memory,
                            fom_ntiles + 1 strictly increasing boundaries from 0 to n (tile t
                            is rows [fom_tile_ptr[t], fom_tile_ptr[t+1])), read during create
                            only; any sizes (the paper's tiles run from 1 to thousands of
                            rows).  NULL: consecutive 64-row tiles. */
    int64_t fom_ntiles;  /* tiles in fom_tile_ptr (ignored when it is NULL) */
} lobpcg_params;

/* Counters of one lobpcg_solve. */
typedef struct {
    int32_t iters;             /* LOBPCG iterations (one SpMM H W each), both phases */
    int32_t iters_fp64;        /* of which in the float64 refinement phase */
    int32_t used_fp64;         /* 1 if the float64 phase ran */
    int32_t converged;         /* 1 if all nev residuals met tol (explicit re-check) */
    int32_t p_dropped;         /* Rayleigh-Ritz steps that dropped P (O not positive definite) */
    int32_t svqb_used;         /* orthonormalisations that fell back to SVQB */
    int32_t explicit_restarts; /* convergence claims refuted by the explicit SpMM re-check */
    int32_t spmm_calls;        /* H W products timed below */
    double time_ms;            /* wall time of the call */
    double spmm_ms;            /* device time of the H W products (CUDA events on the handle's stream) */
} lobpcg_stats;

/* Facts about the stored matrix and its device layout (lobpcg_matrix_info). */
typedef struct {
    int64_t n, nnz;          /* as given */
    int64_t row_blocks;      /* ceil(n/16) */
    int64_t chunks;          /* (row block, 16-column tile) groups, diagonal chunks included */
    int64_t padded_nnz;      /* stored entries incl. padding to 4-entry boundaries */
    int64_t full_chunks;     /* chunks holding all 256 entries of their tile */
    int64_t device_bytes;    /* device memory held by the handle */
    double gershgorin;       /* ||H||_G = max_i sum_j |h_ij| over full rows */
    int32_t num_sms;
    int32_t warps;           /* warps the tiled SpMM kernel launches */
    int32_t tile_format;     /* as created */
    int32_t pad_;
    int64_t stream_bytes;    /* bytes of the tiled entry stream one SpMM reads */
} lobpcg_info;

/*
 * Create a handle for H.  Copies the triangle into the library's tiled
 * layout (values converted to float32), validates it (error BOUNDS on an
 * unsorted row, a column > row or out of range), computes ||H||_G and
 * allocates every workspace the solver needs (Section 4.4: handles and
 * work space are set up once, before the iteration loop).
 *   stream : cudaStream_t to order all work on (NULL = legacy default).
 * On failure *out is set to NULL and no memory is kept.
 */
LOBPCG_API lobpcg_status lobpcg_create(lobpcg_t *out, const lobpcg_matrix *A,
                            const lobpcg_params *params, void *stream);

/* Release every resource of the handle (NULL is accepted), on the handle's
 * device whatever device is current. */
LOBPCG_API lobpcg_status lobpcg_destroy(lobpcg_t h);

/*
 * Device check.  Every call below that reaches the device (all but
 * lobpcg_destroy, lobpcg_last_error and lobpcg_matrix_info) first checks
 * that the device current on the calling thread is the one that was current
 * at create, and returns ERR_ARG (the two ordinals in lobpcg_last_error)
 * without touching the device otherwise.
 *
 * Test hook for that check: overwrite the device ordinal recorded in the
 * handle (no CUDA call).  A handle whose ordinal is not the current device
 * refuses every device call; set the true ordinal back to use it again.
 */
LOBPCG_API lobpcg_status lobpcg_test_set_device_ordinal(lobpcg_t h, int32_t device);

/* One-line text of the last error on h (or of the last failed create if h is NULL). */
LOBPCG_API const char *lobpcg_last_error(lobpcg_t h);

/* Fill *info (host pointer). */
LOBPCG_API lobpcg_status lobpcg_matrix_info(lobpcg_t h, lobpcg_info *info);

/*
 * Wait for all work queued on the handle's stream and report device-side
 * failures of earlier calls (ERR_TIMEOUT if a bounded wait in a kernel gave
 * up).  Stream-ordered calls such as lobpcg_spmm_sym do not synchronise;
 * their device-side errors surface here or in the next synchronising call.
 */
LOBPCG_API lobpcg_status lobpcg_sync(lobpcg_t h);

/*
 * Y = H X from the stored triangle in one pass over it: every stored
 * h_ij (j <= i) adds h_ij x_j to y_i and, for j < i, h_ij x_i to y_j.
 * This is the product the paper computes as the local SpMM of Algorithm 2
 * plus its transpose (Sections 3.2-3.3, eqs. upd1-upd2: the one SpMM per
 * iteration), fused here into a single pass.
 *   X : float32 n x k row-major (read only)
 *   Y : float32 n x k row-major (overwritten); must not overlap X
 *       X and Y are both device pointers, or both host pointers (pinned
 *       memory gives asynchronous copies): host blocks are copied through
 *       device staging buffers held by the handle, and Y is complete once
 *       the stream has been synchronised (lobpcg_sync).
 *   k : 1..32.  k % 4 == 0 with 16-byte aligned X and Y takes the tiled
 *       kernel; any other k or alignment takes a simpler atomic kernel.
 * Accumulation is float32; the order of additions is not fixed, so results
 * may differ in the last bits from call to call.  NaN/Inf in X propagates to
 * every row that shares a 16x16 tile with it.
 * Returns LOBPCG_OK, or ERR_ARG (k, NULL, overlap), ERR_CUDA, ERR_TIMEOUT.
 */
LOBPCG_API lobpcg_status lobpcg_spmm_sym(lobpcg_t h, const float *X, float *Y, int32_t k);

/*
 * Same product, FP64 vectors: X, Y float64 n x k row-major; the stored
 * float32 values are used exactly; accumulation in float64.  Used to check
 * and polish converged eigenpairs.  k: 1..32.
 */
LOBPCG_API lobpcg_status lobpcg_spmm_sym_f64(lobpcg_t h, const double *X, double *Y, int32_t k);

/*
 * W = K^{-1} R: the preconditioning step of Algorithm 1 (line 6), K the
 * block-diagonal matrix of shifted diagonal tiles of H (Section 3.3).  The
 * shift for column j is theta[j]; a shifted pivot t is guarded as
 * g(t) = sign(t) max(|t|, 1e-3 max(1, |theta_j|)).
 *   mode 0: K = I (W = R)
 *   mode 1: 1x1 tiles, w_ij = r_ij / g(h_ii - theta_j)
 *   mode 2: 64-row tiles solved exactly through their eigendecompositions
 *           (needs params.precond == 2 at create, else ERR_UNSUPPORTED)
 *   mode 3: the learned tile network (needs params.precond == 3 at create
 *           and weights from lobpcg_precond_train or lobpcg_mlp_set_params);
 *           k <= params.k.  A tile column whose correction is not finite
 *           keeps its mode-1 value; a correction longer (over the tile) than
 *           the mode-1 value is scaled down to that length.
 *   mode 4: params.fom_steps iterations of the Full Orthogonalization Method
 *           (Section 3.3) on (H_T - theta_j I) w_T = r_T for every diagonal
 *           tile T and column j, from w = 0: Arnoldi basis of
 *           K_s(H_T - theta_j I, r_T), then the Galerkin solve of the small
 *           Hessenberg system (Gaussian elimination with partial pivoting,
 *           pivots guarded by g).  The Krylov space of a column stops growing when
 *           the new basis direction has norm <= 1e-6 of (H_T - theta_j I) v
 *           (an invariant subspace).  Tiles: params.fom_tile_ptr (else 64
 *           rows).  Needs params.precond == 4 at create; k <= params.k when
 *           a tile is longer than 64 rows (its scratch is sized at create).
 *   R, W  : float32 n x k row-major, device (may be the same buffer)
 *   theta : float64[k], device
 */
LOBPCG_API lobpcg_status lobpcg_precond_apply(lobpcg_t h, const float *R, const double *theta, float *W,
                                              int32_t k, int32_t mode);

/*
 * Rayleigh-Ritz on the subspace spanned by the m columns of S (eq. rreig):
 * G = S^T (H S), O = S^T S (FP64 accumulation), then the k leftmost
 * eigenpairs of the pencil G C = O C D.  Cholesky of O first; if O is not
 * numerically positive definite, the eigendecomposition of O with
 * directions below 1e-12 of its largest eigenvalue dropped.
 *   S, HS : float32 n x m row-major, device (HS = H S, e.g. from spmm_sym)
 *   m     : 1..96;  k: 1..m
 *   C     : float64 m x k row-major, device;  theta: float64[k], device
 * Returns ERR_BREAKDOWN if fewer than k directions remain.
 */
LOBPCG_API lobpcg_status lobpcg_rayleigh_ritz(lobpcg_t h, const float *S, const float *HS, int32_t m, int32_t k,
                                              double *C, double *theta);

/*
 * lobpcg_rayleigh_ritz with no allocation.  The paper has no counterpart: it
 * is the same computation as lobpcg_rayleigh_ritz (same arguments, results
 * and errors) for callers that must not let a library call allocate (a loop
 * that reserved all device memory up front, a hard memory budget, or a loop
 * where an allocator call could block on other device work).  Its G and O
 * workspaces live in one statically sized device array of the library
 * (147,472 bytes per device: m <= 96; a larger m gives ERR_ARG with the
 * sizes in lobpcg_last_error).  The call clears G and O itself; nothing has
 * to be zero beforehand.
 *   - The array's device address is looked up once per device, on that
 *     device's first call; make that first call before any stream capture
 *     and with the handle's device current.
 *   - The array is shared by all calls on a device: calls that overlap in
 *     time (other streams, threads or handles) race on it and their results
 *     are undefined.  After return it keeps the last call's contents.
 *   - Synchronises the handle's stream (to read the breakdown status).
 */
LOBPCG_API lobpcg_status lobpcg_rayleigh_ritz_noalloc(lobpcg_t h, const float *S, const float *HS, int32_t m,
                                                      int32_t k, double *C, double *theta);

/*
 * The k leftmost eigenpairs of H by block LOBPCG (Algorithm 1), with the
 * preconditioner, tolerance and limits of the create parameters.  Only one
 * SpMM (H W) per iteration: HX and HP follow the recurrences of eqs.
 * upd1-upd2.  The iteration runs with float32 vectors; when its residual
 * stalls above tol (float32 rounding) and params.polish_fp64 is set, it
 * continues with float64 vectors.  Convergence is confirmed with an explicit
 * SpMM.
 *   X     : float32 n x k row-major; in: initial guess X0, out: Ritz vectors
 *           (device or host pointer; host memory is copied in and out)
 *   evals : host float64[nev], Ritz values ascending
 *   resid : host float64[nev], relative residual norms (params.resid_mode)
 *   st    : host stats (may be NULL)
 * Returns OK, ERR_NOT_CONVERGED (outputs still written), ERR_BREAKDOWN,
 * ERR_NONFINITE, ERR_CUDA.  Synchronises the stream.
 */
LOBPCG_API lobpcg_status lobpcg_solve(lobpcg_t h, float *X, double *evals, double *resid, lobpcg_stats *st);

/*
 * The k leftmost eigenpairs of H by block Davidson on the same SpMM,
 * preconditioner (params.precond), tolerance and limits: the paper notes
 * (Section 1) that its techniques carry over to other block eigensolvers.
 * Each iteration takes the k leftmost Ritz pairs of (V^T H V, V^T V) on the
 * orthonormal basis V, and, unless the nev leftmost have converged, appends
 * the preconditioned residuals orthonormalised against V (one SpMM per
 * iteration); when V holds max_blocks blocks it restarts from the k Ritz
 * vectors.  float32 vectors; when the residual stalls above tol and
 * params.polish_fp64 is set, the same iteration continues in float64 (with
 * the float64 SpMM).  Convergence is confirmed with an explicit SpMM.
 *   X          : as lobpcg_solve (in: X0, out: Ritz vectors; device or host)
 *   max_blocks : basis limit in blocks of k columns, 2 .. min(6, 96 / k)
 *   evals, resid, stats : as lobpcg_solve
 * The first call allocates 2 max_blocks blocks of n x k float32 (and of
 * float64 with polish_fp64) for the life of the handle; a later call may not
 * ask for more blocks (ERR_ARG).  Errors as lobpcg_solve.
 */
LOBPCG_API lobpcg_status lobpcg_davidson(lobpcg_t h, float *X, int32_t max_blocks, double *evals, double *resid,
                                         lobpcg_stats *stats);

/*
 * Run exactly `steps` float32 LOBPCG iterations (Algorithm 1, lines 6-12,
 * without the exit test; the residual norms are still formed and read back
 * each iteration as in lobpcg_solve).  X0 (n x k float32, device or host)
 * starts a new run from X0; X0 == NULL continues the previous run on this
 * handle.  theta (host float64[k], may be NULL) receives the current Ritz
 * values.  For benchmarking one iteration of the method.
 */
LOBPCG_API lobpcg_status lobpcg_iterate(lobpcg_t h, const float *X0, int32_t steps, double *theta,
                                        lobpcg_stats *st);

/* The last solve's Ritz vectors in float64 (n x k row-major, device or host). */
LOBPCG_API lobpcg_status lobpcg_get_x_f64(lobpcg_t h, double *X);

/*
 * Learned tile preconditioner (mode 3).  The paper has no counterpart: its K
 * (Section 3.3) solves each shifted diagonal tile by a few FOM iterations;
 * here one network, shared by every 64-row diagonal tile T, corrects the
 * mode-1 (diagonal) solve.  It maps
 *   x = [ r_T / s , (d_T - theta_j) / g , theta_j / g ]   (129 inputs)
 * through h = relu(W1 x + b1) (256) to y = W2 h + b2 (64) and returns
 * w_T = D^{-1} r_T + (s / g) y, D^{-1} r_T the mode-1 result, with
 * s = ||r_T||_2 (a tile with s = 0 gives w_T = 0), d_T the tile's diagonal
 * and g = ||H||_G (Gershgorin bound, lobpcg_info).
 * A ragged last tile is zero-padded.  Products run on the tensor cores with
 * bfloat16 operands (rounded from float32 master weights) and float32
 * accumulation.  All entry points below need params.precond == 3 at create
 * (ERR_UNSUPPORTED otherwise).
 *
 * Parameter vector (float32, LOBPCG_MLP_NPARAM entries, row-major blocks):
 *   W1 [256][129] | b1 [256] | W2 [64][256] | b2 [64]
 */
#define LOBPCG_MLP_NPARAM 49728

/* Load the weights (host or device pointer, `count` must equal
 * LOBPCG_MLP_NPARAM); resets the Adam state.  Synchronises the stream. */
LOBPCG_API lobpcg_status lobpcg_mlp_set_params(lobpcg_t h, const float *params, int64_t count);

/* Copy out the weights (which = 0) or the gradients of the last
 * lobpcg_mlp_grad / training batch (which = 1), same layout, host or device
 * pointer.  Synchronises the stream. */
LOBPCG_API lobpcg_status lobpcg_mlp_get_params(lobpcg_t h, float *out, int64_t count, int32_t which);

/* Forward pass on B input rows: Xin float32 B x 129 row-major, Y float32
 * B x 64 row-major, both device.  B >= 1.  Device scratch is taken from the
 * stream-ordered pool and returned before the call ends. */
LOBPCG_API lobpcg_status lobpcg_mlp_forward(lobpcg_t h, const float *Xin, int64_t B, float *Y);

/* Mean squared error L = sum (Y - T)^2 / (64 B) of the forward pass on Xin
 * against targets T (float32 B x 64, device), and its gradients with respect
 * to every weight (kept on the handle; read them with lobpcg_mlp_get_params
 * which = 1).  loss: host double (may be NULL).  Synchronises the stream. */
LOBPCG_API lobpcg_status lobpcg_mlp_grad(lobpcg_t h, const float *Xin, const float *T, int64_t B, double *loss);

/* One Adam step (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8, bias
 * corrected by the handle's step count) of the weights along the held
 * gradients, learning rate lr > 0. */
LOBPCG_API lobpcg_status lobpcg_mlp_adam(lobpcg_t h, float lr);

/*
 * Train the network on pairs the solver itself produces.  (1) Run
 * harvest_iters float32 LOBPCG iterations from X0 with the exact block-Jacobi
 * tile solves; in each, every (tile, column) pair is kept with probability
 * about n_pairs / (harvest_iters * tiles * k) (seeded by params.seed) and
 * stored as (x, t = clip(g (y_T - D^{-1} r_T) / s, +-1e3)), y_T the exact
 * shifted solve.  (2) If no weights were set, draw initial weights from
 * params.seed: W1 He-normal, b1, W2 and b2 zero (so that the untrained form
 * is the diagonal one).  (3) The last tenth of the pairs is held out; the
 * rest is visited `epochs` times with mean-squared-error Adam steps
 * (learning rate lr) over batches of up to 4096 pairs in a permuted order,
 * and the weights with the lowest held-out loss (before training or after an
 * epoch) are kept.
 *   X0        : float32 n x k (device or host), the solve's initial guess
 *   n_pairs   : capacity of the pair buffer (>= 4096); 772 bytes each
 *   loss_hist : host double[epochs + 1], held-out mean squared error before
 *               training and after each epoch (may be NULL)
 *   pairs_used: host (may be NULL), pairs actually harvested (<= n_pairs)
 * The pair buffer is freed before return.  Returns ERR_ARG when fewer than
 * 4096 pairs were harvested.  Synchronises the stream.
 */
LOBPCG_API lobpcg_status lobpcg_precond_train(lobpcg_t h, int32_t harvest_iters, int64_t n_pairs, int32_t epochs,
                                              const float *X0, float lr, double *loss_hist, int64_t *pairs_used);

#ifdef __cplusplus
}
#endif

#endif /* LOBPCG_H */
