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
    int32_t precond;     /* 0 none, 1 diagonal, 2 block-Jacobi (64-row tiles), 3 learned MLP */
    int32_t resid_mode;  /* 0: ||r||/(max(|theta|,1e-12||H||_G)||x||), 1: ||r||/(||H||_G||x||) */
    int32_t polish_fp64; /* 1: finish with FP64 vectors once FP32 stagnates */
    int32_t reserved;
    uint64_t seed;
} lobpcg_params;

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
    int32_t warps;           /* warps the SpMM partition is cut for */
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

/* Release every resource of the handle (NULL is accepted). */
LOBPCG_API lobpcg_status lobpcg_destroy(lobpcg_t h);

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

#ifdef __cplusplus
}
#endif

#endif /* LOBPCG_H */
