"""CPU FP64 oracle for the symmetric SpMM and block LOBPCG (arXiv 2109.00485).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2109_00485_gb300``) and never imports it.

Contents
  spmm.c    SpMM from the stored triangle, two independent forms (Algorithm 2
            plus its transposed loop; full-storage expansion), sampled rows,
            Gershgorin bound, diagonal and dense diagonal blocks.
  dense.c   cyclic Jacobi eigensolver, Cholesky, LU with partial pivoting.
  lobpcg.py Algorithm 1 with the HX/HP recurrences of eqs. (upd1)-(upd2),
            Cholesky-QR (Section 3.4) and the Rayleigh-Ritz pencil (rreig).
  precond.py the diagonal and block-Jacobi forms of K (Section 3.3).
  mlp.py    the learned tile preconditioner's network (not in the paper).

Parity status of each function is listed in its docstring; a function with
no independent pin says "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRCS = ["spmm.c", "dense.c"]
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, OpenMP, no FMA contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-std=c11", *srcs, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        vp, i64, i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        L.oracle_spmm_tri.argtypes = [i64, vp, vp, vp, c_int, vp, i32, vp]
        L.oracle_spmm_full.argtypes = [i64, vp, vp, vp, c_int, vp, i32, vp]
        L.oracle_spmm_full.restype = c_int
        L.oracle_spmm_rows.argtypes = [i64, vp, vp, vp, c_int, vp, i32, i64, vp, vp]
        L.oracle_gershgorin.argtypes = [i64, vp, vp, vp, c_int]
        L.oracle_gershgorin.restype = ctypes.c_double
        L.oracle_diag.argtypes = [i64, vp, vp, vp, c_int, vp]
        L.oracle_dense_block.argtypes = [i64, vp, vp, vp, c_int, i64, i32, vp]
        L.oracle_jacobi_eig.argtypes = [i32, vp, vp, vp, i32]
        L.oracle_jacobi_eig.restype = c_int
        L.oracle_cholesky.argtypes = [i32, vp, vp]
        L.oracle_cholesky.restype = c_int
        L.oracle_lu_solve.argtypes = [i32, vp, i32, vp]
        L.oracle_lu_solve.restype = c_int
        L.oracle_num_threads.restype = c_int
        _lib = L
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _csr_args(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val)
    if val.dtype not in (np.float32, np.float64):
        raise TypeError("values must be float32 or float64")
    return rp, col, val, 1 if val.dtype == np.float32 else 0


def spmm_tri(A, X: np.ndarray) -> np.ndarray:
    """Y = H X, form (i): Algorithm 2 over the triangle plus the separate
    transposed loop of Section 3.2/3.3.  Pinned by form (ii), brute-force dense
    products and the symmetry identity (tests/test_oracle_spmm.py)."""
    rp, col, val, f32 = _csr_args(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, k = X.shape
    Y = np.empty((n, k), dtype=np.float64)
    lib().oracle_spmm_tri(A.n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, f32,
                          X.ctypes.data, k, Y.ctypes.data)
    return Y


def spmm_full(A, X: np.ndarray) -> np.ndarray:
    """Y = H X, form (ii): expand to full symmetric CSR, one row loop."""
    rp, col, val, f32 = _csr_args(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, k = X.shape
    Y = np.empty((n, k), dtype=np.float64)
    if lib().oracle_spmm_full(A.n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, f32,
                              X.ctypes.data, k, Y.ctypes.data) != 0:
        raise MemoryError("oracle_spmm_full")
    return Y


def spmm_rows(A, X: np.ndarray, rows) -> np.ndarray:
    """Rows ``rows`` of H X, each from the definition (O(nnz) per row)."""
    rp, col, val, f32 = _csr_args(A)
    X = np.ascontiguousarray(X, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    k = X.shape[1]
    out = np.empty((rows.size, k), dtype=np.float64)
    lib().oracle_spmm_rows(A.n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, f32,
                           X.ctypes.data, k, rows.size, rows.ctypes.data, out.ctypes.data)
    return out


def gershgorin(A) -> float:
    rp, col, val, f32 = _csr_args(A)
    return float(lib().oracle_gershgorin(A.n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, f32))


def diagonal(A) -> np.ndarray:
    rp, col, val, f32 = _csr_args(A)
    d = np.empty(A.n, dtype=np.float64)
    lib().oracle_diag(A.n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, f32, d.ctypes.data)
    return d


def dense_block(A, r0: int, m: int) -> np.ndarray:
    """Dense symmetric H[r0:r0+m, r0:r0+m] (rows past n left zero)."""
    rp, col, val, f32 = _csr_args(A)
    B = np.empty((m, m), dtype=np.float64)
    lib().oracle_dense_block(A.n, rp.ctypes.data, col.ctypes.data, val.ctypes.data, f32,
                             int(r0), int(m), B.ctypes.data)
    return B


def to_dense(A) -> np.ndarray:
    """Full dense symmetric H (small matrices only)."""
    return dense_block(A, 0, A.n)


def jacobi_eig(M: np.ndarray, max_sweeps: int = 100):
    """Eigenpairs of the symmetric matrix M by cyclic Jacobi (Golub & Van
    Loan, Section 8.5).  Returns (w ascending, V).  Pinned by closed-form
    spectra (tests/test_oracle_dense.py)."""
    A = np.array(M, dtype=np.float64, order="C", copy=True)
    m = A.shape[0]
    w = np.empty(m)
    V = np.empty((m, m))
    if m == 0:
        return w, V
    if lib().oracle_jacobi_eig(m, A.ctypes.data, w.ctypes.data, V.ctypes.data, int(max_sweeps)) < 0:
        raise RuntimeError("Jacobi did not converge")
    return w, V


def cholesky(M: np.ndarray):
    """Lower Cholesky factor of M, or None if M is not positive definite."""
    A = np.ascontiguousarray(M, dtype=np.float64)
    m = A.shape[0]
    L = np.empty((m, m))
    if lib().oracle_cholesky(m, A.ctypes.data, L.ctypes.data) != 0:
        return None
    return L


def lu_solve(M: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve M Y = B by Gaussian elimination with partial pivoting."""
    A = np.array(M, dtype=np.float64, order="C", copy=True)
    Bc = np.array(B, dtype=np.float64, order="C", copy=True)
    if Bc.ndim == 1:
        Bc = Bc[:, None]
    m, r = Bc.shape
    if lib().oracle_lu_solve(m, A.ctypes.data, r, Bc.ctypes.data) != 0:
        raise np.linalg.LinAlgError("singular")
    return Bc.reshape(B.shape)
