"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

Holds no eigensolver arithmetic: only random draws and their layout (see
``gen.c`` for the matrix recipe).  The matrices stand in for the nuclear CI
Hamiltonians of the paper (Section 5.1, Table "tbl:dataset"), which are not
available; the structure follows Section 3.3 (block -> tile -> element, every
diagonal tile and diagonal element nonzero).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``gen.c`` into ``libsynth.so`` (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-std=c11", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i64, u64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
        lib.synth_plan_create.restype = vp
        lib.synth_plan_create.argtypes = [i64, dbl, u64, dbl, dbl]
        lib.synth_plan_nnz.restype = i64
        lib.synth_plan_nnz.argtypes = [vp]
        lib.synth_plan_row_ptr.argtypes = [vp, vp]
        lib.synth_plan_fill.argtypes = [vp, vp, vp, ctypes.c_int]
        lib.synth_plan_destroy.argtypes = [vp]
        lib.synth_normal_block.argtypes = [i64, i32, u64, vp, ctypes.c_int]
        lib.synth_uniform.argtypes = [i64, u64, u64, dbl, dbl, vp]
        lib.synth_normals.argtypes = [i64, u64, u64, vp]
        lib.synth_u64.argtypes = [i64, u64, u64, vp]
        _lib = lib
    return _lib


@dataclass
class CSR:
    """Lower triangle (incl. diagonal) of a symmetric matrix, CSR, sorted columns."""
    n: int
    row_ptr: np.ndarray   # int64[n+1]
    col: np.ndarray       # int32[nnz]
    val: np.ndarray       # float64 or float32 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def tile_matrix(n: int, nnz_per_row: float, seed: int, fp32: bool = False,
                scatter_frac: float = 0.10, window_frac: float = 0.05, alloc=None) -> CSR:
    """Seeded tile-clustered lower-triangle CSR (see ``gen.c``).

    ``alloc(shape, dtype)`` may supply the output arrays (e.g. pinned host
    memory); it defaults to ``np.empty``.
    """
    lib = _load()
    h = lib.synth_plan_create(int(n), float(nnz_per_row), int(seed) & (2**64 - 1),
                              float(scatter_frac), float(window_frac))
    if not h:
        raise ValueError("synth_plan_create failed")
    try:
        alloc = alloc or (lambda shape, dt: np.empty(shape, dtype=dt))
        nnz = lib.synth_plan_nnz(h)
        row_ptr = alloc((n + 1,), np.int64)
        col = alloc((nnz,), np.int32)
        val = alloc((nnz,), np.float32 if fp32 else np.float64)
        lib.synth_plan_row_ptr(h, row_ptr.ctypes.data)
        lib.synth_plan_fill(h, col.ctypes.data, val.ctypes.data, 1 if fp32 else 0)
    finally:
        lib.synth_plan_destroy(h)
    return CSR(n=int(n), row_ptr=row_ptr, col=col, val=val)


def normal_block(n: int, k: int, seed: int, fp32: bool = False, out: np.ndarray | None = None) -> np.ndarray:
    """n x k row-major block of N(0,1) draws (the initial guess X0)."""
    lib = _load()
    dt = np.float32 if fp32 else np.float64
    if out is None:
        out = np.empty((n, k), dtype=dt)
    assert out.dtype == dt and out.flags.c_contiguous and out.shape == (n, k)
    lib.synth_normal_block(int(n), int(k), int(seed) & (2**64 - 1), out.ctypes.data, 1 if fp32 else 0)
    return out


def uniform(m: int, seed: int, tag: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(m, dtype=np.float64)
    _load().synth_uniform(int(m), int(seed) & (2**64 - 1), int(tag), float(lo), float(hi), out.ctypes.data)
    return out


def normals(m: int, seed: int, tag: int) -> np.ndarray:
    out = np.empty(m, dtype=np.float64)
    _load().synth_normals(int(m), int(seed) & (2**64 - 1), int(tag), out.ctypes.data)
    return out


def u64(m: int, seed: int, tag: int) -> np.ndarray:
    out = np.empty(m, dtype=np.uint64)
    _load().synth_u64(int(m), int(seed) & (2**64 - 1), int(tag), out.ctypes.data)
    return out


def tile_partition(n: int, seed: int, median: float = 200.0, sigma: float = 1.0, max_size: int = 6000,
                   tag: int = 7) -> np.ndarray:
    """Row partition into diagonal tiles of varying size (int64 boundaries,
    0 .. n): sizes round(median * exp(sigma * z)), z ~ N(0,1) seeded, clipped
    to [1, max_size], the last tile cut at n.  Stands in for the paper's
    diagonal tiles, which run from 1 to ~6000 rows, mostly a few hundred
    (Section 4, diagonal tile size histogram)."""
    sizes = []
    total, drawn = 0, 0
    while total < n:
        z = normals(max(64, n // max(1, int(median)) + 64), seed, tag + drawn)
        drawn += 1
        for v in z:
            sz = int(min(max(round(median * float(np.exp(sigma * v))), 1), max_size))
            sz = min(sz, n - total)
            sizes.append(sz)
            total += sz
            if total >= n:
                break
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def csr_from_dense_lower(a: np.ndarray, fp32: bool = False) -> CSR:
    """Lower-triangle CSR of a dense symmetric matrix (explicit zeros dropped,
    diagonal always kept).  Used to build small hand-made test matrices."""
    n = a.shape[0]
    rows, cols, vals = [], [], []
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for i in range(n):
        js = [j for j in range(i + 1) if a[i, j] != 0.0 or j == i]
        row_ptr[i + 1] = row_ptr[i] + len(js)
        cols.extend(js)
        vals.extend(a[i, j] for j in js)
    return CSR(n=n, row_ptr=row_ptr, col=np.asarray(cols, dtype=np.int32),
               val=np.asarray(vals, dtype=np.float32 if fp32 else np.float64))


# Workload shapes (seeded synthetic stand-ins; seeds fixed per workload).
WORKLOADS = {
    "small_n20k": dict(n=20_000, nnz_per_row=100.0, k=8, nev=5, seed=1, fp32=False),
    "full_n2m": dict(n=2_000_000, nnz_per_row=400.0, k=16, nev=8, seed=2, fp32=True),
    "largest_n8m": dict(n=8_000_000, nnz_per_row=250.0, k=20, nev=10, seed=5, fp32=True),
    # same structure at a quarter of the rows: ~1.6 GB, still far larger than L2 (profiling captures)
    "profile_n500k": dict(n=500_000, nnz_per_row=400.0, k=16, nev=8, seed=3, fp32=True),
}
X0_SEED_OFFSET = 1000


def initial_guess(A: CSR, k: int, seed: int, noise: float = 1e-5, fp32: bool = False) -> np.ndarray:
    """Initial block X0 (n x k): unit vectors at the k smallest stored diagonal
    entries (ties broken by row index), plus ``noise`` times seeded N(0,1).

    The paper leaves X0 open (Algorithm 1 takes it as an input).  For these
    matrices, whose diagonal spans [0, 200] and dominates each row, a random
    X0 starts the Ritz values mid-spectrum and the shifted diagonal
    preconditioner then steers toward interior eigenvalues; starting on the
    smallest diagonal entries does not.
    """
    n = A.n
    # in a lower triangle with sorted columns a stored diagonal entry is the
    # last entry of its row
    d = np.zeros(n, dtype=np.float64)
    rows = np.nonzero(np.diff(A.row_ptr) > 0)[0]
    last = A.row_ptr[rows + 1] - 1
    hit = A.col[last].astype(np.int64) == rows
    d[rows[hit]] = A.val[last[hit]]
    order = np.lexsort((np.arange(n), d))[:k]
    X0 = normal_block(n, k, seed) * noise
    X0[order, np.arange(min(k, n))] += 1.0
    return X0.astype(np.float32) if fp32 else X0
