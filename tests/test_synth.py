"""The seeded input generator: determinism and the stated structure."""
import os
import subprocess
import sys

import numpy as np

import synth


def test_deterministic_and_structure():
    A = synth.tile_matrix(2003, 100, seed=7)
    B = synth.tile_matrix(2003, 100, seed=7)
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col, B.col) and np.array_equal(A.val, B.val)
    C = synth.tile_matrix(2003, 100, seed=8)
    assert not np.array_equal(A.col, C.col)
    n = A.n
    assert A.row_ptr[0] == 0 and np.all(np.diff(A.row_ptr) >= 1)
    for i in range(n):
        c = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and c[-1] == i and c[0] >= 0
    diag = A.val[A.row_ptr[1:] - 1]
    assert diag.min() >= 0 and diag.max() < 200
    assert abs(A.nnz / n - 100) < 10


def test_thread_count_independent():
    code = ("import synth, numpy as np; A = synth.tile_matrix(5000, 60, seed=3);"
            "print(int(A.col.sum()), repr(float(A.val.sum())))")
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t, PYTHONPATH=os.path.dirname(os.path.dirname(__file__)))
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env).strip())
    assert outs[0] == outs[1]


def test_initial_guess():
    A = synth.tile_matrix(500, 30, seed=2)
    X = synth.initial_guess(A, 4, seed=9)
    d = A.val[A.row_ptr[1:] - 1]
    top = np.argsort(d, kind="stable")[:4]
    assert np.array_equal(np.argmax(np.abs(X), axis=0), top)
    assert np.all(np.abs(X[top, range(4)] - 1) < 1e-4)
