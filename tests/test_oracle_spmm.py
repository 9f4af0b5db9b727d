"""Pins for the oracle's symmetric SpMM (form (i): Algorithm 2 plus its
transposed loop; form (ii): full-storage expansion).  Each pin is
independent of the oracle's own code: hand-worked values, brute-force dense
products built here, identities of the mathematics."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_spmm_golden(name):
    ent, xs, ys = [], {}, {}
    n = k = None
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "n":
            n = int(line[1])
        elif line[0] == "k":
            k = int(line[1])
        elif line[0] == "entry":
            ent.append((int(line[1]), int(line[2]), float(line[3])))
        elif line[0] == "x":
            xs[int(line[1])] = [float(v) for v in line[2:]]
        elif line[0] == "y":
            ys[int(line[1])] = [float(v) for v in line[2:]]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    for i, _, _ in ent:
        row_ptr[i + 1] += 1
    row_ptr = np.cumsum(row_ptr)
    A = synth.CSR(n=n, row_ptr=row_ptr, col=np.array([e[1] for e in ent], dtype=np.int32),
                  val=np.array([e[2] for e in ent]))
    X = np.array([xs[i] for i in range(n)])
    Y = np.array([ys[i] for i in range(n)])
    return A, X, Y


def dense_by_hand(A):
    """Dense H from the triangle, written independently of the oracle."""
    H = np.zeros((A.n, A.n))
    for i in range(A.n):
        for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = int(A.col[e])
            H[i, j] = A.val[e]
            H[j, i] = A.val[e]
    return H


def random_lower(n, density, seed, fp32=False, empty_rows=()):
    rng = np.random.default_rng(seed)
    a = np.zeros((n, n))
    mask = rng.random((n, n)) < density
    a[mask] = rng.standard_normal(mask.sum())
    a = np.tril(a)
    a = a + np.tril(a, -1).T
    np.fill_diagonal(a, rng.uniform(0, 10, n))
    for i in empty_rows:
        a[i, :] = 0.0
        a[:, i] = 0.0
    A = synth.csr_from_dense_lower(a, fp32=fp32)
    if empty_rows:   # drop the kept diagonal of empty rows too
        keep = np.ones(A.nnz, bool)
        for i in empty_rows:
            keep[A.row_ptr[i + 1] - 1] = False
        rows = np.repeat(np.arange(n), np.diff(A.row_ptr))[keep]
        rp = np.zeros(n + 1, dtype=np.int64)
        np.add.at(rp, rows + 1, 1)
        A = synth.CSR(n=n, row_ptr=np.cumsum(rp), col=A.col[keep], val=A.val[keep])
    return A


def test_golden_3x3():
    A, X, Y = read_spmm_golden("spmm_3x3.txt")
    assert np.array_equal(oracle.spmm_tri(A, X), Y)
    assert np.array_equal(oracle.spmm_full(A, X), Y)
    assert np.array_equal(oracle.spmm_rows(A, X, [0, 1, 2]), Y)


@pytest.mark.parametrize("n,npr,k", [(1000, 40, 1), (2003, 60, 5), (3000, 100, 8)])
def test_tile_matrix_brute_force(n, npr, k):
    A = synth.tile_matrix(n, npr, seed=11 + n)
    X = synth.normal_block(n, k, seed=5)
    H = dense_by_hand(A)
    Yd = H @ X
    scale = np.abs(H) @ np.abs(X)
    for Y in (oracle.spmm_tri(A, X), oracle.spmm_full(A, X)):
        assert np.all(np.abs(Y - Yd) <= 1e-13 * scale + 1e-300)


def test_forms_agree_fp32_values():
    A = synth.tile_matrix(5000, 80, seed=3, fp32=True)
    X = synth.normal_block(5000, 16, seed=9)
    Y1 = oracle.spmm_tri(A, X)
    Y2 = oracle.spmm_full(A, X)
    assert np.max(np.abs(Y1 - Y2)) <= 1e-14 * np.max(np.abs(Y1))
    rows = [0, 1, 17, 2500, 4999]
    assert np.allclose(oracle.spmm_rows(A, X, rows), Y1[rows], rtol=0, atol=1e-12 * np.abs(Y1).max())


def test_random_sparsity_and_empty_rows():
    A = random_lower(300, 0.05, seed=4, empty_rows=(0, 7, 299))
    X = np.random.default_rng(1).standard_normal((300, 3))
    H = dense_by_hand(A)
    for Y in (oracle.spmm_tri(A, X), oracle.spmm_full(A, X)):
        assert np.allclose(Y, H @ X, rtol=1e-13, atol=1e-13)
        assert np.all(Y[[0, 7, 299]] == 0.0)


def test_diagonal_only_exact():
    n, k = 257, 4
    d = np.linspace(-3, 7, n)
    A = synth.CSR(n=n, row_ptr=np.arange(n + 1, dtype=np.int64),
                  col=np.arange(n, dtype=np.int32), val=d.copy())
    X = np.random.default_rng(2).standard_normal((n, k))
    assert np.array_equal(oracle.spmm_tri(A, X), d[:, None] * X)
    assert np.array_equal(oracle.spmm_full(A, X), d[:, None] * X)


def test_symmetry_identity():
    """X2^T (H X1) = (H X2)^T X1 for symmetric H."""
    A = synth.tile_matrix(4000, 60, seed=8)
    X1 = synth.normal_block(4000, 6, seed=1)
    X2 = synth.normal_block(4000, 6, seed=2)
    a = X2.T @ oracle.spmm_tri(A, X1)
    b = oracle.spmm_tri(A, X2).T @ X1
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))


def test_dense_tile_brute_force():
    """A single dense 16x16 symmetric tile against a loop-by-loop product."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((16, 16))
    a = a + a.T
    A = synth.csr_from_dense_lower(a)
    X = rng.standard_normal((16, 3))
    Y = np.zeros((16, 3))
    for i in range(16):
        for j in range(16):
            for q in range(3):
                Y[i, q] += a[i, j] * X[j, q]
    assert np.allclose(oracle.spmm_tri(A, X), Y, rtol=1e-14, atol=1e-13)


def test_planted_mistake_is_caught():
    """Applying the diagonal twice (a plausible slip with half storage) fails
    the brute-force pin: the pins are sharp enough to see it."""
    A = synth.tile_matrix(500, 40, seed=2)
    X = synth.normal_block(500, 2, seed=3)
    H = dense_by_hand(A)
    Y_bad = oracle.spmm_tri(A, X) + oracle.diagonal(A)[:, None] * X
    assert not np.allclose(Y_bad, H @ X, rtol=1e-10, atol=1e-10)


def test_gershgorin_and_diag():
    A = synth.tile_matrix(700, 30, seed=6)
    H = dense_by_hand(A)
    assert np.isclose(oracle.gershgorin(A), np.abs(H).sum(1).max(), rtol=1e-14)
    assert np.array_equal(oracle.diagonal(A), np.diag(H))
    B = oracle.dense_block(A, 64, 64)
    assert np.array_equal(B, H[64:128, 64:128])
    Bt = oracle.dense_block(A, 640, 64)          # ragged tail: rows past n stay zero
    assert np.array_equal(Bt[:60, :60], H[640:700, 640:700]) and not Bt[60:].any()
