"""Pins for the oracle's dense kernels: cyclic Jacobi against closed-form
spectra, Cholesky and LU against their defining identities."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def laplacian(n):
    return 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)


def test_jacobi_golden_laplacian():
    vals = {}
    for line in open(os.path.join(GOLDEN, "laplacian_1d.txt")):
        t = line.split("#")[0].split()
        if t and t[0] == "n":
            n = int(t[1])
        elif t and t[0] == "lambda":
            vals[int(t[1])] = float(t[2])
    w, V = oracle.jacobi_eig(laplacian(n))
    for j, lam in vals.items():
        assert abs(w[j - 1] - lam) < 1e-11


@pytest.mark.parametrize("n", [1, 2, 7, 33, 64, 120])
def test_jacobi_laplacian_closed_form(n):
    w, V = oracle.jacobi_eig(laplacian(n))
    exact = np.array([2 - 2 * math.cos(j * math.pi / (n + 1)) for j in range(1, n + 1)])
    assert np.max(np.abs(w - exact)) < 1e-13 * max(1, n)
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-13 * max(1, n)
    assert np.max(np.abs(laplacian(n) @ V - V * w)) < 1e-12 * max(1, n)


def test_jacobi_diagonal_sorted():
    d = np.array([3.0, -1.0, 2.5, 0.0, -7.25, 11.0])
    w, V = oracle.jacobi_eig(np.diag(d))
    assert np.array_equal(w, np.sort(d))
    assert np.array_equal(np.abs(V), np.eye(6)[:, np.argsort(d)])


def secular_roots(d, u, rho):
    """Eigenvalues of diag(d) + rho u u^T (rho > 0, distinct d): entries with
    u_i = 0 are eigenvalues d_i; the rest are the roots of
    1 + rho sum u_i^2 / (d_i - lam), one in each interval (d_(i), d_(i+1))
    and the last in (d_max, d_max + rho ||u||^2), found by bisection."""
    nz = u != 0
    roots = list(d[~nz])
    dd = np.sort(d[nz])
    uu = u[nz][np.argsort(d[nz])]
    f = lambda lam: 1.0 + rho * np.sum(uu ** 2 / (dd - lam))
    uppers = list(dd[1:]) + [dd[-1] + rho * np.sum(uu ** 2)]
    for lo, hi in zip(dd, uppers):
        a, b = lo, hi
        for _ in range(200):
            m = 0.5 * (a + b)
            if m == a or m == b:
                break
            if f(m) > 0:     # f increases across each interval from -inf to +inf
                b = m
            else:
                a = m
        roots.append(0.5 * (a + b))
    return np.sort(np.array(roots))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_jacobi_diag_plus_rank_one(seed):
    rng = np.random.default_rng(seed)
    n = 40
    d = np.sort(rng.uniform(-5, 5, n))
    u = rng.standard_normal(n)
    u[rng.random(n) < 0.3] = 0.0            # sparse u: some d_i stay eigenvalues
    rho = 0.7
    w, _ = oracle.jacobi_eig(np.diag(d) + rho * np.outer(u, u))
    assert np.max(np.abs(w - secular_roots(d, u, rho))) < 1e-12 * max(1.0, np.abs(d).max())


def test_jacobi_random_reconstruct():
    rng = np.random.default_rng(5)
    M = rng.standard_normal((60, 60))
    M = M + M.T
    w, V = oracle.jacobi_eig(M)
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(V @ np.diag(w) @ V.T - M)) < 1e-12 * np.abs(M).max()
    assert np.max(np.abs(V.T @ V - np.eye(60))) < 1e-13


def test_cholesky_identity_and_failure():
    rng = np.random.default_rng(6)
    B = rng.standard_normal((30, 12))
    M = B.T @ B
    L = oracle.cholesky(M)
    assert np.allclose(L, np.tril(L))
    assert np.max(np.abs(L @ L.T - M)) < 1e-12 * np.abs(M).max()
    assert oracle.cholesky(np.diag([1.0, -1.0, 2.0])) is None
    assert oracle.cholesky(np.zeros((3, 3))) is None


def test_lu_solve_known_solution():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((50, 50))
    Y = rng.standard_normal((50, 4))
    B = M @ Y
    assert np.max(np.abs(oracle.lu_solve(M, B) - Y)) < 1e-10
    # a matrix that needs pivoting (zero leading entry)
    P = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.allclose(oracle.lu_solve(P, np.array([[2.0], [3.0]])), [[3.0], [2.0]])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.lu_solve(np.zeros((2, 2)), np.ones((2, 1)))
