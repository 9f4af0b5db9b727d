"""Pins for the oracle LOBPCG (Algorithm 1) and its dense steps, against a
library eigensolver, closed-form spectra and the invariants of the method."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from oracle import lobpcg as olb
from oracle.precond import apply_bjacobi, apply_diag, guard, tile_eigs, tile_solve_lu


def laplacian_csr(n):
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        if i > 0:
            cols.append(i - 1)
            vals.append(-1.0)
        cols.append(i)
        vals.append(2.0)
        rp[i + 1] = len(cols)
    return synth.CSR(n=n, row_ptr=rp, col=np.array(cols, dtype=np.int32), val=np.array(vals))


@pytest.mark.parametrize("n,npr,k,nev,pc", [(256, 40, 8, 5, "diag"), (512, 60, 8, 5, "bjacobi"),
                                            (300, 30, 6, 3, "none"), (200, 50, 4, 4, "diag")])
def test_lobpcg_vs_library_eigvalsh(n, npr, k, nev, pc):
    A = synth.tile_matrix(n, npr, seed=n)
    H = oracle.to_dense(A)
    lam = np.linalg.eigvalsh(H)
    X0 = synth.initial_guess(A, k, seed=n + 1000)
    r = olb.lobpcg(A, X0, nev, tol=1e-10, maxiter=2000, precond=pc)
    assert r.converged
    assert np.max(np.abs(r.evals - lam[:nev]) / np.maximum(np.abs(lam[:nev]), 1e-3)) < 1e-10
    # residual of the returned pairs, recomputed by brute force
    R = H @ r.X - r.X * r.evals
    rho = np.linalg.norm(R, axis=0) / (np.abs(r.evals) * np.linalg.norm(r.X, axis=0))
    assert np.all(rho <= 1e-10 * 1.01)
    assert np.max(np.abs(r.X.T @ r.X - np.eye(nev))) < 1e-10


def test_lobpcg_laplacian_closed_form():
    n, k, nev = 200, 6, 4
    A = laplacian_csr(n)
    X0 = synth.normal_block(n, k, seed=3)
    r = olb.lobpcg(A, X0, nev, tol=1e-9, maxiter=3000, precond="diag")
    exact = np.array([2 - 2 * math.cos(j * math.pi / (n + 1)) for j in range(1, nev + 1)])
    assert r.converged
    assert np.max(np.abs(r.evals - exact) / exact) < 1e-9


def test_dense_lowest_closed_form_and_jacobi():
    """The dense reference (the plain definition: nev smallest eigenvalues of
    H) against the 1-D Laplacian closed form and the Jacobi oracle."""
    n = 60
    w, V = olb.dense_lowest(laplacian_csr(n), 5)
    exact = np.array([2 - 2 * math.cos(j * math.pi / (n + 1)) for j in range(1, 6)])
    assert np.max(np.abs(w - exact)) < 1e-13
    A = synth.tile_matrix(150, 40, seed=21)
    w, V = olb.dense_lowest(A, 7)
    wj, _ = oracle.jacobi_eig(oracle.to_dense(A))
    assert np.max(np.abs(w - wj[:7])) < 1e-12 * np.abs(wj).max()
    H = oracle.to_dense(A)
    assert np.max(np.abs(H @ V - V * w)) < 1e-11 * np.abs(wj).max()


@pytest.mark.parametrize("k,nev,pc", [(12, 6, "diag"), (20, 10, "diag"), (16, 8, "bjacobi")])
def test_lobpcg_explicit_products_vs_dense(k, nev, pc):
    """The explicit-product form (HX, HP by SpMM each iteration) reaches the
    dense eigenvalues at tol 1e-10 for block sizes up to 20."""
    A = synth.tile_matrix(1500, 50, seed=23)
    lam, _ = olb.dense_lowest(A, nev)
    X0 = synth.initial_guess(A, k, seed=1023)
    r = olb.lobpcg(A, X0, nev, tol=1e-10, maxiter=500, precond=pc, explicit=True)
    assert r.converged
    assert np.max(np.abs(r.evals - lam) / np.maximum(np.abs(lam), 1e-3)) < 1e-10
    H = oracle.to_dense(A)
    R = H @ r.X - r.X * r.evals
    rho = np.linalg.norm(R, axis=0) / (np.abs(r.evals) * np.linalg.norm(r.X, axis=0))
    assert np.all(rho <= 1e-10 * 1.01)


def test_ritz_values_monotone():
    """span(S_i) contains span(X_i), so each Ritz value can only decrease
    (Courant-Fischer), up to rounding."""
    A = synth.tile_matrix(400, 40, seed=9)
    X0 = synth.normal_block(400, 6, seed=4)
    r = olb.lobpcg(A, X0, 4, tol=1e-9, maxiter=500, precond="diag")
    th = np.array(r.theta_hist)
    assert np.all(np.diff(th, axis=0) <= 1e-10 * np.abs(th).max())


def test_rayleigh_ritz_vs_library_generalised():
    rng = np.random.default_rng(1)
    S = rng.standard_normal((100, 9))
    M = rng.standard_normal((100, 100))
    Hm = M + M.T
    G, O = S.T @ Hm @ S, S.T @ S
    th, C = olb.rayleigh_ritz(G, O, 4)
    w = scipy.linalg.eigh(G, O, eigvals_only=True)
    assert np.max(np.abs(th - w[:4])) < 1e-10 * np.abs(w).max()
    assert np.max(np.abs(C.T @ O @ C - np.eye(4))) < 1e-10
    assert np.max(np.abs(G @ C - O @ C * th)) < 1e-9 * np.abs(G).max()
    with pytest.raises(olb.RRFailure):
        olb.rayleigh_ritz(G, np.diag([1.0] * 8 + [-1.0]), 4)


def test_cholqr_and_svqb():
    rng = np.random.default_rng(2)
    X = np.linalg.qr(rng.standard_normal((500, 4)))[0]
    W = rng.standard_normal((500, 5))
    Q = olb.orthonormalize_w(W, X)
    assert np.max(np.abs(Q.T @ Q - np.eye(5))) < 1e-13
    assert np.max(np.abs(X.T @ Q)) < 1e-13
    # span is preserved modulo X
    Pw = W - X @ (X.T @ W)
    assert np.linalg.matrix_rank(np.hstack([Q, Pw]), tol=1e-9) == 5
    # a dependent column is dropped by SVQB
    Wd = np.hstack([W[:, :3], W[:, :1] + W[:, 1:2]])
    Qd = olb.svqb(Wd)
    assert Qd.shape[1] == 3 and np.max(np.abs(Qd.T @ Qd - np.eye(3))) < 1e-8


def test_resid_norm_definitions():
    R = np.array([[3.0, 0.0], [4.0, 1e-20]])
    X = np.array([[1.0, 0.0], [0.0, 2.0]])
    th = np.array([-10.0, 0.0])
    rho0 = olb.resid_norms(R, X, th, normG=5.0, mode=0)
    assert rho0[0] == pytest.approx(0.5)
    assert rho0[1] == pytest.approx(1e-20 / (1e-12 * 5.0 * 2.0))
    rho1 = olb.resid_norms(R, X, th, normG=5.0, mode=1)
    assert rho1[0] == pytest.approx(1.0)


# ---------------------------------------------------------------- preconditioners

def test_guard():
    th = np.array([0.0, 5.0, -2000.0])
    assert np.array_equal(guard(np.array([0.0, 0.0, 0.0]), th), [1e-3, 5e-3, 2.0])
    assert np.array_equal(guard(np.array([-1e-9, 3.0, -7.0]), th), [-1e-3, 3.0, -7.0])


def test_diag_precond_plain_division():
    rng = np.random.default_rng(3)
    d = rng.uniform(1, 10, 50)
    R = rng.standard_normal((50, 3))
    th = np.array([-1.0, 0.0, 0.5])
    assert np.array_equal(apply_diag(d, R, th), R / (d[:, None] - th[None, :]))


def test_bjacobi_equals_lu_solve_and_diag_case():
    A = synth.tile_matrix(150, 40, seed=12)          # tiles of 64, 64, 22 rows
    R = synth.normal_block(150, 3, seed=2)
    th = np.array([-100.0, -50.0, -75.0])           # below every tile spectrum: no guard
    W = apply_bjacobi(A, R, th)
    for t in range(3):
        m = min(64, 150 - 64 * t)
        for j in range(3):
            y = tile_solve_lu(A, t, R[64 * t:64 * t + m, j], th[j])
            assert np.max(np.abs(W[64 * t:64 * t + m, j] - y)) < 1e-12 * np.abs(y).max()
    # a diagonal matrix: block-Jacobi reduces to the diagonal preconditioner
    n = 130
    d = np.linspace(1, 9, n)
    D = synth.CSR(n=n, row_ptr=np.arange(n + 1, dtype=np.int64), col=np.arange(n, dtype=np.int32), val=d)
    Rd = synth.normal_block(n, 2, seed=1)
    thd = np.array([0.25, -3.0])
    assert np.allclose(apply_bjacobi(D, Rd, thd), apply_diag(d, Rd, thd), rtol=1e-14, atol=0)
    lam, Q = tile_eigs(D)
    assert lam.shape == (3, 64) and np.allclose(lam[2, :2], d[128:])
