"""Pins for the oracle block Davidson (the paper's SpMM and preconditioner
inside another block eigensolver): a library eigensolver, the whole-space
limit, the interlacing of Ritz values on nested subspaces, and a closed-form
spectrum."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle.davidson import davidson


@pytest.mark.parametrize("n,npr,k,nev,pc,blocks", [(256, 40, 8, 5, "diag", 4), (300, 30, 6, 3, "none", 6),
                                                   (256, 50, 8, 4, "bjacobi", 3), (200, 40, 4, 4, "fom", 5)])
def test_davidson_vs_library_eigvalsh(n, npr, k, nev, pc, blocks):
    A = synth.tile_matrix(n, npr, seed=n + 7)
    H = oracle.to_dense(A)
    lam = np.linalg.eigvalsh(H)
    X0 = synth.initial_guess(A, k, seed=n + 99)
    r = davidson(A, X0, nev, tol=1e-10, maxiter=3000, precond=pc, max_blocks=blocks)
    assert r.converged
    assert np.max(np.abs(r.evals - lam[:nev]) / np.maximum(np.abs(lam[:nev]), 1e-3)) < 1e-10
    R = H @ r.X - r.X * r.evals
    rho = np.linalg.norm(R, axis=0) / (np.abs(r.evals) * np.linalg.norm(r.X, axis=0))
    assert np.all(rho <= 1e-10 * 1.01)


def test_whole_space_gives_exact_eigenvalues():
    # n = 24, k = 4: after five extensions the basis spans all 24 dimensions,
    # so the sixth Rayleigh-Ritz step returns the exact 4 lowest eigenvalues
    A = synth.tile_matrix(24, 24, seed=3)
    lam = np.linalg.eigvalsh(oracle.to_dense(A))
    X0 = synth.normal_block(24, 4, seed=4)
    r = davidson(A, X0, 4, tol=1e-300, maxiter=5, precond="none", max_blocks=6)
    assert np.allclose(r.theta_hist[5], lam[:4], rtol=0, atol=1e-11 * np.abs(lam).max())


def test_ritz_values_do_not_increase_between_restarts():
    # nested subspaces: every Ritz value is non-increasing until a restart
    A = synth.tile_matrix(400, 40, seed=8)
    X0 = synth.initial_guess(A, 6, seed=9)
    r = davidson(A, X0, 6, tol=1e-300, maxiter=30, precond="diag", max_blocks=40)
    th = np.array(r.theta_hist)
    assert r.restarts == 0
    assert np.all(np.diff(th, axis=0) <= 1e-10 * np.abs(th).max())


def test_laplacian_closed_form():
    n = 150
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        if i:
            cols.append(i - 1)
            vals.append(-1.0)
        cols.append(i)
        vals.append(2.0)
        rp[i + 1] = len(cols)
    A = synth.CSR(n=n, row_ptr=rp, col=np.array(cols, dtype=np.int32), val=np.array(vals))
    X0 = synth.normal_block(n, 6, seed=11)
    r = davidson(A, X0, 3, tol=1e-9, maxiter=3000, precond="diag", max_blocks=6)
    exact = np.array([2 - 2 * math.cos(j * math.pi / (n + 1)) for j in range(1, 4)])
    assert r.converged
    assert np.all(np.abs(r.evals - exact) / exact <= 1e-8)
