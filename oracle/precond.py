"""Oracle forms of the preconditioner K of Algorithm 1 (W = K^{-1} R).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.3 builds K block-diagonally from the shifted diagonal tiles of H,
each shift close to one desired eigenvalue.  Readings taken here:
  * the shift for column j of R is the current Ritz value theta_j;
  * a near-zero shifted pivot t is guarded as g(t) = sign(t) max(|t|, delta),
    sign(0) = +1, delta = 1e-3 max(1, |theta_j|);
  * "diag" is the tile size 1 case: w_ij = r_ij / g(d_i - theta_j);
  * "bjacobi" solves each 64-row tile exactly, (H_T - theta_j I) w_T = r_T,
    through the eigendecomposition H_T = Q diag(lam) Q^T with the same guard
    applied to lam - theta_j (the paper uses 3-5 FOM iterations instead).
"""
from __future__ import annotations

import numpy as np

from . import dense_block, diagonal, jacobi_eig, lu_solve


def guard(t: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """g(t) = sign(t) max(|t|, delta), delta = 1e-3 max(1, |theta|), sign(0)=+1."""
    delta = 1e-3 * np.maximum(1.0, np.abs(theta))
    s = np.where(t >= 0.0, 1.0, -1.0)
    return s * np.maximum(np.abs(t), delta)


def apply_diag(d: np.ndarray, R: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """w_ij = r_ij / g(d_i - theta_j).  Pinned: for theta below every d_i it
    equals a plain division (tests/test_oracle_precond.py)."""
    return R / guard(d[:, None] - theta[None, :], theta[None, :])


def tile_eigs(A, tile: int = 64):
    """Per-tile eigendecompositions (lam [ntiles, tile], Q [ntiles, tile, tile])
    of the diagonal tiles H[t*tile:(t+1)*tile, ...]; a ragged last tile is
    padded with an identity block whose eigenpairs are never used."""
    n = A.n
    nt = (n + tile - 1) // tile
    lam = np.zeros((nt, tile))
    Q = np.zeros((nt, tile, tile))
    for t in range(nt):
        m = min(tile, n - t * tile)
        B = dense_block(A, t * tile, m)
        w, V = jacobi_eig(B)
        lam[t, :m] = w
        Q[t, :m, :m] = V
        if m < tile:
            Q[t, m:, m:] = np.eye(tile - m)
    return lam, Q


def apply_bjacobi(A, R: np.ndarray, theta: np.ndarray, tile: int = 64, eigs=None) -> np.ndarray:
    """w_T = Q_T diag(1/g(lam_T - theta_j)) Q_T^T r_T per 64-row tile.
    Pinned against the LU solve of (H_T - theta_j I) w_T = r_T on tiles whose
    shifted eigenvalues are all outside the guard (tests)."""
    n, k = R.shape
    lam, Q = eigs if eigs is not None else tile_eigs(A, tile)
    W = np.zeros_like(R, dtype=np.float64)
    for t in range(lam.shape[0]):
        m = min(tile, n - t * tile)
        rT = R[t * tile:t * tile + m]
        QT = Q[t, :m, :m]
        z = QT.T @ rT                                          # Q^T r
        z = z / guard(lam[t, :m, None] - theta[None, :], theta[None, :])
        W[t * tile:t * tile + m] = QT @ z
    return W


def tile_solve_lu(A, t: int, r: np.ndarray, theta: float, tile: int = 64) -> np.ndarray:
    """(H_T - theta I)^{-1} r for tile t by LU with partial pivoting (no guard)."""
    m = min(tile, A.n - t * tile)
    B = dense_block(A, t * tile, m) - theta * np.eye(m)
    return lu_solve(B, r)


def diag_of(A) -> np.ndarray:
    return diagonal(A)
