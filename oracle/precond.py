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
    applied to lam - theta_j;
  * "fom" is the paper's own K^{-1}: a few iterations (three to five,
    Section 3.3) of the Full Orthogonalization Method on each 64-row shifted
    tile, every column of R its own Krylov space, x_0 = 0.  FOM is the
    Arnoldi process (modified Gram-Schmidt) followed by the Galerkin solve
    H_s y = beta e_1, x = V_s y.  Readings: the Arnoldi process stops early
    (s = j) when h_{j+1,j} <= 1e-6 ||M v_j|| (the Krylov space is invariant);
    the small Hessenberg system (the paper leaves its solution open) is
    solved by Gaussian elimination with partial pivoting -- a row exchange
    between neighbouring rows where the subdiagonal entry is the larger --
    each pivot guarded with g() like the tiles above, so that one step
    reduces to the shifted Rayleigh quotient of r.
"""
from __future__ import annotations

import numpy as np

from . import dense_block, diagonal, jacobi_eig, lu_solve

FOM_BREAKDOWN = 1e-6


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


def hessenberg_solve_guarded(Hs: np.ndarray, beta: float, theta: float) -> np.ndarray:
    """y with H_s y = beta e_1 for an upper Hessenberg H_s (s x s): Gaussian
    elimination with partial pivoting (column i has nonzeros in rows i and
    i + 1 only, so a pivot search is one comparison and an exchange of the two
    rows), pivots guarded by g(), then back substitution."""
    s = Hs.shape[0]
    U = np.array(Hs, dtype=np.float64, copy=True)
    b = np.zeros(s)
    b[0] = beta
    th = np.array([theta])
    for i in range(s):
        if i + 1 < s and abs(U[i + 1, i]) > abs(U[i, i]):
            U[[i, i + 1], i:] = U[[i + 1, i], i:]
            b[[i, i + 1]] = b[[i + 1, i]]
        U[i, i] = guard(np.array([U[i, i]]), th)[0]
        if i + 1 < s:
            l = U[i + 1, i] / U[i, i]
            U[i + 1, i:] -= l * U[i, i:]
            b[i + 1] -= l * b[i]
    y = np.zeros(s)
    for i in range(s - 1, -1, -1):
        y[i] = (b[i] - U[i, i + 1:] @ y[i + 1:]) / U[i, i]
    return y


def fom_solve(M: np.ndarray, r: np.ndarray, steps: int, theta: float, trace: dict | None = None) -> np.ndarray:
    """Approximate M^{-1} r by ``steps`` iterations of FOM from x_0 = 0
    (Arnoldi with modified Gram-Schmidt, then the Galerkin solve).  ``trace``
    (optional) receives the basis V_s and the Hessenberg matrix H_s."""
    m = M.shape[0]
    beta = float(np.linalg.norm(r))
    if beta == 0.0:
        return np.zeros(m)
    V = np.zeros((m, steps + 1))
    H = np.zeros((steps + 1, steps))
    V[:, 0] = r / beta
    s = steps
    for j in range(steps):
        w = M @ V[:, j]
        wnorm = float(np.linalg.norm(w))
        for i in range(j + 1):                       # modified Gram-Schmidt
            H[i, j] = w @ V[:, i]
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = float(np.linalg.norm(w))
        if H[j + 1, j] <= FOM_BREAKDOWN * wnorm:      # invariant Krylov space: stop at s = j + 1
            s = j + 1
            break
        if j + 1 < steps:
            V[:, j + 1] = w / H[j + 1, j]
    y = hessenberg_solve_guarded(H[:s, :s], beta, theta)
    if trace is not None:
        trace["V"] = V[:, :s].copy()
        trace["H"] = H[:s + 1, :s].copy()
    return V[:, :s] @ y


def tile_bounds(n: int, tile: int = 64, tile_ptr=None) -> np.ndarray:
    """Row partition of the diagonal tiles: the given ``tile_ptr`` (strictly
    increasing, 0 .. n), else consecutive ``tile``-row tiles."""
    if tile_ptr is None:
        return np.append(np.arange(0, n, tile, dtype=np.int64), np.int64(n))
    tp = np.asarray(tile_ptr, dtype=np.int64)
    assert tp[0] == 0 and tp[-1] == n and np.all(np.diff(tp) > 0)
    return tp


def apply_fom(A, R: np.ndarray, theta: np.ndarray, steps: int = 4, tile: int = 64, tile_ptr=None) -> np.ndarray:
    """w_T,j = FOM_steps(H_T - theta_j I, r_T,j) for every diagonal tile T and
    column j.  Tiles: ``tile_ptr`` (any sizes, as the paper's diagonal tiles of
    1 to thousands of rows), else 64-row tiles with a ragged last one."""
    n, k = R.shape
    W = np.zeros((n, k))
    tp = tile_bounds(n, tile, tile_ptr)
    for t in range(tp.size - 1):
        a, m = int(tp[t]), int(tp[t + 1] - tp[t])
        B = dense_block(A, a, m)
        for j in range(k):
            W[a:a + m, j] = fom_solve(B - theta[j] * np.eye(m), R[a:a + m, j], steps, float(theta[j]))
    return W


def diag_of(A) -> np.ndarray:
    return diagonal(A)
