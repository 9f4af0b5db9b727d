"""Oracle block LOBPCG in FP64 (Algorithm 1 of the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The k lowest eigenpairs solve the trace-minimisation problem (Section 2,
eq. tracemin); LOBPCG reaches them by the update of eq. (xupd) with
coefficients from the Rayleigh-Ritz pencil of eq. (rreig) on
S = [X W P] (eq. rrsubspace).  Steps, in the paper's order:

  1. [C, Theta] = RayleighRitz(H, X0); X = X0 C            (Algorithm 1, lines 1-2)
  2. R = HX - X Theta; P = empty                          (lines 3-4)
  3. loop: count converged columns of R; exit when all nev
     have converged                                        (lines 11-12)
     W = K^{-1} R                                          (line 6)
     W <- W - X (X^T W), twice; Cholesky-QR of W, twice   (Section 3.4)
     HW = H W  -- the only SpMM per iteration               (Section 2, after eq. upd2)
     S = [X W P], HS = [HX HW HP]
     G = S^T HS, O = S^T S; solve G C = O C D, keep the k
     leftmost pairs                                        (eqs. go, rreig)
     X = S C; HX = HS C; P = W C2 + P C3; HP = HW C2 + HP C3 (eqs. xupd, pupd, upd1, upd2)
     R = HX - X Theta                                      (line 10)

Readings where the paper is silent (each listed in the design notes):
  * residual norm: rho_j = ||r_j|| / (max(|theta_j|, 1e-12 ||H||_G) ||x_j||)
    (resid_mode 0) or ||r_j|| / (||H||_G ||x_j||) (resid_mode 1);
  * exit when the nev leftmost columns have rho_j <= tol (nev <= k; the other
    k - nev columns are guard vectors, no locking);
  * W is projected against X before Cholesky-QR; its columns are scaled to
    unit norm first; a failed Cholesky falls back to SVQB (Stathopoulos & Wu
    2002) which drops directions with sigma < 1e-12 sigma_max;
  * P and HP columns are scaled to unit ||p_j|| before the Rayleigh-Ritz step;
  * if O is not numerically positive definite (Cholesky fails or its
    pivots span more than 1e4, i.e. cond(O) above about 1e8), P is dropped
    for that iteration;
  * on exit HX is recomputed by an explicit SpMM and convergence re-checked;
    if it no longer holds the iteration continues from the explicit HX;
  * ``explicit=True`` (reference runs): HX and HP are formed by explicit
    SpMMs each iteration instead of the recurrences of eqs. upd1-upd2.  The
    recurrences are exact in exact arithmetic, but once some columns have
    converged to rounding level their P columns are tiny differences that
    the unit scaling magnifies, so the recurrence HP drifts away from H P
    and the Ritz values can fall below the eigenvalues (k = 20, n = 8000:
    the residual climbed from 1e-13 back to 5e-4 and stayed there).
    Explicit products cost two extra SpMMs per iteration and reach the
    dense eigenvalues to 3e-14.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import cholesky, gershgorin, jacobi_eig, spmm_tri
from .precond import apply_bjacobi, apply_diag, apply_fom, diag_of, tile_eigs


class RRFailure(RuntimeError):
    pass


def sym(M: np.ndarray) -> np.ndarray:
    return 0.5 * (M + M.T)


def tri_inv_lower(L: np.ndarray) -> np.ndarray:
    """Inverse of a lower-triangular matrix by forward substitution."""
    m = L.shape[0]
    Inv = np.zeros_like(L)
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        for i in range(m):
            e[i] = (e[i] - L[i, :i] @ Inv[:i, j]) / L[i, i] if i >= j else 0.0
            Inv[i, j] = e[i]
    return Inv


def rayleigh_ritz(G: np.ndarray, O: np.ndarray, k: int, pivot_span: float = 1e4):
    """Solve the pencil G C = O C D (eq. rreig) and keep the k leftmost pairs.

    O = L L^T (Cholesky); G_hat = L^{-1} G L^{-T}; G_hat = V D V^T (Jacobi);
    C = L^{-T} V[:, :k].  Raises RRFailure when O is not numerically positive
    definite (Cholesky fails or max L_jj / min L_jj > pivot_span).
    Pinned against closed forms and a library generalised eigensolver."""
    L = cholesky(sym(O))
    if L is None:
        raise RRFailure("O not positive definite")
    dg = np.diag(L)
    if dg.max() > pivot_span * dg.min():
        raise RRFailure("O numerically singular")
    Li = tri_inv_lower(L)
    Gh = sym(Li @ sym(G) @ Li.T)
    w, V = jacobi_eig(Gh)
    C = Li.T @ V[:, :k]
    return w[:k].copy(), C


def cholqr(W: np.ndarray):
    """One Cholesky-QR pass (Section 3.4): B = W^T W = R^T R, W <- W R^{-1}.
    Returns None if the Cholesky factorisation fails."""
    L = cholesky(sym(W.T @ W))
    if L is None:
        return None
    return W @ tri_inv_lower(L).T


def svqb(W: np.ndarray, drop: float = 1e-12) -> np.ndarray:
    """SVQB orthonormalisation (Stathopoulos & Wu 2002): B = W^T W,
    D = diag(B)^{-1/2}, D B D = V diag(s) V^T, W <- W D V diag(s)^{-1/2},
    dropping directions with s < drop * max(s)."""
    B = sym(W.T @ W)
    dd = np.sqrt(np.maximum(np.diag(B), np.finfo(float).tiny))
    Dm = np.diag(1.0 / dd)
    s, V = jacobi_eig(sym(Dm @ B @ Dm))
    keep = s > drop * s.max()
    return W @ Dm @ V[:, keep] @ np.diag(1.0 / np.sqrt(s[keep]))


def unit_columns(W: np.ndarray) -> np.ndarray:
    nrm = np.linalg.norm(W, axis=0)
    nrm[nrm == 0.0] = 1.0
    return W / nrm


def orthonormalize_w(W: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Two passes of: unit columns, W <- W - X (X^T W), unit columns,
    Cholesky-QR.  The second pass repairs what cancellation left of X in W
    when W was nearly inside span(X).  SVQB replaces a failed Cholesky-QR."""
    for _ in range(2):
        W = unit_columns(W)
        W = W - X @ (X.T @ W)
        W = unit_columns(W)
        Q = cholqr(W)
        W = Q if Q is not None else svqb(W)
    return W


def resid_norms(R, X, theta, normG, mode=0):
    rn = np.linalg.norm(R, axis=0)
    xn = np.linalg.norm(X, axis=0)
    if mode == 0:
        return rn / (np.maximum(np.abs(theta), 1e-12 * normG) * xn)
    return rn / (normG * xn)


def dense_lowest(A, nev: int):
    """The nev smallest eigenvalues of H and their eigenvectors, from the
    dense matrix: the plain definition of what LOBPCG computes (Section 2,
    eq. tracemin), by a library symmetric eigensolver (LAPACK through
    ``scipy.linalg.eigh``).  For small n only (n^2 doubles).  Pinned against
    the 1-D Laplacian closed form and the Jacobi oracle (tests)."""
    import scipy.linalg
    from . import to_dense
    w, V = scipy.linalg.eigh(to_dense(A), subset_by_index=[0, nev - 1])
    return w, V


@dataclass
class Result:
    evals: np.ndarray
    X: np.ndarray
    rho: np.ndarray
    iters: int
    converged: bool
    theta_hist: list = field(default_factory=list)
    rho_hist: list = field(default_factory=list)
    p_dropped: int = 0
    svqb_used: int = 0


def lobpcg(A, X0: np.ndarray, nev: int, tol: float = 1e-6, maxiter: int = 1000,
           precond: str = "diag", resid_mode: int = 0, tile: int = 64,
           precond_fn=None, max_explicit_restarts: int = 5, fom_steps: int = 4,
           fom_tile_ptr=None, explicit: bool = False) -> Result:
    """FP64 block LOBPCG on the symmetric H stored as its lower triangle ``A``.

    ``precond``: "none", "diag", "bjacobi" (64-row tiles), "fom" (``fom_steps``
    FOM iterations per diagonal tile: ``fom_tile_ptr``, else 64-row tiles) or "custom"
    (``precond_fn(R, theta) -> W``).  ``explicit``: HX and HP by explicit
    SpMMs instead of the recurrences (see the module notes).  Returns the nev
    leftmost Ritz pairs."""
    X0 = np.asarray(X0, dtype=np.float64)
    n, k = X0.shape
    assert 1 <= nev <= k
    normG = gershgorin(A)
    if precond == "diag":
        d = diag_of(A)
        K = lambda R, th: apply_diag(d, R, th)
    elif precond == "bjacobi":
        eigs = tile_eigs(A, tile)
        K = lambda R, th: apply_bjacobi(A, R, th, tile, eigs)
    elif precond == "fom":
        K = lambda R, th: apply_fom(A, R, th, fom_steps, tile, fom_tile_ptr)
    elif precond == "none":
        K = lambda R, th: R.copy()
    elif precond == "custom":
        K = precond_fn
    else:
        raise ValueError(precond)

    # Algorithm 1, lines 1-4
    HX0 = spmm_tri(A, X0)
    theta, C = rayleigh_ritz(X0.T @ HX0, X0.T @ X0, k)
    X = X0 @ C
    HX = HX0 @ C
    R = HX - X * theta
    P = HP = None
    res = Result(evals=theta, X=X, rho=None, iters=0, converged=False)
    restarts = 0
    it = 0
    while True:
        rho = resid_norms(R, X, theta, normG, resid_mode)
        res.theta_hist.append(theta.copy())
        res.rho_hist.append(rho.copy())
        if np.all(rho[:nev] <= tol):
            HXe = spmm_tri(A, X)                      # explicit re-check
            Re = HXe - X * theta
            rho_e = resid_norms(Re, X, theta, normG, resid_mode)
            if np.all(rho_e[:nev] <= tol) or restarts >= max_explicit_restarts:
                res.converged = bool(np.all(rho_e[:nev] <= tol))
                rho = rho_e
                break
            HX, R = HXe, Re
            restarts += 1
            continue
        if it >= maxiter:
            break
        it += 1
        W = K(R, theta)                               # line 6
        W = orthonormalize_w(W, X)
        if W.shape[1] < k:
            res.svqb_used += 1
        HW = spmm_tri(A, W)                           # the one SpMM
        if P is not None:
            pn = np.linalg.norm(P, axis=0)
            pn[pn == 0.0] = 1.0
            P, HP = P / pn, HP / pn
            if explicit:
                HP = spmm_tri(A, P)
        kw = W.shape[1]
        try:
            if P is None:
                raise RRFailure("no P")
            S = np.hstack([X, W, P])
            HS = np.hstack([HX, HW, HP])
            theta_new, C = rayleigh_ritz(S.T @ HS, S.T @ S, k)
        except RRFailure as e:
            if P is not None:
                res.p_dropped += 1
            S = np.hstack([X, W])
            HS = np.hstack([HX, HW])
            theta_new, C = rayleigh_ritz(S.T @ HS, S.T @ S, k)
        X = S @ C                                     # eq. (xupd)
        HX = spmm_tri(A, X) if explicit else HS @ C   # eq. (upd1)
        P = S[:, k:] @ C[k:]                          # eq. (pupd)
        HP = HS[:, k:] @ C[k:]                        # eq. (upd2)
        theta = theta_new
        R = HX - X * theta                            # line 10
    res.evals = theta[:nev].copy()
    res.X = X[:, :nev].copy()
    res.rho = rho[:nev].copy()
    res.iters = it
    return res
