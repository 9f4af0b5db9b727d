"""Oracle block Davidson in FP64 on the same half-stored H.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper (Section 1) notes that its techniques -- the symmetric SpMM from
the stored triangle and the tile preconditioner -- carry over to other
block eigensolvers.  Block (generalised) Davidson is the one built here: it
keeps a growing orthonormal basis V of the search space, takes the k
leftmost Ritz pairs of H on span(V) each iteration, and extends V by the
preconditioned residuals.  Steps, in order:

  1. V = orthonormal basis of X0 (unit columns, Cholesky-QR); HV = H V
  2. loop:
       G = V^T HV, O = V^T V; the k leftmost pairs of G C = O C D
       (the Rayleigh-Ritz step of the paper's eq. rreig on S = V)
       X = V C; HX = HV C; R = HX - X Theta; exit when the nev leftmost
       columns have rho_j <= tol (checked again with an explicit SpMM)
       W = K^{-1} R  (any of the oracle preconditioners)
       when V already holds max_blocks blocks: restart, V = X, HV = HX
       W <- W - V (V^T W) and Cholesky-QR, twice (as for LOBPCG's W)
       HW = H W -- the one SpMM per iteration; V = [V W], HV = [HV HW]

Readings (listed in the design notes): restart keeps exactly the k current
Ritz vectors (thick restart without the previous directions); rho_j, the
exit test, the explicit re-check and the orthonormalisation of W are those
of the LOBPCG oracle.
"""
from __future__ import annotations

import numpy as np

from . import gershgorin, spmm_tri
from .lobpcg import Result, orthonormalize_w, rayleigh_ritz, resid_norms, unit_columns, cholqr, svqb
from .precond import apply_bjacobi, apply_diag, apply_fom, diag_of, tile_eigs


def davidson(A, X0: np.ndarray, nev: int, tol: float = 1e-6, maxiter: int = 1000, precond: str = "diag",
             max_blocks: int = 6, resid_mode: int = 0, tile: int = 64, fom_steps: int = 4,
             max_explicit_restarts: int = 5) -> Result:
    """FP64 block Davidson for the nev leftmost eigenpairs of the symmetric H
    stored as its lower triangle ``A``; the basis holds at most max_blocks
    blocks of k = X0.shape[1] columns."""
    X0 = np.asarray(X0, dtype=np.float64)
    n, k = X0.shape
    assert 1 <= nev <= k and max_blocks >= 2
    normG = gershgorin(A)
    if precond == "diag":
        d = diag_of(A)
        K = lambda R, th: apply_diag(d, R, th)
    elif precond == "bjacobi":
        eigs = tile_eigs(A, tile)
        K = lambda R, th: apply_bjacobi(A, R, th, tile, eigs)
    elif precond == "fom":
        K = lambda R, th: apply_fom(A, R, th, fom_steps, tile)
    elif precond == "none":
        K = lambda R, th: R.copy()
    else:
        raise ValueError(precond)

    V = unit_columns(X0)
    Q = cholqr(V)
    V = Q if Q is not None else svqb(V)
    HV = spmm_tri(A, V)
    res = Result(evals=None, X=None, rho=None, iters=0, converged=False)
    res.restarts = 0
    restarts = 0
    it = 0
    while True:
        theta, C = rayleigh_ritz(V.T @ HV, V.T @ V, k)
        X = V @ C
        HX = HV @ C
        R = HX - X * theta
        rho = resid_norms(R, X, theta, normG, resid_mode)
        res.theta_hist.append(theta.copy())
        res.rho_hist.append(rho.copy())
        if np.all(rho[:nev] <= tol):
            HXe = spmm_tri(A, X)                          # explicit re-check
            rho_e = resid_norms(HXe - X * theta, X, theta, normG, resid_mode)
            if np.all(rho_e[:nev] <= tol) or restarts >= max_explicit_restarts:
                res.converged = bool(np.all(rho_e[:nev] <= tol))
                rho = rho_e
                break
            restarts += 1
            V, HV = X, HXe                                # continue from the explicit product
            continue
        if it >= maxiter:
            break
        it += 1
        W = K(R, theta)
        if V.shape[1] >= max_blocks * k:                  # restart with the Ritz vectors
            V, HV = X, HX
            res.restarts += 1
        W = orthonormalize_w(W, V)
        if W.shape[1] < k:
            res.svqb_used += 1
        HW = spmm_tri(A, W)                               # the one SpMM
        V = np.hstack([V, W])
        HV = np.hstack([HV, HW])
    res.evals = theta[:nev].copy()
    res.X = X[:, :nev].copy()
    res.rho = rho[:nev].copy()
    res.iters = it
    return res
