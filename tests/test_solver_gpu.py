"""Parity of the CUDA LOBPCG solve, preconditioners and Rayleigh-Ritz step
(through the C ABI) with the FP64 CPU oracle.

Eigenvalue error (reading of the "1e-8 relative" target for eigenvalues near
zero): |theta - lambda| / max(|lambda|, 1e-3 ||H||_G) <= 1e-8, against the
oracle run to a residual of 1e-10 on the same (float32-valued) matrix.
Residuals of the returned vectors are recomputed by the oracle's SpMM."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import synth
from conftest import has_gpu
from oracle import lobpcg as olb
from oracle.precond import apply_bjacobi, apply_diag

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def _pkg():
    import paper_2109_00485_gb300 as pkg
    pkg.load()
    return pkg


def f32_matrix(A):
    return synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32))


def eig_err(theta, lam, normG):
    return np.abs(theta - lam) / np.maximum(np.abs(lam), 1e-3 * normG)


def residuals_fp64(A, X, theta):
    R = oracle.spmm_tri(A, X) - X * theta
    return np.linalg.norm(R, axis=0) / (np.abs(theta) * np.linalg.norm(X, axis=0))


def run_gpu_solve(A, k, nev, precond="diag", tol=1e-6, maxiter=1000, seed=1001):
    pkg = _pkg()
    X0 = synth.initial_guess(A, k, seed=seed, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=tol, maxiter=maxiter, precond=precond, polish_fp64=1)
    X, ev, rs, st = h.solve(X0)
    X64 = h.get_x_f64().cpu().numpy()
    h.destroy()
    return X0, X, X64, ev, rs, st


@pytest.mark.parametrize("precond", ["diag", "bjacobi"])
def test_solve_small_matches_oracle(precond):
    A = f32_matrix(synth.tile_matrix(3000, 60, seed=4))
    k, nev = 8, 5
    X0, X, X64, ev, rs, st = run_gpu_solve(A, k, nev, precond=precond)
    assert st["converged"] == 1 and np.all(rs <= 1e-6)
    ref = olb.lobpcg(A, X0.astype(np.float64), nev, tol=1e-10, maxiter=2000, precond=precond)
    assert ref.converged
    normG = oracle.gershgorin(A)
    assert np.all(eig_err(ev, ref.evals, normG) <= 1e-8), (ev, ref.evals)
    rho = residuals_fp64(A, X64[:, :nev], ev)
    assert np.all(rho <= 1.05e-6), rho


@pytest.mark.parametrize("precond", ["diag", "bjacobi"])
def test_small_workload_n20k(precond):
    """The small workload (n = 20,000, ~100 stored entries per row, float64
    values, k = 8, nev = 5, tol 1e-6), diagonal and block-Jacobi forms."""
    p = synth.WORKLOADS["small_n20k"]
    A64 = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=False)
    A = f32_matrix(A64)                     # the matrix the GPU stores
    X0, X, X64, ev, rs, st = run_gpu_solve(A64, p["k"], p["nev"], precond=precond,
                                           seed=p["seed"] + synth.X0_SEED_OFFSET)
    assert st["converged"] == 1
    ref = olb.lobpcg(A, X0.astype(np.float64), p["nev"], tol=1e-10, maxiter=2000, precond=precond)
    normG = oracle.gershgorin(A)
    assert np.all(eig_err(ev, ref.evals, normG) <= 1e-8)
    assert np.all(residuals_fp64(A, X64[:, :p["nev"]], ev) <= 1.05e-6)
    # against the float64 matrix: the float32 rounding of H moves eigenvalues
    # by at most ||dH||_2 <= eps32 ||H||_G (Weyl)
    ref64 = olb.lobpcg(A64, X0.astype(np.float64), p["nev"], tol=1e-10, maxiter=2000, precond=precond)
    assert np.all(np.abs(ev - ref64.evals) <= 6e-8 * normG + 1e-8 * np.abs(ref64.evals))


def test_laplacian_closed_form():
    n, k, nev = 120, 6, 3
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        if i:
            cols.append(i - 1)
            vals.append(-1.0)
        cols.append(i)
        vals.append(2.0)
        rp[i + 1] = len(cols)
    A = synth.CSR(n=n, row_ptr=rp, col=np.array(cols, dtype=np.int32), val=np.array(vals, dtype=np.float32))
    pkg = _pkg()
    X0 = synth.normal_block(n, k, seed=9, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=1e-7, maxiter=3000, precond="diag", polish_fp64=1)
    X, ev, rs, st = h.solve(X0)
    h.destroy()
    exact = np.array([2 - 2 * math.cos(j * math.pi / (n + 1)) for j in range(1, nev + 1)])
    assert st["converged"] == 1
    assert np.all(np.abs(ev - exact) / exact <= 1e-8), (ev, exact)


def test_host_x_round_trip():
    A = f32_matrix(synth.tile_matrix(1500, 50, seed=8))
    pkg = _pkg()
    X0 = synth.initial_guess(A, 4, seed=3, fp32=True)
    h = pkg.from_csr(A, k=4, nev=2, tol=1e-6, maxiter=500, precond="diag")
    X, ev, rs, st = h.solve(X0)              # numpy in, numpy out
    assert isinstance(X, np.ndarray) and X.shape == X0.shape
    import torch
    Xd, ev2, rs2, st2 = h.solve(torch.from_numpy(X0).cuda())
    h.destroy()
    assert np.allclose(ev, ev2, rtol=1e-9, atol=1e-12)


def test_precond_apply_matches_oracle():
    import torch
    pkg = _pkg()
    A = f32_matrix(synth.tile_matrix(1000, 60, seed=10))   # 15 full tiles + a ragged one (40 rows)
    k = 8
    R = synth.normal_block(A.n, k, seed=2, fp32=True)
    theta = np.linspace(-3.0, 40.0, k)
    h = pkg.from_csr(A, k=k, nev=1, precond="bjacobi")
    Rd = torch.from_numpy(R).cuda()
    td = torch.from_numpy(theta).cuda()
    Wd = h.precond_apply(Rd, td, mode="diag").cpu().numpy()
    Wo = apply_diag(oracle.diagonal(A), R.astype(np.float64), theta)
    assert np.max(np.abs(Wd - Wo) / (np.abs(Wo) + 1e-30)) <= 1e-6
    Wb = h.precond_apply(Rd, td, mode="bjacobi").cpu().numpy()
    Wbo = apply_bjacobi(A, R.astype(np.float64), theta)
    # float32 tile eigenvectors: error relative to the size of the tile solve
    scale = np.linalg.norm(Wbo, axis=0)
    assert np.all(np.linalg.norm(Wb - Wbo, axis=0) <= 2e-4 * scale)
    W0 = h.precond_apply(Rd, td, mode="none").cpu().numpy()
    assert np.array_equal(W0, R)
    h.destroy()


def test_rayleigh_ritz_matches_library():
    import torch
    pkg = _pkg()
    A = f32_matrix(synth.tile_matrix(2000, 50, seed=12))
    m, k = 24, 8
    S = synth.normal_block(A.n, m, seed=4, fp32=True)
    h = pkg.from_csr(A, k=k, nev=1)
    Sd = torch.from_numpy(S).cuda()
    HS = h.spmm_sym(Sd)
    C, th = h.rayleigh_ritz(Sd, HS, k)
    C = C.cpu().numpy()
    th = th.cpu().numpy()
    h.destroy()
    S64 = S.astype(np.float64)
    G = S64.T @ oracle.spmm_tri(A, S64)
    O = S64.T @ S64
    w = scipy.linalg.eigh(G, O, eigvals_only=True)[:k]
    assert np.all(np.abs(th - w) <= 1e-6 * np.abs(w).max())
    assert np.max(np.abs(C.T @ O @ C - np.eye(k))) <= 1e-5
    assert np.max(np.abs(G @ C - O @ C * th)) <= 1e-5 * np.abs(G).max()
