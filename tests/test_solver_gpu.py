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


def _pencil_case(m, kind, seed):
    """Float32 S, HS (n = m rows) whose Gram blocks are exactly G = S^T HS and
    O = S^T S in float64: S = diag(2^-e) (powers of two), HS = diag(2^e) G."""
    rng = np.random.default_rng(seed)
    if kind == "clustered":
        # the spectrum of a Ritz pencil: a few close eigenvalues below zero,
        # the rest spread up to ||H|| ~ 200
        lam = np.concatenate([[-0.8229, -0.8229 + 1e-6, -0.7129, -0.6859, -0.6858, -0.658],
                              rng.uniform(-0.6, 200.0, m - 6)])[:m]
        Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
        G = (Q * lam) @ Q.T
    elif kind == "repeated":
        # two identical diagonal blocks: every eigenvalue exactly twice
        h = m // 2
        B = rng.standard_normal((h, h))
        B = B + B.T
        G = np.zeros((m, m))
        G[:h, :h] = B
        G[h:2 * h, h:2 * h] = B
        if m % 2:
            G[m - 1, m - 1] = 50.0
    else:
        B = rng.standard_normal((m, m))
        G = B + B.T
    # 14 significant bits: the Gram kernel's split products are then exact,
    # so the GPU receives exactly G
    G = np.tril(G.astype(np.float32)).view(np.uint32) & np.uint32(0xFFFFFE00)
    G = G.view(np.float32)
    G = G + np.tril(G, -1).T
    top = 10 if kind == "illcond" else 3
    e = rng.integers(0, top + 1, m)
    if kind == "eigen_route":
        e[1] = 15
    s = np.exp2(-e.astype(np.float64)).astype(np.float32)
    S = np.diag(s).astype(np.float32)
    HS = (np.exp2(e.astype(np.float64))[:, None] * G).astype(np.float32)
    Gx = S.astype(np.float64).T @ HS.astype(np.float64)
    Ox = S.astype(np.float64).T @ S.astype(np.float64)
    return S, HS, Gx, Ox


@pytest.mark.parametrize("m,k,kind", [(5, 1, "random"), (24, 8, "clustered"), (47, 16, "random"),
                                      (48, 16, "clustered"), (48, 16, "repeated"), (48, 16, "illcond"),
                                      (60, 20, "clustered"), (96, 32, "random"), (48, 16, "eigen_route")])
def test_rayleigh_ritz_pencils(m, k, kind):
    """Rayleigh-Ritz on pencils known exactly in float64 (G with clustered or
    exactly repeated eigenvalues, O = diag(4^-e) with pivot spans up to 2^3,
    2^10, or 2^15 for the route through the eigendecomposition of O), against
    the oracle's Cholesky + Jacobi solve (or, past the pivot span, the
    standard problem O^-1/2 G O^-1/2).  A backward-stable solve in float64
    determines every eigenvalue to a few eps64 ||O^-1/2 G O^-1/2||."""
    import torch
    pkg = _pkg()
    S, HS, Gx, Ox = _pencil_case(m, kind, seed=m * 7 + k)
    n = m
    A = synth.CSR(n=n, row_ptr=np.arange(n + 1, dtype=np.int64), col=np.arange(n, dtype=np.int32),
                  val=np.ones(n, dtype=np.float32))
    h = pkg.from_csr(A, k=min(k, 32), nev=1)
    C, th = h.rayleigh_ritz(torch.from_numpy(S).cuda(), torch.from_numpy(HS).cuda(), k)
    C = C.cpu().numpy()
    th = th.cpu().numpy()
    h.destroy()
    dsq = 1.0 / np.sqrt(np.diag(Ox))
    lam_all = np.linalg.eigvalsh(dsq[:, None] * Gx * dsq[None, :])
    if kind == "eigen_route":
        # past the pivot span the pencil is solved in the eigenbasis of O,
        # dropping directions with eigenvalue below 1e-8 of the largest
        keep = np.diag(Ox) >= 1e-8 * np.diag(Ox).max()
        lam_all = np.linalg.eigvalsh((dsq[:, None] * Gx * dsq[None, :])[np.ix_(keep, keep)])
        lam = lam_all[:k]
    else:
        lam, _ = olb.rayleigh_ritz(Gx, Ox, k)
    scale = np.abs(lam_all).max()
    assert np.all(np.abs(th - lam) <= 1e-12 * m * scale), np.abs(th - lam).max() / scale
    assert np.max(np.abs(C.T @ Ox @ C - np.eye(k))) <= 1e-9 * scale / np.abs(lam).max()
    # residual of the pencil in the O^-1/2-scaled basis
    resid = dsq[:, None] * (Gx @ C - Ox @ C * th)
    if kind == "eigen_route":
        resid = resid[keep]
    assert np.max(np.abs(resid)) <= 1e-12 * m * scale * max(1.0, np.abs(C / dsq[:, None]).max())


def test_umma_gram_path_solve_matches_oracle():
    """The tensor-memory Gram kernel (tcgen05.mma, chosen by LOBPCG_GRAM=umma)
    in a full solve, run in a child process: eigenvalues and residuals against
    the oracle as in test_solve_small_matches_oracle."""
    import json
    import os
    import subprocess
    import sys
    code = r"""
import json, numpy as np, synth
import paper_2109_00485_gb300 as pkg
pkg.load()
A = synth.tile_matrix(3000, 60, seed=4)
A = synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32))
X0 = synth.initial_guess(A, 8, seed=1001, fp32=True)
h = pkg.from_csr(A, k=8, nev=5, tol=1e-6, maxiter=1000, precond="diag", polish_fp64=1)
X, ev, rs, st = h.solve(X0)
X64 = h.get_x_f64().cpu().numpy()
h.destroy()
np.save("/tmp/umma_x64.npy", X64[:, :5])
print(json.dumps({"ev": [float(v) for v in ev], "rs": [float(v) for v in rs], "conv": int(st["converged"])}))
"""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, LOBPCG_GRAM="umma", PYTHONPATH=root)
    out = subprocess.run([sys.executable, "-c", code], env=env, cwd=root, capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res = json.loads(out.stdout.strip().splitlines()[-1])
    A = f32_matrix(synth.tile_matrix(3000, 60, seed=4))
    X0 = synth.initial_guess(A, 8, seed=1001, fp32=True)
    ev = np.array(res["ev"])
    assert res["conv"] == 1 and np.all(np.array(res["rs"]) <= 1e-6)
    ref = olb.lobpcg(A, X0.astype(np.float64), 5, tol=1e-10, maxiter=2000, precond="diag")
    normG = oracle.gershgorin(A)
    assert np.all(eig_err(ev, ref.evals, normG) <= 1e-8), (ev, ref.evals)
    rho = residuals_fp64(A, np.load("/tmp/umma_x64.npy"), ev)
    assert np.all(rho <= 1.05e-6), rho


def test_solve_value_only_tiles_matches_oracle():
    """The solve with tile_format 1 (value-only complete tiles): eigenvalues
    and residuals against the oracle as in test_solve_small_matches_oracle."""
    pkg = _pkg()
    A = f32_matrix(synth.tile_matrix(3000, 60, seed=4))
    X0 = synth.initial_guess(A, 8, seed=1001, fp32=True)
    h = pkg.from_csr(A, k=8, nev=5, tol=1e-6, maxiter=1000, precond="diag", polish_fp64=1, tile_format=1)
    X, ev, rs, st = h.solve(X0)
    X64 = h.get_x_f64().cpu().numpy()
    h.destroy()
    assert st["converged"] == 1 and np.all(rs <= 1e-6)
    ref = olb.lobpcg(A, X0.astype(np.float64), 5, tol=1e-10, maxiter=2000, precond="diag")
    normG = oracle.gershgorin(A)
    assert np.all(eig_err(ev, ref.evals, normG) <= 1e-8), (ev, ref.evals)
    assert np.all(residuals_fp64(A, X64[:, :5], ev) <= 1.05e-6)
