"""Parity of the CUDA LOBPCG solve with the FP64 oracle at every block size
the workloads use: (k, nev) = (8, 5), (16, 8) and (20, 10), with the
diagonal, block-Jacobi and FOM preconditioners (and the learned form at
k = 16), and of the n = 2,000,000 workload's eight lowest eigenvalues with
the oracle's stored run.

Reference eigenvalues: the nev smallest eigenvalues of the dense H (the plain
definition of what Algorithm 1 computes; LAPACK through the oracle's
dense_lowest) on the same float32-valued matrix.  Eigenvalue error
|theta - lambda| / max(|lambda|, 1e-3 ||H||_G) <= 1e-8 at the solver's
tolerance 1e-6; residuals of the float64 Ritz vectors recomputed by the
oracle's SpMM <= 1.05e-6 (the solver confirms 1e-6 with its own explicit
float64 product)."""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from conftest import has_gpu
from oracle import lobpcg as olb

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_n2m_oracle_evals.json")

# n not a multiple of 16 or 64: ragged last row block and last diagonal tile
N, NNZ_ROW, SEED = 6007, 60, 4
_cache = {}


def _pkg():
    import paper_2109_00485_gb300 as pkg
    pkg.load()
    return pkg


def matrix():
    if "A" not in _cache:
        A = synth.tile_matrix(N, NNZ_ROW, seed=SEED)
        _cache["A"] = synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32))
    return _cache["A"]


def reference(nev):
    if "w" not in _cache:
        _cache["w"], _ = olb.dense_lowest(matrix(), 10)
    return _cache["w"][:nev]


def eig_err(theta, lam, normG):
    return np.abs(theta - lam) / np.maximum(np.abs(lam), 1e-3 * normG)


def residuals_fp64(A, X, theta):
    R = oracle.spmm_tri(A, X) - X * theta
    return np.linalg.norm(R, axis=0) / (np.abs(theta) * np.linalg.norm(X, axis=0))


def check(A, k, nev, h, X0):
    X, ev, rs, st = h.solve(X0)
    X64 = h.get_x_f64().cpu().numpy()
    h.destroy()
    assert st["converged"] == 1 and np.all(rs <= 1e-6), (st, rs)
    lam = reference(nev)
    normG = oracle.gershgorin(A)
    err = eig_err(ev, lam, normG)
    assert np.all(err <= 1e-8), (err, ev, lam)
    rho = residuals_fp64(A, X64[:, :nev], ev)
    assert np.all(rho <= 1.05e-6), rho
    return st


@pytest.mark.parametrize("k,nev", [(8, 5), (16, 8), (20, 10)])
@pytest.mark.parametrize("precond", ["diag", "bjacobi", "fom"])
def test_solve_block_sizes_match_oracle(k, nev, precond):
    pkg = _pkg()
    A = matrix()
    X0 = synth.initial_guess(A, k, seed=1001, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=1e-6, maxiter=1000, precond=precond, polish_fp64=1)
    check(A, k, nev, h, X0)


@pytest.mark.parametrize("k,nev", [(7, 4), (32, 10)])
def test_refinement_odd_and_largest_block(k, nev):
    """A tolerance of 1e-9 is below the float32 phase's rounding floor, so
    the solve goes through the float64 refinement: its Gram of X and HX
    (lower triangles on 2 x 2 sub-blocks, columns padded to an even count
    at k = 7, two sub-blocks on some threads at k = 32) and its fused
    update-and-residual kernel.  Eigenvalues within 1e-8, float64 residuals
    of the returned vectors within the tolerance."""
    pkg = _pkg()
    A = matrix()
    X0 = synth.initial_guess(A, k, seed=1003, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=1e-9, maxiter=2000, precond="diag", polish_fp64=1)
    X, ev, rs, st = h.solve(X0)
    X64 = h.get_x_f64().cpu().numpy()
    h.destroy()
    assert st["converged"] == 1 and st["used_fp64"] == 1 and st["iters_fp64"] > 0, st
    err = eig_err(ev, reference(nev), oracle.gershgorin(A))
    assert np.all(err <= 1e-8), err
    rho = residuals_fp64(A, X64[:, :nev], ev)
    assert np.all(rho <= 1.05e-9), rho


def test_oracle_lobpcg_agrees_with_dense_reference():
    """The oracle's LOBPCG (explicit products, tol 1e-10) on the same matrix
    at k = 20 gives the dense eigenvalues: the two references agree."""
    A = matrix()
    X0 = synth.initial_guess(A, 20, seed=1001, fp32=True).astype(np.float64)
    r = olb.lobpcg(A, X0, 10, tol=1e-10, maxiter=500, precond="diag", explicit=True)
    assert r.converged
    assert np.all(np.abs(r.evals - reference(10)) <= 1e-12 * oracle.gershgorin(A))


def test_learned_form_k16_matches_oracle():
    """Learned tile preconditioner at k = 16, nev = 8: trained on pairs from
    20 block-Jacobi iterations, then solved from the same X0."""
    pkg = _pkg()
    A = matrix()
    k, nev = 16, 8
    X0 = synth.initial_guess(A, k, seed=1001, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=1e-6, maxiter=1000, precond="mlp", polish_fp64=1, seed=77)
    hist, used = h.precond_train(X0, harvest_iters=20, n_pairs=1 << 15, epochs=5, lr=1e-3)
    assert used >= 4096 and np.all(np.isfinite(hist))
    check(A, k, nev, h, X0)


@pytest.mark.slow
def test_full_n2m_matches_oracle_golden():
    """The n = 2,000,000 workload (k = 16, nev = 8, diagonal form, tol 1e-6)
    against the eight eigenvalues of the oracle's run to 1e-10 stored in
    tests/golden/full_n2m_oracle_evals.json (written by
    tests/golden/make_full_n2m_oracle.py from oracle/ and synth/ alone).
    Residuals: the float64 Ritz vectors through the float64 SpMM on the GPU,
    whose rows are checked on a sample against the oracle's row products."""
    with open(GOLDEN) as f:
        gold = json.load(f)
    p = synth.WORKLOADS["full_n2m"]
    assert gold["n"] == p["n"] and gold["k"] == p["k"] and gold["nev"] == p["nev"] and gold["converged"]
    pkg = _pkg()
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True)
    assert A.nnz == gold["nnz"]
    X0 = synth.initial_guess(A, p["k"], seed=gold["x0_seed"], fp32=True)
    h = pkg.from_csr(A, k=p["k"], nev=p["nev"], tol=1e-6, maxiter=1000, precond="diag", polish_fp64=1)
    X, ev, rs, st = h.solve(X0)
    assert st["converged"] == 1 and np.all(rs <= 1e-6)
    lam = np.array(gold["evals"])
    err = eig_err(ev, lam, gold["gershgorin"])
    assert np.all(err <= 1e-8), (err, ev, lam)
    X64 = h.get_x_f64()[:, :p["nev"]].contiguous()
    HX64 = h.spmm_sym_f64(X64)
    x64, hx64 = X64.cpu().numpy(), HX64.cpu().numpy()
    h.destroy()
    rows = np.sort(synth.u64(512, 9, 1) % np.uint64(p["n"])).astype(np.int64)
    ref_rows = oracle.spmm_rows(A, x64, rows)
    assert np.allclose(hx64[rows], ref_rows, rtol=0, atol=1e-12 * gold["gershgorin"])
    rho = np.linalg.norm(hx64 - x64 * ev, axis=0) / (np.abs(ev) * np.linalg.norm(x64, axis=0))
    assert np.all(rho <= 1.05e-6), rho
