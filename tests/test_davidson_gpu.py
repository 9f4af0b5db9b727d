"""Parity of the block Davidson solve (lobpcg_davidson: the same SpMM,
preconditioners, Gram, combine and Rayleigh-Ritz kernels inside block
Davidson) with the FP64 oracle Davidson, through the C ABI.  Eigenvalue
error |theta - lambda| / max(|lambda|, 1e-3 ||H||_G) <= 1e-8 against the
oracle run to a residual of 1e-10; residuals recomputed by the oracle SpMM."""
import numpy as np
import pytest

import oracle
import synth
from conftest import has_gpu
from oracle.davidson import davidson as dav_oracle

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


@pytest.mark.parametrize("precond,blocks", [("diag", 4), ("fom", 3), ("none", 6), ("bjacobi", 2)])
def test_davidson_matches_oracle(precond, blocks):
    A = f32_matrix(synth.tile_matrix(3000, 60, seed=4))
    k, nev = 8, 5
    pkg = _pkg()
    X0 = synth.initial_guess(A, k, seed=1001, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=1e-6, maxiter=2000, precond=precond, polish_fp64=1)
    X, ev, rs, st = h.davidson(X0, max_blocks=blocks)
    X64 = h.get_x_f64().cpu().numpy()
    h.destroy()
    assert st["converged"] == 1 and np.all(rs <= 1e-6), st
    ref = dav_oracle(A, X0.astype(np.float64), nev, tol=1e-10, maxiter=3000, precond=precond, max_blocks=blocks)
    assert ref.converged
    normG = oracle.gershgorin(A)
    assert np.all(eig_err(ev, ref.evals, normG) <= 1e-8), (ev, ref.evals)
    assert np.all(residuals_fp64(A, X64[:, :nev], ev) <= 1.05e-6)


def test_davidson_and_lobpcg_agree():
    A = f32_matrix(synth.tile_matrix(5000, 80, seed=17))
    k, nev = 16, 8
    pkg = _pkg()
    X0 = synth.initial_guess(A, k, seed=5, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=1e-6, maxiter=2000, precond="diag", polish_fp64=1)
    _, ev_d, rs_d, st_d = h.davidson(X0, max_blocks=6)
    _, ev_l, rs_l, st_l = h.solve(X0)
    h.destroy()
    assert st_d["converged"] == 1 and st_l["converged"] == 1
    assert np.all(eig_err(ev_d, ev_l, oracle.gershgorin(A)) <= 2e-8), (ev_d, ev_l)


def test_davidson_float64_values_and_host_x():
    p = synth.WORKLOADS["small_n20k"]
    A64 = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=False)
    A = f32_matrix(A64)
    pkg = _pkg()
    X0 = synth.initial_guess(A64, p["k"], seed=p["seed"] + synth.X0_SEED_OFFSET, fp32=True)
    h = pkg.from_csr(A64, k=p["k"], nev=p["nev"], tol=1e-6, maxiter=2000, precond="diag", polish_fp64=1)
    X, ev, rs, st = h.davidson(X0)                 # host numpy in, host numpy out
    X64 = h.get_x_f64().cpu().numpy()
    h.destroy()
    assert isinstance(X, np.ndarray) and st["converged"] == 1
    ref = dav_oracle(A, X0.astype(np.float64), p["nev"], tol=1e-10, maxiter=3000, precond="diag", max_blocks=6)
    assert np.all(eig_err(ev, ref.evals, oracle.gershgorin(A)) <= 1e-8)
    assert np.all(residuals_fp64(A, X64[:, :p["nev"]], ev) <= 1.05e-6)


def test_davidson_argument_checks():
    pkg = _pkg()
    A = f32_matrix(synth.tile_matrix(600, 30, seed=2))
    X0 = synth.initial_guess(A, 16, seed=3, fp32=True)
    h = pkg.from_csr(A, k=16, nev=4, tol=1e-5, maxiter=500, precond="diag")
    for bad in (1, 7, 0 - 1):
        with pytest.raises(pkg.LobpcgError):
            h.davidson(X0, max_blocks=bad)
    h.davidson(X0, max_blocks=3)
    with pytest.raises(pkg.LobpcgError):            # more blocks than the first call allocated
        h.davidson(X0, max_blocks=5)
    h.destroy()
    h = pkg.from_csr(A, k=32, nev=4, tol=1e-5, maxiter=500, precond="diag")
    with pytest.raises(pkg.LobpcgError):            # 4 x 32 > 96 columns
        h.davidson(synth.initial_guess(A, 32, seed=3, fp32=True), max_blocks=4)
    h.destroy()
