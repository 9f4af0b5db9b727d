"""Parity of the FOM preconditioner (Section 3.3; precond mode 4) of the CUDA
path with the FP64 oracle, through the C ABI.

Tolerance: the kernel runs FOM in float32, so its result is the exact FOM
result of a problem perturbed by a few float32 roundings per entry (64-term
dot products).  Per tile column the bound used is
||x_gpu - x_ref|| <= 64 eps32 (1 + kappa) ||x_ref||, kappa the condition
number of the oracle's Hessenberg matrix H_s for that column."""
import numpy as np
import pytest

import oracle
import synth
from conftest import has_gpu
from oracle import lobpcg as olb
from oracle.precond import fom_solve

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]

EPS32 = 2.0 ** -24


def _pkg():
    import paper_2109_00485_gb300 as pkg
    pkg.load()
    return pkg


def f32_matrix(A):
    return synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32))


def apply_gpu(A, R, theta, steps=0, precond_create="fom", tile_ptr=None):
    import torch
    pkg = _pkg()
    h = pkg.from_csr(A, k=R.shape[1], nev=1, precond=precond_create, fom_steps=steps, fom_tile_ptr=tile_ptr)
    W = h.precond_apply(torch.from_numpy(R).cuda(), torch.from_numpy(theta).cuda(), mode="fom").cpu().numpy()
    h.destroy()
    return W


def check_tiles(A, R, theta, W, steps, tiles, tile_ptr=None):
    """Compare the GPU result on the given tiles (indices into tile_ptr, else
    64-row tiles) with the oracle, column by column, against
    64 eps32 (1 + kappa(H_s))."""
    worst = 0.0
    for t in tiles:
        if tile_ptr is None:
            r0 = 64 * t
            m = min(64, A.n - r0)
        else:
            r0, m = int(tile_ptr[t]), int(tile_ptr[t + 1] - tile_ptr[t])
        B = oracle.dense_block(A, r0, m)
        for j in range(R.shape[1]):
            tr = {}
            x = fom_solve(B - theta[j] * np.eye(m), R[r0:r0 + m, j].astype(np.float64), steps, float(theta[j]), trace=tr)
            kappa = np.linalg.cond(tr["H"][:-1]) if tr else 1.0
            err = np.linalg.norm(W[r0:r0 + m, j] - x)
            bound = 64 * EPS32 * (1.0 + kappa) * np.linalg.norm(x)
            assert err <= bound, (t, j, err / max(np.linalg.norm(x), 1e-300), kappa)
            worst = max(worst, err / bound if bound > 0 else 0.0)
    return worst


@pytest.mark.parametrize("k", [1, 8, 12, 16, 20, 32])
def test_fom_apply_matches_oracle(k):
    # 15 full tiles and a ragged one of 40 rows; shifts from below the
    # spectrum to well inside it (indefinite tiles)
    A = f32_matrix(synth.tile_matrix(1000, 60, seed=10))
    R = synth.normal_block(A.n, k, seed=2 + k, fp32=True)
    theta = np.linspace(-3.0, 40.0, k)
    W = apply_gpu(A, R, theta)
    assert W.shape == R.shape and np.all(np.isfinite(W))
    check_tiles(A, R, theta, W, 4, range(16))


@pytest.mark.parametrize("steps", [1, 2, 3, 5, 6])
def test_fom_apply_step_counts(steps):
    A = f32_matrix(synth.tile_matrix(700, 80, seed=14))
    k = 16
    R = synth.normal_block(A.n, k, seed=5, fp32=True)
    theta = np.linspace(-1.0, 25.0, k)
    W = apply_gpu(A, R, theta, steps=steps)
    check_tiles(A, R, theta, W, steps, range(11))


@pytest.mark.parametrize("k", [4, 16, 20])
def test_fom_variable_tiles_match_oracle(k):
    # tiles of 7 to 783 rows (both kernels), plus 1-row tiles and the 64 / 66
    # rows either side of the small / large boundary at the front
    A = f32_matrix(synth.tile_matrix(3000, 60, seed=4))
    tp = synth.tile_partition(3000 - 132, 4, median=40) + 132
    tp = np.concatenate([[0, 1, 2, 66], tp]).astype(np.int64)   # tiles of 1, 1, 64 and 66 rows first
    assert np.all(np.diff(tp) > 0) and tp[-1] == 3000
    R = synth.normal_block(A.n, k, seed=9 + k, fp32=True)
    theta = np.linspace(-3.0, 40.0, k)
    W = apply_gpu(A, R, theta, tile_ptr=tp)
    assert np.all(np.isfinite(W))
    check_tiles(A, R, theta, W, 4, range(tp.size - 1), tile_ptr=tp)
    # one FOM step on 1-row tiles is the diagonal preconditioner
    np.testing.assert_allclose(W[:2], R[:2] / (oracle.diagonal(A)[:2, None] - theta[None, :]), rtol=1e-6)


def test_fom_apply_degenerate_columns():
    # a diagonal matrix: a right-hand side with one nonzero per tile is an
    # eigenvector of its tile, so the Krylov space stops after one step and
    # FOM is exact; a zero column gives a zero column; a column whose shift
    # equals the diagonal entry meets the guard (pivot 0 -> +1e-3 max(1,|theta|))
    n = 200
    d = np.linspace(1.0, 9.0, n).astype(np.float32)
    A = synth.CSR(n=n, row_ptr=np.arange(n + 1, dtype=np.int64), col=np.arange(n, dtype=np.int32), val=d)
    k = 4
    R = np.zeros((n, k), dtype=np.float32)
    rows = np.array([5, 70, 130, 199])
    R[rows, 0] = [1.0, -2.0, 3.0, 0.5]
    R[rows, 2] = 1.0
    R[:, 3] = synth.normal_block(n, 1, seed=3, fp32=True)[:, 0]
    theta = np.array([0.25, 0.0, float(d[70]), -2.0])
    W = apply_gpu(A, R, theta)
    want0 = np.zeros(n)
    want0[rows] = R[rows, 0] / (d[rows].astype(np.float64) - 0.25)
    assert np.allclose(W[:, 0], want0, rtol=2e-6, atol=0)
    assert np.array_equal(W[:, 1], np.zeros(n, dtype=np.float32))
    # column 2: row 70 has d - theta = 0 exactly (guarded to 1e-3 max(1, theta)),
    # the other rows divide by d - theta
    sh = d[rows].astype(np.float64) - float(d[70])
    sh[1] = 1e-3 * max(1.0, float(d[70]))
    want2 = np.zeros(n)
    want2[rows] = 1.0 / sh
    assert np.allclose(W[:, 2], want2, rtol=2e-6, atol=0)
    check_tiles(A, R, theta, W, 4, range(4))


def test_fom_argument_checks():
    import torch
    pkg = _pkg()
    A = f32_matrix(synth.tile_matrix(300, 30, seed=1))
    with pytest.raises(pkg.LobpcgError):
        pkg.from_csr(A, k=4, nev=1, precond="fom", fom_steps=7)
    with pytest.raises(pkg.LobpcgError):
        pkg.from_csr(A, k=4, nev=1, precond=5)
    h = pkg.from_csr(A, k=4, nev=1, precond="diag")
    R = torch.zeros((300, 4), device="cuda")
    th = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LobpcgError):
        h.precond_apply(R, th, mode="fom")          # no tiles stored: needs precond = 4 at create
    h.destroy()


def test_solve_with_fom_matches_oracle():
    A = f32_matrix(synth.tile_matrix(3000, 60, seed=4))
    k, nev = 8, 5
    pkg = _pkg()
    X0 = synth.initial_guess(A, k, seed=1001, fp32=True)
    h = pkg.from_csr(A, k=k, nev=nev, tol=1e-6, maxiter=1000, precond="fom", polish_fp64=1)
    X, ev, rs, st = h.solve(X0)
    X64 = h.get_x_f64().cpu().numpy()
    h.destroy()
    assert st["converged"] == 1 and np.all(rs <= 1e-6)
    ref = olb.lobpcg(A, X0.astype(np.float64), nev, tol=1e-10, maxiter=2000, precond="fom")
    assert ref.converged
    normG = oracle.gershgorin(A)
    assert np.all(np.abs(ev - ref.evals) / np.maximum(np.abs(ref.evals), 1e-3 * normG) <= 1e-8)
    R = oracle.spmm_tri(A, X64[:, :nev]) - X64[:, :nev] * ev
    rho = np.linalg.norm(R, axis=0) / (np.abs(ev) * np.linalg.norm(X64[:, :nev], axis=0))
    assert np.all(rho <= 1.05e-6), rho


def test_fom_variable_tiles_solve_and_steps():
    A = f32_matrix(synth.tile_matrix(2500, 60, seed=6))
    tp = synth.tile_partition(2500, 6, median=120)
    for steps in (1, 3, 6):
        R = synth.normal_block(A.n, 12, seed=steps, fp32=True)
        theta = np.linspace(-2.0, 30.0, 12)
        W = apply_gpu(A, R, theta, steps=steps, tile_ptr=tp)
        check_tiles(A, R, theta, W, steps, range(tp.size - 1), tile_ptr=tp)
    pkg = _pkg()
    X0 = synth.initial_guess(A, 8, seed=77, fp32=True)
    h = pkg.from_csr(A, k=8, nev=5, tol=1e-6, maxiter=1000, precond="fom", polish_fp64=1, fom_tile_ptr=tp)
    X, ev, rs, st = h.solve(X0)
    h.destroy()
    assert st["converged"] == 1
    ref = olb.lobpcg(A, X0.astype(np.float64), 5, tol=1e-10, maxiter=2000, precond="fom", fom_tile_ptr=tp)
    normG = oracle.gershgorin(A)
    assert np.all(np.abs(ev - ref.evals) / np.maximum(np.abs(ref.evals), 1e-3 * normG) <= 1e-8)


def test_fom_partition_argument_checks():
    pkg = _pkg()
    A = f32_matrix(synth.tile_matrix(300, 30, seed=1))
    for bad in ([0, 100, 100, 300], [1, 300], [0, 299], [0, 200, 150, 300]):
        with pytest.raises(pkg.LobpcgError):
            pkg.from_csr(A, k=4, nev=1, precond="fom", fom_tile_ptr=np.array(bad))


@pytest.mark.slow
def test_fom_full_size_n2m_sampled_tiles():
    """The bench workload's matrix (n = 2M, ~400 stored entries per row,
    k = 16) in the solver's launch configuration: sampled tiles against the
    oracle computed tile by tile."""
    p = synth.WORKLOADS["full_n2m"]
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True)
    k = p["k"]
    R = synth.normal_block(A.n, k, seed=41, fp32=True)
    theta = np.linspace(-2.0, 30.0, k)
    W = apply_gpu(A, R, theta)
    nt = A.n // 64
    tiles = np.unique(np.concatenate([[0, 1, nt - 1], (synth.u64(13, 78, 1) % np.uint64(nt)).astype(np.int64)]))
    check_tiles(A, R, theta, W, 4, tiles)
    assert np.all(np.isfinite(W))


@pytest.mark.slow
def test_fom_full_size_n2m_variable_tiles():
    """The bench matrix with a partition of 5 to 6000-row tiles (median about
    200): the largest tiles, the smallest and a seeded sample against the
    oracle."""
    p = synth.WORKLOADS["full_n2m"]
    A = synth.tile_matrix(p["n"], p["nnz_per_row"], seed=p["seed"], fp32=True)
    k = p["k"]
    tp = synth.tile_partition(A.n, p["seed"])
    R = synth.normal_block(A.n, k, seed=43, fp32=True)
    theta = np.linspace(-2.0, 30.0, k)
    W = apply_gpu(A, R, theta, tile_ptr=tp)
    assert np.all(np.isfinite(W))
    sizes = np.diff(tp)
    order = np.argsort(sizes)
    tiles = np.unique(np.concatenate([order[:3], order[-2:], [0, sizes.size - 1],
                                      (synth.u64(8, 79, 1) % np.uint64(sizes.size)).astype(np.int64)]))
    check_tiles(A, R, theta, W, 4, tiles, tile_ptr=tp)
