"""Pins for the oracle FOM preconditioner (Section 3.3: a few iterations of the
Full Orthogonalization Method on each shifted diagonal tile), against direct
solves, the one-step closed form, the Galerkin condition on an independently
built Krylov basis, and conjugate gradients on positive definite tiles."""
import numpy as np
import pytest

import oracle
import synth
from oracle import lobpcg as olb
from oracle.precond import apply_bjacobi, apply_fom, fom_solve, tile_solve_lu


def _tile(n, npr, seed, m=64, t=0):
    A = synth.tile_matrix(n, npr, seed=seed)
    return A, oracle.dense_block(A, t * 64, m)


def test_full_krylov_dimension_is_the_direct_solve():
    # s >= m Arnoldi steps span the whole space: FOM is the exact solve
    A, B = _tile(200, 30, seed=5)
    lam = np.linalg.eigvalsh(B)
    rng = np.random.default_rng(1)
    for m in (5, 12, 22):
        M = B[:m, :m] - (lam[0] - 1.0) * np.eye(m)      # positive definite shift
        r = rng.standard_normal(m)
        x = fom_solve(M, r, steps=m + 2, theta=lam[0] - 1.0)
        ref = np.linalg.solve(M, r)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref)


def test_one_step_is_the_shifted_rayleigh_quotient():
    A, B = _tile(128, 40, seed=7)
    rng = np.random.default_rng(2)
    for theta in (-3.0, 0.1, 2.5):
        M = B - theta * np.eye(64)
        r = rng.standard_normal(64)
        x = fom_solve(M, r, steps=1, theta=theta)
        assert np.allclose(x, r * (r @ r) / (r @ M @ r), rtol=1e-13, atol=0)


@pytest.mark.parametrize("steps", [2, 3, 4, 5])
def test_galerkin_condition_on_qr_krylov_basis(steps):
    # x lies in K_s(M, r) and r - M x is orthogonal to it; the basis here comes
    # from a QR factorisation of [r, M r, ..., M^{s-1} r], not from the Arnoldi
    # process under test.  The shift sits inside the spectrum (indefinite M).
    A, B = _tile(256, 50, seed=11 + steps)
    lam = np.linalg.eigvalsh(B)
    rng = np.random.default_rng(steps)
    theta = 0.5 * (lam[20] + lam[21])
    M = B - theta * np.eye(64)
    r = rng.standard_normal(64)
    x = fom_solve(M, r, steps=steps, theta=theta)
    K = np.empty((64, steps))
    K[:, 0] = r / np.linalg.norm(r)
    for j in range(1, steps):
        K[:, j] = M @ K[:, j - 1]
        K[:, j] /= np.linalg.norm(K[:, j])
    Q, _ = np.linalg.qr(K)
    assert np.linalg.norm(x - Q @ (Q.T @ x)) <= 1e-9 * np.linalg.norm(x)
    assert np.linalg.norm(Q.T @ (r - M @ x)) <= 1e-9 * np.linalg.norm(r)


@pytest.mark.parametrize("steps", [1, 3, 5, 9])
def test_positive_definite_tile_matches_conjugate_gradients(steps):
    # on a positive definite system FOM and CG produce the same iterates
    A, B = _tile(300, 30, seed=21)
    lam = np.linalg.eigvalsh(B)
    M = B - (lam[0] - 0.3) * np.eye(64)
    r = np.random.default_rng(9).standard_normal(64)
    x = np.zeros(64)
    res = r.copy()
    p = res.copy()
    for _ in range(steps):                       # textbook CG from x_0 = 0
        Mp = M @ p
        a = (res @ res) / (p @ Mp)
        x = x + a * p
        res_new = res - a * Mp
        p = res_new + ((res_new @ res_new) / (res @ res)) * p
        res = res_new
    got = fom_solve(M, r, steps=steps, theta=lam[0] - 0.3)
    assert np.linalg.norm(got - x) <= 1e-10 * np.linalg.norm(x)


def test_degenerate_inputs():
    M = np.diag(np.linspace(1.0, 4.0, 16))
    # zero right-hand side
    assert np.array_equal(fom_solve(M, np.zeros(16), 4, 0.0), np.zeros(16))
    # r an eigenvector: the Krylov space is invariant after one step
    e = np.zeros(16)
    e[3] = 2.0
    assert np.allclose(fom_solve(M, e, 4, 0.0), e / M[3, 3], rtol=1e-15, atol=0)
    # a zero tile: the single pivot 0 is guarded to +1e-3 max(1, |theta|)
    r = np.arange(1.0, 17.0)
    assert np.allclose(fom_solve(np.zeros((16, 16)), r, 4, 0.0), r / 1e-3, rtol=1e-15, atol=0)
    assert np.allclose(fom_solve(np.zeros((16, 16)), r, 4, -5000.0), r / 5.0, rtol=1e-15, atol=0)
    # a zero leading pivot of a nonsingular H_s: [[0, 1], [1, 0]] from M = the
    # 2 x 2 exchange matrix and r = e_1 -- the row exchange solves it exactly
    M2 = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.array_equal(fom_solve(M2, np.array([3.0, 0.0]), 2, 0.0), [0.0, 3.0])


def test_apply_fom_per_tile_and_full_dimension_limit():
    # tiles of 64, 64, 22 rows; each column its own system with its own shift
    A = synth.tile_matrix(150, 40, seed=12)
    R = synth.normal_block(150, 3, seed=2)
    th = np.array([-100.0, -50.0, -75.0])           # below every tile spectrum
    W = apply_fom(A, R, th, steps=4)
    for t in range(3):
        m = min(64, 150 - 64 * t)
        B = oracle.dense_block(A, 64 * t, m)
        for j in range(3):
            x = fom_solve(B - th[j] * np.eye(m), R[64 * t:64 * t + m, j], 4, th[j])
            assert np.array_equal(W[64 * t:64 * t + m, j], x)
    # with as many steps as tile rows FOM is the exact tile solve: it equals
    # the eigendecomposition form and the LU solve
    Wf = apply_fom(A, R, th, steps=64)
    Wb = apply_bjacobi(A, R, th)
    assert np.linalg.norm(Wf - Wb) <= 1e-9 * np.linalg.norm(Wb)
    y = tile_solve_lu(A, 2, R[128:150, 1], th[1])
    assert np.linalg.norm(Wf[128:150, 1] - y) <= 1e-10 * np.linalg.norm(y)


def test_lobpcg_with_fom_preconditioner_vs_library():
    A = synth.tile_matrix(256, 40, seed=256)
    lam = np.linalg.eigvalsh(oracle.to_dense(A))
    X0 = synth.initial_guess(A, 8, seed=1256)
    r = olb.lobpcg(A, X0, 5, tol=1e-10, maxiter=2000, precond="fom")
    assert r.converged
    assert np.max(np.abs(r.evals - lam[:5]) / np.maximum(np.abs(lam[:5]), 1e-3)) < 1e-10


def test_apply_fom_tile_partitions():
    from oracle.precond import apply_diag, tile_bounds
    A = synth.tile_matrix(150, 40, seed=12)
    R = synth.normal_block(150, 3, seed=2)
    th = np.array([-100.0, -50.0, -75.0])
    # an explicit partition into the default 64-row tiles is the default
    assert np.array_equal(apply_fom(A, R, th, 4, tile_ptr=[0, 64, 128, 150]), apply_fom(A, R, th, 4))
    assert np.array_equal(tile_bounds(150), [0, 64, 128, 150])
    # 1-row tiles: one FOM step on a 1 x 1 system is the diagonal preconditioner
    th2 = np.array([0.5, 3.0, -1.0])
    W1 = apply_fom(A, R, th2, 4, tile_ptr=np.arange(151))
    assert np.allclose(W1, apply_diag(oracle.diagonal(A), R, th2), rtol=1e-14, atol=0)
    # tiles of varying size (5, 12, 83, 50 rows) with as many steps as rows:
    # each tile's exact shifted solve
    tp = [0, 5, 17, 100, 150]
    Wv = apply_fom(A, R, th, 100, tile_ptr=tp)
    for a, b in zip(tp[:-1], tp[1:]):
        B = oracle.dense_block(A, a, b - a)
        for j in range(3):
            y = np.linalg.solve(B - th[j] * np.eye(b - a), R[a:b, j])
            assert np.linalg.norm(Wv[a:b, j] - y) <= 1e-9 * np.linalg.norm(y)


def test_tile_partition_generator():
    tp = synth.tile_partition(100_000, 3)
    d = np.diff(tp)
    assert tp[0] == 0 and tp[-1] == 100_000 and np.all(d >= 1) and np.all(d <= 6000)
    assert 100 <= np.median(d) <= 400                    # mostly a few hundred rows
    assert np.array_equal(tp, synth.tile_partition(100_000, 3))
