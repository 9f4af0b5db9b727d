"""The float32 bound used by the FOM parity tests, checked on the CPU.

The CUDA kernels run FOM in float32 with classical Gram-Schmidt applied
twice, h_{j+1,j}^2 = ||w1||^2 - ||c||^2, and Gaussian elimination with
partial pivoting on H_s.  This test restates that arithmetic in numpy
float32 (test code only: it shares nothing with the kernels or the oracle)
and checks that, over a few hundred tile columns -- 5 to 200 rows, shifts
below and inside the tile spectra -- its distance to the FP64 oracle stays
within ||x32 - x|| <= 64 eps32 (1 + kappa(H_s)) ||x||, the bound the GPU
parity tests apply."""
import numpy as np

import oracle
import synth
from oracle.precond import fom_solve

EPS32 = 2.0 ** -24
F = np.float32


def fom_f32(M, r, steps, theta):
    m = M.shape[0]
    M = M.astype(F)
    r = r.astype(F)
    beta = np.sqrt(F(r @ r))
    if beta == 0:
        return np.zeros(m)
    V = np.zeros((m, steps), F)
    H = np.zeros((steps + 1, steps), F)
    V[:, 0] = r / beta
    s = steps
    for j in range(steps):
        w = (M @ V[:, j]).astype(F)
        wn = np.sqrt(F(w @ w))
        h = (V[:, :j + 1].T @ w).astype(F)
        w = (w - V[:, :j + 1] @ h).astype(F)
        c = (V[:, :j + 1].T @ w).astype(F)
        n1 = F(w @ w)
        w = (w - V[:, :j + 1] @ c).astype(F)
        hs = np.sqrt(max(F(n1 - c @ c), F(0)))
        H[:j + 1, j] = h + c
        H[j + 1, j] = hs
        if hs <= F(1e-6) * wn:
            s = j + 1
            break
        if j + 1 < steps:
            V[:, j + 1] = w / hs
    U = H[:s, :s].copy()
    b = np.zeros(s, F)
    b[0] = beta
    delta = F(1e-3 * max(1.0, abs(theta)))
    for i in range(s):
        if i + 1 < s and abs(U[i + 1, i]) > abs(U[i, i]):
            U[[i, i + 1], i:] = U[[i + 1, i], i:]
            b[[i, i + 1]] = b[[i + 1, i]]
        U[i, i] = (F(1) if U[i, i] >= 0 else F(-1)) * max(abs(U[i, i]), delta)
        if i + 1 < s:
            l = F(U[i + 1, i] / U[i, i])
            U[i + 1, i:] = (U[i + 1, i:] - l * U[i, i:]).astype(F)
            b[i + 1] = F(b[i + 1] - l * b[i])
    y = np.zeros(s, F)
    for i in range(s - 1, -1, -1):
        y[i] = F((b[i] - U[i, i + 1:] @ y[i + 1:]) / U[i, i])
    return (V[:, :s] @ y).astype(np.float64)


def test_float32_fom_within_the_parity_bound():
    A = synth.tile_matrix(3000, 60, seed=31)
    A = synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32).astype(np.float64))
    tp = synth.tile_partition(3000, 32, median=40)
    tp = tp[:40] if tp.size > 40 else tp
    rng = np.random.default_rng(5)
    worst, cases = 0.0, 0
    for t in range(tp.size - 1):
        a, m = int(tp[t]), int(tp[t + 1] - tp[t])
        if m > 200:
            continue
        B = oracle.dense_block(A, a, m)
        lam = np.linalg.eigvalsh(B)
        for theta in (lam[0] - 1.0, 0.5 * (lam[m // 3] + lam[m // 3 + 1]) if m > 3 else lam[0] + 0.1, lam[-1] * 0.6):
            for steps in (2, 4, 6):
                r = rng.standard_normal(m).astype(np.float32).astype(np.float64)
                tr = {}
                x = fom_solve(B - theta * np.eye(m), r, steps, float(theta), trace=tr)
                x32 = fom_f32(B - theta * np.eye(m), r, steps, float(theta))
                kappa = np.linalg.cond(tr["H"][:-1])
                bound = 64 * EPS32 * (1 + kappa) * np.linalg.norm(x)
                err = np.linalg.norm(x32 - x)
                assert err <= bound, (t, m, theta, steps, err / np.linalg.norm(x), kappa)
                worst = max(worst, err / bound)
                cases += 1
    assert cases >= 200
    assert worst < 1.0
