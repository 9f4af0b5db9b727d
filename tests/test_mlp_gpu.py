"""The learned tile preconditioner on the GPU (through the C ABI) against the
FP64 oracle network: forward pass, gradients, Adam, the tile apply (diagonal
solve plus the network's correction), the fallback to the diagonal solve on
non-finite outputs, the initial weights, and training on pairs harvested from
the solver's own block-Jacobi iterations.

Tolerances (bfloat16 operands, float32 accumulation): outputs within 1e-2 of
the oracle relative to their Frobenius norm, gradient blocks within 2e-2."""
import numpy as np
import pytest

import oracle
import synth
from conftest import has_gpu
from oracle import lobpcg as olb
from oracle import mlp as omlp
from oracle.precond import apply_diag

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")]


def _pkg():
    import paper_2109_00485_gb300 as pkg
    pkg.load()
    return pkg


def f32_matrix(A):
    return synth.CSR(n=A.n, row_ptr=A.row_ptr, col=A.col, val=A.val.astype(np.float32))


def oracle_params(seed):
    """Initial weights with a random output layer and biases, so that every
    block takes part."""
    p = omlp.init_params(synth.normals(omlp.N_HID * omlp.N_IN, seed, 1))
    p["W2"] = synth.normals(omlp.N_OUT * omlp.N_HID, seed, 2).reshape(64, 256) * np.sqrt(2 / 256)
    p["b1"] = 0.1 * synth.normals(omlp.N_HID, seed, 3)
    p["b2"] = 0.1 * synth.normals(omlp.N_OUT, seed, 4)
    return p


def pack(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"]]).astype(np.float32)


def unpack(v):
    v = v.astype(np.float64)
    o = 0
    out = {}
    for key, shape in (("W1", (256, 129)), ("b1", (256,)), ("W2", (64, 256)), ("b2", (64,))):
        size = int(np.prod(shape))
        out[key] = v[o:o + size].reshape(shape)
        o += size
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def handle(pkg, A, k=8, nev=4, **kw):
    return pkg.from_csr(A, k=k, nev=nev, precond="mlp", **kw)


def small_matrix():
    return f32_matrix(synth.tile_matrix(1000, 40, seed=21))   # 15 full tiles and a ragged one of 40 rows


def rounded(p):
    """The weights as the device holds them (float32)."""
    return {key: v.astype(np.float32).astype(np.float64) for key, v in p.items()}


def test_params_round_trip_and_forward():
    import torch
    pkg = _pkg()
    h = handle(pkg, small_matrix())
    p = oracle_params(5)
    v = pack(p)
    h.mlp_set_params(v)
    assert np.array_equal(h.mlp_get_params(), v)
    B = 3001                                          # ragged against the 64-row GEMM tiles
    X = synth.normal_block(B, 129, seed=6, fp32=True)
    Y = h.mlp_forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Yo, _ = omlp.forward(rounded(p), X.astype(np.float64))
    assert rel(Y, Yo) <= 1e-2
    h.destroy()


def test_gradients_and_adam_match_oracle():
    import torch
    pkg = _pkg()
    h = handle(pkg, small_matrix())
    p = oracle_params(7)
    h.mlp_set_params(pack(p))
    p = rounded(p)
    B = 2500
    X = synth.normal_block(B, 129, seed=8, fp32=True)
    T = synth.normal_block(B, 64, seed=9, fp32=True)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    loss = h.mlp_grad(Xd, Td)
    Lo, go = omlp.loss_and_grads(p, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - Lo) <= 1e-2 * Lo
    g = unpack(h.mlp_get_params("grads"))
    for key in ("W1", "b1", "W2", "b2"):
        assert rel(g[key], go[key]) <= 2e-2, key
    # Adam on the device's own gradients: two steps against the textbook update
    m = {key: np.zeros_like(v) for key, v in p.items()}
    v2 = {key: np.zeros_like(v) for key, v in p.items()}
    pref = {key: v.copy() for key, v in p.items()}
    for t in (1, 2):
        if t == 2:
            h.mlp_grad(Xd, Td)
            g = unpack(h.mlp_get_params("grads"))
        h.mlp_adam(1e-3)
        pref, m, v2 = omlp.adam_step(pref, g, m, v2, t=t, lr=1e-3)
        got = unpack(h.mlp_get_params())
        for key in p:
            assert np.max(np.abs(got[key] - pref[key])) <= 1e-6 + 1e-6 * np.abs(pref[key]).max(), (t, key)
    h.destroy()


@pytest.mark.parametrize("k", [8, 20])
def test_tile_apply_matches_oracle(k):
    """The fused apply kernel takes (tile, column) pairs in batches of 64:
    at k = 8 a batch is 8 whole tiles, at k = 20 batches start and end
    inside a tile's columns."""
    import torch
    pkg = _pkg()
    A = small_matrix()
    h = handle(pkg, A, k=k)
    p = oracle_params(11)
    h.mlp_set_params(pack(p))
    R = synth.normal_block(A.n, k, seed=12, fp32=True)
    R[64:128, 2] = 0.0                                  # a tile column with s = 0 gives w = 0
    theta = np.linspace(-2.0, 30.0, k)
    W = h.precond_apply(torch.from_numpy(R).cuda(), torch.from_numpy(theta).cuda(), mode="mlp").cpu().numpy()
    normG = h.info()["gershgorin"]
    d = oracle.diagonal(A)
    Wo = omlp.apply(rounded(p), R.astype(np.float64), d, theta, normG)
    Wd = apply_diag(d, R.astype(np.float64), theta)
    for j in range(k):
        assert rel(W[:, j], Wo[:, j]) <= 1e-2, j
    # element by element: each row within 2 % of the largest correction of
    # its tile column (bfloat16 operands: 2^-9 per rounding, two layers)
    for t0 in range(0, A.n, 64):
        sl = slice(t0, min(t0 + 64, A.n))
        cmax = np.abs(Wo[sl] - Wd[sl]).max(axis=0)
        err = np.abs(W[sl] - Wo[sl])
        assert np.all(err <= 1e-5 * np.abs(Wo[sl]) + 2e-2 * cmax[None, :]), (t0, (err / (cmax + 1e-300)).max())
    assert not W[64:128, 2].any()
    h.destroy()


def test_nonfinite_output_falls_back_to_diagonal():
    import torch
    pkg = _pkg()
    A = small_matrix()
    k = 4
    h = handle(pkg, A, k=k)
    p = oracle_params(13)
    p["b2"][:] = np.nan
    h.mlp_set_params(pack(p))
    R = synth.normal_block(A.n, k, seed=14, fp32=True)
    theta = np.array([-1.0, 0.5, 3.0, 10.0])
    W = h.precond_apply(torch.from_numpy(R).cuda(), torch.from_numpy(theta).cuda(), mode="mlp").cpu().numpy()
    Wo = apply_diag(oracle.diagonal(A), R.astype(np.float64), theta)
    assert np.max(np.abs(W - Wo) / (np.abs(Wo) + 1e-30)) <= 1e-6
    h.destroy()


def test_initial_weights_and_short_training():
    """Harvest from 40 block-Jacobi iterations of a small matrix, zero epochs:
    the drawn weights have W1 ~ N(0, 2/129) and zero b1, W2, b2, so the
    apply equals the diagonal solve; one epoch then moves the weights."""
    import torch
    pkg = _pkg()
    A = small_matrix()
    k = 8
    h = handle(pkg, A, k=k, seed=5)
    X0 = synth.initial_guess(A, k, seed=6, fp32=True)
    hist, used = h.precond_train(X0, harvest_iters=40, n_pairs=8192, epochs=0)
    assert used == 40 * 16 * k
    p = unpack(h.mlp_get_params())
    assert abs(p["W1"].std() - np.sqrt(2 / 129)) < 0.01 and abs(p["W1"].mean()) < 0.01
    assert not p["b1"].any() and not p["W2"].any() and not p["b2"].any()
    R = synth.normal_block(A.n, k, seed=7, fp32=True)
    theta = np.linspace(-1.0, 5.0, k)
    W = h.precond_apply(torch.from_numpy(R).cuda(), torch.from_numpy(theta).cuda(), mode="mlp").cpu().numpy()
    Wo = apply_diag(oracle.diagonal(A), R.astype(np.float64), theta)
    assert np.max(np.abs(W - Wo) / (np.abs(Wo) + 1e-30)) <= 1e-6
    assert hist.shape == (1,) and hist[0] > 0
    hist, used = h.precond_train(X0, harvest_iters=40, n_pairs=8192, epochs=3, lr=1e-3)
    assert hist.shape == (4,) and np.all(np.isfinite(hist))
    # early stopping keeps the weights of the lowest held-out loss
    moved = unpack(h.mlp_get_params())["W2"].any()
    assert moved == (hist[1:].min() < hist[0])
    h.destroy()


def test_untrained_solve_is_refused():
    pkg = _pkg()
    A = small_matrix()
    h = handle(pkg, A, k=4, nev=2)
    X0 = synth.initial_guess(A, 4, seed=3, fp32=True)
    with pytest.raises(pkg.LobpcgError) as e:
        h.solve(X0)
    assert e.value.status == 9
    h.destroy()


def test_training_learns_and_solve_converges():
    """Harvest pairs from 20 block-Jacobi iterations of the small workload
    (n = 20,000, k = 8), train, then solve with the learned form from the
    same X0: the training loss does not grow, the eigenvalues match the oracle
    within 1e-8, and the iteration counts of the learned, diagonal,
    block-Jacobi and unpreconditioned forms are reported side by side.  The
    learned form needs fewer iterations than no preconditioner.  (Counts of
    one form vary by tens of percent from run to run: the float32 product's
    order of additions is not fixed, and the switch to the float64 phase
    depends on it.)"""
    pkg = _pkg()
    w = synth.WORKLOADS["small_n20k"]
    A64 = synth.tile_matrix(w["n"], w["nnz_per_row"], seed=w["seed"], fp32=False)
    A = f32_matrix(A64)
    k, nev = w["k"], w["nev"]
    X0 = synth.initial_guess(A64, k, seed=w["seed"] + synth.X0_SEED_OFFSET, fp32=True)
    # 5 epochs (the bench setting): longer training over-fits these pairs and
    # has taken the learned solve from 40-56 to 194-394 iterations
    h = pkg.from_csr(A64, k=k, nev=nev, tol=1e-6, maxiter=3000, precond="mlp", polish_fp64=1, seed=77)
    hist, used = h.precond_train(X0, harvest_iters=20, n_pairs=1 << 16, epochs=5, lr=1e-3)
    assert used >= 20 * 313 * k * 0.9
    assert np.all(np.isfinite(hist)) and hist.min() <= hist[0], hist
    X, ev, rs, st = h.solve(X0)
    h.destroy()
    assert st["converged"] == 1
    ref = olb.lobpcg(A, X0.astype(np.float64), nev, tol=1e-10, maxiter=2000, precond="diag")
    normG = oracle.gershgorin(A)
    assert np.all(np.abs(ev - ref.evals) / np.maximum(np.abs(ref.evals), 1e-3 * normG) <= 1e-8)
    iters = {}
    for pc in ("none", "diag", "bjacobi"):
        hp = pkg.from_csr(A64, k=k, nev=nev, tol=1e-6, maxiter=3000, precond=pc, polish_fp64=1)
        try:
            _, _, _, sp = hp.solve(X0)
        except pkg.LobpcgError as e:          # no preconditioner may not converge in 3000
            assert e.status == 6
            sp = e.result[3]
        hp.destroy()
        iters[pc] = sp["iters"]
    iters["mlp"] = st["iters"]
    print("iterations to 1e-6:", iters, "held-out loss:", hist)
    assert iters["mlp"] < iters["none"], iters


def test_learned_form_iterations_against_diagonal():
    """The learned form against the plain diagonal form on the small workload
    (n = 20,000, k = 8, nev = 5, tol 1e-6), three solves each from the same
    X0 (the learned form retrained each time).  Measured on GB300: medians
    57 (learned) and 57 (diagonal) over five runs each, block-Jacobi 59; in
    another run 67 and 57 (ratio 1.18).  The learned form gains nothing over
    the diagonal one on these matrices; the test holds it to within 40 % of
    the diagonal form's median (counts vary by 10-20 % from run to run) and
    to the same eigenvalues."""
    pkg = _pkg()
    w = synth.WORKLOADS["small_n20k"]
    A64 = synth.tile_matrix(w["n"], w["nnz_per_row"], seed=w["seed"], fp32=False)
    k, nev = w["k"], w["nev"]
    X0 = synth.initial_guess(A64, k, seed=w["seed"] + synth.X0_SEED_OFFSET, fp32=True)
    iters, evs = {"diag": [], "mlp": []}, {}
    for pc in iters:
        for _ in range(3):
            h = pkg.from_csr(A64, k=k, nev=nev, tol=1e-6, maxiter=3000, precond=pc, polish_fp64=1, seed=77)
            if pc == "mlp":
                h.precond_train(X0, harvest_iters=20, n_pairs=1 << 16, epochs=5, lr=1e-3)
            X, ev, rs, st = h.solve(X0)
            h.destroy()
            assert st["converged"] == 1
            iters[pc].append(st["iters"])
            evs[pc] = ev
    print("iterations to 1e-6 (three solves each):", iters)
    ratio = np.median(iters["mlp"]) / np.median(iters["diag"])
    assert ratio <= 1.4, (ratio, iters)
    normG = oracle.gershgorin(f32_matrix(A64))
    assert np.all(np.abs(evs["mlp"] - evs["diag"]) <= 1e-8 * np.maximum(np.abs(evs["diag"]), 1e-3 * normG))
