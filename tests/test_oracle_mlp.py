"""Pins for the oracle network of the learned preconditioner: central
finite differences of the loss for every parameter block, a linear special
case with a closed-form gradient, and Adam against its textbook update."""
import numpy as np

import synth
from oracle import mlp


def small_params(seed=0):
    """Initial weights with a random output layer (the initial one is zero),
    so that every gradient block is exercised."""
    p = mlp.init_params(synth.normals(mlp.N_HID * mlp.N_IN, seed, 1))
    p["W2"] = synth.normals(mlp.N_OUT * mlp.N_HID, seed, 2).reshape(64, 256) * np.sqrt(2 / 256)
    return p


def test_init_scale():
    p = mlp.init_params(synth.normals(mlp.N_HID * mlp.N_IN, 0, 1))
    assert p["W1"].shape == (256, 129) and p["W2"].shape == (64, 256)
    assert abs(p["W1"].std() - np.sqrt(2 / 129)) < 0.01
    assert not p["b1"].any() and not p["W2"].any() and not p["b2"].any()


def test_gradients_finite_differences():
    rng = np.random.default_rng(1)
    p = small_params(3)
    p["b1"] = rng.standard_normal(256) * 0.1
    p["b2"] = rng.standard_normal(64) * 0.1
    X = rng.standard_normal((7, 129))
    T = rng.standard_normal((7, 64))
    L, g = mlp.loss_and_grads(p, X, T)
    h = 1e-6
    for key in ("W1", "b1", "W2", "b2"):
        flat = p[key].reshape(-1)
        for idx in rng.choice(flat.size, size=12, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = mlp.loss_and_grads(p, X, T)
            flat[idx] = old - h
            lm, _ = mlp.loss_and_grads(p, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (key, idx, fd, an)


def test_linear_case_closed_form():
    """With all pre-activations positive the net is affine: Y = X A^T + c with
    A = W2 W1, and dL/db2 = 2 (Y - T) summed / (B 64)."""
    rng = np.random.default_rng(2)
    p = small_params(5)
    p["W1"] = np.abs(p["W1"])
    p["b1"] = np.full(256, 10.0)
    X = np.abs(rng.standard_normal((5, 129)))
    T = rng.standard_normal((5, 64))
    Y, _ = mlp.forward(p, X)
    A = p["W2"] @ p["W1"]
    c = p["W2"] @ p["b1"] + p["b2"]
    assert np.allclose(Y, X @ A.T + c, rtol=1e-12, atol=1e-10)
    _, g = mlp.loss_and_grads(p, X, T)
    assert np.allclose(g["b2"], 2 * (Y - T).sum(0) / (5 * 64), rtol=1e-12)


def test_adam_textbook():
    p = {"a": np.array([1.0, -2.0])}
    g = {"a": np.array([0.5, 0.25])}
    m = {"a": np.zeros(2)}
    v = {"a": np.zeros(2)}
    p, m, v = mlp.adam_step(p, g, m, v, t=1, lr=0.1)
    # first step of bias-corrected Adam moves each weight by lr * sign(g) (up to eps)
    assert np.allclose(p["a"], [1.0 - 0.1, -2.0 - 0.1], atol=1e-6)


def test_tile_inputs_and_target():
    r = np.zeros(64)
    r[3] = 3.0
    r[5] = 4.0
    d = np.linspace(1, 2, 64)
    x, s = mlp.tile_inputs(r, d, 0.5, 10.0)
    assert s == 5.0 and x.shape == (129,)
    assert x[3] == 0.6 and x[5] == 0.8 and np.isclose(x[64], 0.05) and x[128] == 0.05
    # target = g (y - r / (d - theta)) / s, clipped
    r = np.ones(64)
    d = np.full(64, 3.0)
    t = mlp.tile_target(np.full(64, 0.75), r, d, 1.0, 4.0)
    assert np.allclose(t, 4.0 * (0.75 - 0.5) / 8.0)
    assert np.all(mlp.tile_target(np.full(64, 1e9), r, d, 1.0, 2.0) == mlp.CLIP)


def test_untrained_apply_is_the_diagonal_solve():
    """A zero output layer leaves exactly the 1x1-tile solve r_i / (d_i - theta_j)
    (pivots kept away from the guard), including a ragged last tile; a random
    output layer changes every tile."""
    rng = np.random.default_rng(4)
    n, k = 150, 3
    R = rng.standard_normal((n, k))
    d = rng.uniform(3, 10, n)
    theta = np.array([-1.0, 0.3, 2.0])
    p = mlp.init_params(synth.normals(mlp.N_HID * mlp.N_IN, 1, 1))
    W = mlp.apply(p, R, d, theta, 12.0)
    assert np.array_equal(W, R / (d[:, None] - theta[None, :]))
    W2 = mlp.apply(small_params(2), R, d, theta, 12.0)
    for t0 in (0, 64, 128):
        assert not np.allclose(W2[t0:t0 + 64], W[t0:t0 + 64])


def _constant_output_params(c: np.ndarray) -> dict:
    """W2 = 0 and b2 = c: the network returns c whatever its input."""
    p = mlp.init_params(synth.normals(mlp.N_HID * mlp.N_IN, 3, 1))
    p["b1"] = np.ones(mlp.N_HID)
    p["b2"] = c.copy()
    return p


def test_apply_scale_and_length_bound_by_hand():
    """w_T = r_T / (d - theta) + (s / g) y with y = b2 (W2 = 0), worked by
    hand on one 64-row tile: r = 1 on rows 0..15 and 0 elsewhere, so
    s = ||r|| = 4; d = 3; g = ||H||_G = 8.
      column 0, theta = 1, b2 = 0.25: diagonal part 0.5 on rows 0..15,
        ||D^-1 r|| = 2; correction (4/8) 0.25 = 0.125 on every row, length
        0.125 * 8 = 1 <= 2, kept: w = 0.625 (rows 0..15), 0.125 (others).
      column 1, theta = 1, b2 = 1: correction 0.5 on every row, length 4 > 2,
        scaled by 2/4: w = 0.75 (rows 0..15), 0.25 (others).
      column 2, theta = 2, b2 = 1: diagonal part 1 on rows 0..15, length 4;
        correction length 4, not longer, kept: w = 1.5, 0.5.
    A slip in the scale (g/s, s^2/g) or in the bound (direction, dn/cn
    inverted) changes at least one of these values."""
    r = np.zeros(64)
    r[:16] = 1.0
    d = np.full(64, 3.0)
    g = 8.0
    cases = [(1.0, 0.25, 0.625, 0.125), (1.0, 1.0, 0.75, 0.25), (2.0, 1.0, 1.5, 0.5)]
    for theta, b2, top, rest in cases:
        p = _constant_output_params(np.full(64, b2))
        W = mlp.apply(p, r[:, None], d, np.array([theta]), g)[:, 0]
        want = np.where(np.arange(64) < 16, top, rest)
        assert np.array_equal(W, want), (theta, b2, W[:3], W[-3:])


def test_apply_bound_keeps_direction_and_ragged_tile():
    """The length bound scales the correction, it does not turn it: with a
    non-constant b2 the clamped correction is b2 times one positive factor
    fixed by hand.  A ragged last tile (n = 64 + 10) uses its own 10 rows of
    r, d and of the network's output only.  Tile 2 (rows 64..73): r = 2 on
    all 10 rows, s = 2 sqrt(10), d = 5, theta = 1: D^-1 r = 0.5 per row,
    length 0.5 sqrt(10); b2[i] = 1 + i (i = 0..9 used): correction
    (s/g) b2 = (2 sqrt(10)/8)(1 + i), its length (sqrt(10)/4) sqrt(385) is
    longer, so it is scaled to 0.5 sqrt(10): w_i = 0.5 + 0.5 sqrt(10)(1 + i)/sqrt(385)."""
    n = 74
    R = np.zeros((n, 1))
    R[64:, 0] = 2.0
    d = np.full(n, 5.0)
    c = np.arange(64, dtype=np.float64) + 1.0
    p = _constant_output_params(c)
    W = mlp.apply(p, R, d, np.array([1.0]), 8.0)[:, 0]
    assert not W[:64].any()                          # s = 0 tile: w = 0
    i = np.arange(10)
    want = 0.5 + 0.5 * np.sqrt(10.0) * (1.0 + i) / np.sqrt(385.0)
    assert np.allclose(W[64:], want, rtol=1e-14, atol=0), (W[64:], want)
