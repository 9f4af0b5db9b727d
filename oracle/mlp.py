"""Oracle for the learned tile preconditioner's network, FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's preconditioner K (Section 3.3) solves each shifted diagonal tile
(H_T - theta I) w_T = r_T (by 3-5 FOM iterations).  The learned form replaces
that solve by one small network shared by every 64-row tile (not in the
paper; its readings are listed in the design notes).  The network supplies a
correction to the diagonal (1x1-tile) solve D_theta^{-1} r_T:

  input  x = [ r_T / s , (d_T - theta) / g , theta / g ]   (64 + 64 + 1 = 129)
           s = ||r_T||_2,  g = ||H||_G,  d_T = diag of the tile
  hidden h = relu(W1 x + b1)                                (256)
  output y = W2 h + b2                                      (64)
  w_T   = D_theta^{-1} r_T + (s / g) y

with D_theta^{-1} the guarded diagonal solve of oracle.precond.apply_diag.
It is trained on the target t = clip(g (y_T - D_theta^{-1} r_T) / s, +-1e3),
y_T the exact tile solve, by mean squared error over the 64 outputs and the
batch, with Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  The
output layer starts at zero, so the untrained form is the diagonal one.
Parameters are a dict of W1 (256 x 129), b1 (256), W2 (64 x 256), b2 (64).
"""
from __future__ import annotations

import numpy as np

from .precond import apply_diag

N_IN, N_HID, N_OUT = 129, 256, 64
TILE = 64
CLIP = 1e3


def init_params(normals_w1: np.ndarray) -> dict:
    """Initial weights: W1 He (Kaiming) normal from given N(0,1) draws,
    W1 ~ N(0, 2 / 129); b1, W2 and b2 zero."""
    return {"W1": normals_w1.reshape(N_HID, N_IN) * np.sqrt(2.0 / N_IN), "b1": np.zeros(N_HID),
            "W2": np.zeros((N_OUT, N_HID)), "b2": np.zeros(N_OUT)}


def forward(p: dict, X: np.ndarray):
    """X: batch x 129.  Returns (Y batch x 64, cache)."""
    Z = X @ p["W1"].T + p["b1"]
    Hh = np.maximum(Z, 0.0)
    Y = Hh @ p["W2"].T + p["b2"]
    return Y, (X, Z, Hh)


def loss_and_grads(p: dict, X: np.ndarray, T: np.ndarray):
    """Mean squared error L = sum((Y - T)^2) / (batch * 64) and its gradients."""
    Y, (X, Z, Hh) = forward(p, X)
    B = X.shape[0]
    D = Y - T
    L = float(np.sum(D * D) / (B * N_OUT))
    dY = 2.0 * D / (B * N_OUT)
    g = {"W2": dY.T @ Hh, "b2": dY.sum(0)}
    dH = (dY @ p["W2"]) * (Z > 0)
    g["W1"] = dH.T @ X
    g["b1"] = dH.sum(0)
    return L, g


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; t >= 1."""
    for key in p:
        m[key] = b1 * m[key] + (1 - b1) * g[key]
        v[key] = b2 * v[key] + (1 - b2) * g[key] * g[key]
        mh = m[key] / (1 - b1 ** t)
        vh = v[key] / (1 - b2 ** t)
        p[key] = p[key] - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def tile_inputs(r: np.ndarray, d: np.ndarray, theta: float, normG: float):
    """Network input and scale s for one tile column r (64), diagonal d (64)."""
    s = float(np.linalg.norm(r))
    x = np.concatenate([r / s if s > 0 else np.zeros_like(r), (d - theta) / normG, [theta / normG]])
    return x, s


def tile_target(y: np.ndarray, r: np.ndarray, d: np.ndarray, theta: float, normG: float) -> np.ndarray:
    """Training target of one tile column: exact solve y, residual r, tile
    diagonal d (all length 64)."""
    s = float(np.linalg.norm(r))
    yd = apply_diag(d, r[:, None], np.array([theta]))[:, 0]
    return np.clip(normG * (y - yd) / s, -CLIP, CLIP)


def apply(p: dict, R: np.ndarray, d: np.ndarray, theta: np.ndarray, normG: float) -> np.ndarray:
    """w_T = D_theta^{-1} r_T + c_T, c_T = (s / g) MLP(x), for every 64-row tile
    and column (a ragged last tile is zero-padded; tiles with s = 0 give
    w_T = 0).  A non-finite c_T is dropped; a c_T longer than D_theta^{-1} r_T
    is scaled down to its length.
    Pinned through its pieces: the forward pass by the gradient checks, the
    diagonal part by apply_diag's own pins, a zero output layer giving
    exactly the diagonal solve, and hand-worked tiles with a constant output
    layer (W2 = 0, b2 = c) that fix the scale s / g and the length bound,
    kept and clamped, on a full and a ragged tile."""
    n, k = R.shape
    W = apply_diag(d, R, theta)
    for t0 in range(0, n, TILE):
        m = min(TILE, n - t0)
        for j in range(k):
            r = np.zeros(TILE)
            dd = np.zeros(TILE)
            r[:m] = R[t0:t0 + m, j]
            dd[:m] = d[t0:t0 + m]
            x, s = tile_inputs(r, dd, theta[j], normG)
            if s == 0.0:
                continue
            y, _ = forward(p, x[None, :])
            c = (s / normG) * y[0, :m]
            if not np.all(np.isfinite(c)):
                continue
            cn, dn = np.linalg.norm(c), np.linalg.norm(W[t0:t0 + m, j])
            W[t0:t0 + m, j] += c * (dn / cn if cn > dn else 1.0)
    return W
