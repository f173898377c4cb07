"""Plain float64 reference of the surrogate's training step (test
infrastructure only; see the package docstring).

The surrogate of the delayed-acceptance stage is the MLP
48 -> 128 -> 128 -> 128 -> 1 with ReLU between layers,

    z1 = X W1^T + b1,  h1 = relu(z1),   z2 = h1 W2^T + b2,  h2 = relu(z2),
    z3 = h2 W3^T + b3, h3 = relu(z3),   y  = h3 w4 + b4,

trained by mean squared error L = (1/B) sum_r (y_r - t_r)^2 / 2 on pairs of
features and exact pair-energy changes, with Adam (Kingma & Ba, ICLR 2015):

    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
    theta <- theta - lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps).

Everything here is written out with numpy matrix products in float64, with
no fusion or blocking; relu'(z) is taken as 1 for z > 0 and 0 otherwise.
"""
from __future__ import annotations

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")


def forward(p, X):
    """Network output y [B] and the intermediate values for the backward pass."""
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ p["w4"] + p["b4"]
    return y, dict(X=X, z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, h3=h3)


def loss(p, X, t):
    y, _ = forward(p, X)
    return float(0.5 * np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def loss_and_grads(p, X, t):
    """L and dL/dtheta for every parameter, by the chain rule layer by layer."""
    y, c = forward(p, X)
    t = np.asarray(t, dtype=np.float64)
    B = y.shape[0]
    dy = (y - t) / B
    g = {}
    g["w4"] = c["h3"].T @ dy
    g["b4"] = float(dy.sum())
    d3 = np.outer(dy, p["w4"]) * (c["z3"] > 0)
    g["W3"] = d3.T @ c["h2"]
    g["b3"] = d3.sum(0)
    d2 = (d3 @ p["W3"]) * (c["z2"] > 0)
    g["W2"] = d2.T @ c["h1"]
    g["b2"] = d2.sum(0)
    d1 = (d2 @ p["W2"]) * (c["z1"] > 0)
    g["W1"] = d1.T @ c["X"]
    g["b1"] = d1.sum(0)
    return float(0.5 * np.mean((y - t) ** 2)), g


def adam_init(p):
    return dict(m={k: np.zeros_like(np.asarray(p[k], dtype=np.float64)) for k in NAMES},
                v={k: np.zeros_like(np.asarray(p[k], dtype=np.float64)) for k in NAMES}, k=0)


def adam_step(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of every parameter (returns new parameters)."""
    state["k"] += 1
    k = state["k"]
    out = {}
    for n in NAMES:
        state["m"][n] = beta1 * state["m"][n] + (1.0 - beta1) * np.asarray(g[n], dtype=np.float64)
        state["v"][n] = beta2 * state["v"][n] + (1.0 - beta2) * np.asarray(g[n], dtype=np.float64) ** 2
        mh = state["m"][n] / (1.0 - beta1 ** k)
        vh = state["v"][n] / (1.0 - beta2 ** k)
        out[n] = np.asarray(p[n], dtype=np.float64) - lr * mh / (np.sqrt(vh) + eps)
    return out


def params_from_bf16(mlp, bf16_to_f32):
    """float64 parameters from the ABI layout (BF16 bit patterns for weights)."""
    return dict(W1=bf16_to_f32(mlp["W1"]).astype(np.float64), b1=np.asarray(mlp["b1"], np.float64),
                W2=bf16_to_f32(mlp["W2"]).astype(np.float64), b2=np.asarray(mlp["b2"], np.float64),
                W3=bf16_to_f32(mlp["W3"]).astype(np.float64), b3=np.asarray(mlp["b3"], np.float64),
                w4=bf16_to_f32(mlp["w4"]).astype(np.float64), b4=float(mlp["b4"]))
