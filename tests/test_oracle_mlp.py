"""Pins of the surrogate training reference (oracle/mlp_oracle.py).

  * gradients equal central finite differences of the loss (float64);
  * with every ReLU active the network is affine and the gradient of the MSE
    has the closed form of linear least squares;
  * the first Adam step moves every parameter by lr * g / (|g| + eps);
  * training reduces the loss on a synthetic regression.
"""
import numpy as np

from oracle import mlp_oracle as M
from paper_2109_07527_gb300 import workloads as W


def _params(seed, gain=1.0):
    return M.params_from_bf16(W.random_mlp(seed=seed, gain=gain, out_gain=1.0), W.bf16_to_f32)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = _params(1)
    X = rng.integers(-6, 7, (16, 48)).astype(np.float64)
    t = rng.normal(size=16)
    _, g = M.loss_and_grads(p, X, t)
    h = 1e-6
    for name in M.NAMES:
        a = np.atleast_1d(np.asarray(p[name], dtype=np.float64))
        flat = a.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            q = {k: (np.array(v, copy=True) if k != "b4" else v) for k, v in p.items()}
            def at(v):
                if name == "b4":
                    q["b4"] = v
                else:
                    qa = q[name].reshape(-1)
                    qa[idx] = v
                return M.loss(q, X, t)
            x0 = flat[idx]
            fd = (at(x0 + h) - at(x0 - h)) / (2 * h)
            an = np.atleast_1d(g[name]).reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-8, (name, idx, fd, an)


def test_affine_regime_has_the_least_squares_gradient():
    """Large positive biases keep every ReLU on: y = X A + c with
    A = W1^T W2^T W3^T w4; then dL/dc = mean(y - t) and dL/db4 equals it."""
    rng = np.random.default_rng(2)
    p = _params(3)
    for k in ("b1", "b2", "b3"):
        p[k] = np.full(128, 1e3)
    p["W2"], p["W3"] = np.abs(p["W2"]), np.abs(p["W3"])  # positive pre-activations throughout
    X = rng.integers(-3, 4, (32, 48)).astype(np.float64)
    t = rng.normal(size=32)
    y, c = M.forward(p, X)
    assert (c["z1"] > 0).all() and (c["z2"] > 0).all() and (c["z3"] > 0).all()
    A = p["W1"].T @ p["W2"].T @ p["W3"].T @ p["w4"]
    const = ((p["b1"] @ p["W2"].T + p["b2"]) @ p["W3"].T + p["b3"]) @ p["w4"] + p["b4"]
    assert np.allclose(y, X @ A + const, rtol=1e-12, atol=1e-9)
    _, g = M.loss_and_grads(p, X, t)
    assert np.isclose(g["b4"], np.mean(y - t), rtol=1e-12, atol=1e-12)
    # w4 gradient = h3^T (y - t) / B with h3 = X (W3 W2 W1)^T + const3
    h3 = X @ (p["W3"] @ p["W2"] @ p["W1"]).T + ((p["b1"] @ p["W2"].T + p["b2"]) @ p["W3"].T + p["b3"])
    assert np.allclose(g["w4"], h3.T @ (y - t) / 32, rtol=1e-10, atol=1e-9)


def test_first_adam_step_closed_form():
    p = _params(4)
    rng = np.random.default_rng(5)
    g = {k: (rng.normal(size=np.shape(p[k])) if k != "b4" else 0.3) for k in M.NAMES}
    st = M.adam_init(p)
    q = M.adam_step(p, g, st, lr=1e-2, eps=1e-8)
    for k in M.NAMES:
        gk = np.asarray(g[k], dtype=np.float64)
        assert np.allclose(q[k], np.asarray(p[k]) - 1e-2 * gk / (np.abs(gk) + 1e-8), rtol=1e-12, atol=1e-14)


def test_training_reduces_the_loss():
    rng = np.random.default_rng(6)
    p = _params(7, gain=0.5)
    X = rng.integers(-5, 6, (512, 48)).astype(np.float64)
    t = 0.2 * X[:, 0] - 0.1 * X[:, 25] + 0.05 * X[:, 3] * (X[:, 3] > 0)
    st = M.adam_init(p)
    l0 = M.loss(p, X, t)
    for _ in range(200):
        _, g = M.loss_and_grads(p, X, t)
        p = M.adam_step(p, g, st, lr=3e-3)
    assert M.loss(p, X, t) < 0.1 * l0
