"""Surrogate training on the tensor cores against the float64 reference
(oracle/mlp_oracle.py), through the C ABI.

  * the tcgen05 product D = A B^T equals the float64 product of the same BF16
    operands within FP32 accumulation error (tiles, a ragged M, a K that is not
    a multiple of the 64-wide stage, split-K accumulation, N = 48 and 128);
  * the loss and every gradient element match the reference within a bound
    (both the fused step and the one-product-per-launch path)
    derived from where the kernels round (activations and back-propagated
    errors stored in BF16 between the products, FP32 accumulation), carried
    through the network layer by layer (_gradient_bounds);
  * Adam (cr_train_apply with given gradients) matches the reference's
    adam_step element by element -- masters and both moments, after one step
    and after ten -- within the FP32 rounding of the update (_adam_bounds);
  * Adam steps reduce the loss like the reference does;
  * a surrogate trained here and loaded into a context keeps the DA parity.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as MO
from paper_2109_07527_gb300 import workloads as W
from parity_util import compare_logs_da, compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_07527_gb300 import crmc
    crmc._lib()
    return torch, crmc


def _bf16_dev(torch, a):
    bits = W.to_bf16_bits(np.asarray(a, np.float32))
    return torch.from_numpy(bits.view(np.int16).copy()).cuda(), W.bf16_to_f32(bits).astype(np.float64)


@pytest.mark.parametrize("M,N,K,acc", [(128, 128, 64, False), (256, 128, 128, False), (200, 48, 64, False),
                                       (128, 128, 1000, False), (128, 128, 8192, True), (128, 48, 4096, True)])
def test_tensor_core_product(env, M, N, K, acc):
    torch, crmc = env
    rng = np.random.default_rng(M + N + K)
    A, Af = _bf16_dev(torch, rng.normal(size=(M, K)))
    B, Bf = _bf16_dev(torch, rng.normal(size=(N, K)))
    D = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    crmc.mma_bf16(A.data_ptr(), B.data_ptr(), D.data_ptr(), M, N, K, accumulate=acc)
    got = D.cpu().numpy().astype(np.float64)
    ref = Af @ Bf.T
    scale = np.abs(Af) @ np.abs(Bf).T
    err = np.abs(got - ref)
    assert np.all(err <= 2e-6 * scale + 1e-6), (err.max(), np.unravel_index(np.argmax(err - 2e-6 * scale), err.shape))
    if acc:  # accumulates into D
        crmc.mma_bf16(A.data_ptr(), B.data_ptr(), D.data_ptr(), M, N, K, accumulate=True)
        assert np.allclose(D.cpu().numpy(), 2 * got, rtol=1e-5, atol=1e-4)


def _batch(rng, B, scale=1.0):
    X = rng.integers(-6, 7, (B, 48)).astype(np.float32)
    t = (0.3 * X[:, 0] - 0.2 * X[:, 24] + 0.1 * np.maximum(X[:, 5], 0) + scale * 0.1 * rng.normal(size=B))
    return X, t.astype(np.float32)


def _split(P):
    o = 0
    out = {}
    for name, shape in (("W1", (128, 48)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)), ("W3", (128, 128)),
                        ("b3", (128,)), ("w4", (128,)), ("b4", ())):
        n = int(np.prod(shape)) if shape else 1
        out[name] = P[o:o + n].reshape(shape) if shape else float(P[o])
        o += n
    assert o == len(P)
    return out


U_BF16 = 2.0 ** -8   # BF16 round to nearest: relative error <= 2^-9; taken twice for margin
U_F32 = 2.0 ** -24


def _gamma(n):
    """Relative error bound of an FP32 sum of n terms (against the sum of
    their magnitudes), doubled over n u for the tensor cores' accumulation."""
    return 4.0 * n * U_F32


def _gradient_bounds(p, X, t):
    """Elementwise bounds on |GPU - float64 reference| for the loss and every
    gradient, by first-order forward error analysis of the training step as
    the kernels compute it: BF16 operands (X and the weights are the same BF16
    values on both sides), FP32 accumulation of every product and sum, h1, h2,
    h3 and the back-propagated errors G3, G2, G1 rounded to BF16 where they are
    stored between products (the bias gradients of the fused step are column
    sums of those stored BF16 values, taken on the tensor cores; the unfused
    path sums the FP32 values, which the same bound covers), a ReLU mask that
    may differ where |z| is within its error bound.  Returns (reference loss,
    reference gradients, loss bound, bounds)."""
    A = np.abs
    B = X.shape[0]
    y, c = MO.forward(p, X)
    ref_loss, ref = MO.loss_and_grads(p, X, t)
    z1, h1, z2, h2, z3, h3 = c["z1"], c["h1"], c["z2"], c["h2"], c["z3"], c["h3"]
    W1, W2, W3, w4 = p["W1"], p["W2"], p["W3"], p["w4"]
    # forward
    e_z1 = _gamma(48) * (A(X) @ A(W1).T + A(p["b1"]))
    e_h1 = e_z1 + U_BF16 * A(h1)
    e_z2 = e_h1 @ A(W2).T + _gamma(128) * (A(h1) @ A(W2).T + A(p["b2"]))
    e_h2 = e_z2 + U_BF16 * A(h2)
    e_z3 = e_h2 @ A(W3).T + _gamma(128) * (A(h2) @ A(W3).T + A(p["b3"]))
    e_h3 = e_z3 + U_BF16 * A(h3)
    e_y = e_h3 @ A(w4) + _gamma(128) * (A(h3) @ A(w4) + abs(p["b4"]))
    dy = (y - t) / B
    e_dy = e_y / B + 2 * U_F32 * A(dy)
    e_loss = float(np.sum(A(y - t) * e_y + 0.5 * e_y ** 2) / B + _gamma(B) * ref_loss)

    def masked(q, e_q, z, e_z):
        """Error of q * [z > 0] when the GPU's z may differ from z by e_z."""
        flip = A(z) <= e_z
        return np.where(flip, A(q) + e_q, np.where(z > 0, e_q, 0.0))

    # output layer and G3 = dy w4 [z3 > 0]
    q3 = np.outer(dy, w4)
    e_g3 = masked(q3, np.outer(e_dy, A(w4)), z3, e_z3)  # FP32 values (bias gradient)
    g3 = q3 * (z3 > 0)
    e_g3s = e_g3 + U_BF16 * A(g3)                          # as stored in BF16 (products)
    bnd = {}
    bnd["w4"] = (e_dy[:, None] * A(h3) + A(dy)[:, None] * e_h3 + e_dy[:, None] * e_h3).sum(0) + \
        _gamma(B) * (A(dy)[:, None] * A(h3)).sum(0)
    bnd["b4"] = float(e_dy.sum() + _gamma(B) * A(dy).sum())
    bnd["W3"] = e_g3s.T @ A(h2) + A(g3).T @ e_h2 + e_g3s.T @ e_h2 + _gamma(B) * (A(g3).T @ A(h2))
    bnd["b3"] = e_g3s.sum(0) + _gamma(B) * A(g3).sum(0)
    # G2 = (G3 W3) [z2 > 0]
    q2 = g3 @ W3
    e_q2 = e_g3s @ A(W3) + _gamma(128) * (A(g3) @ A(W3))
    e_g2 = masked(q2, e_q2, z2, e_z2)
    g2 = q2 * (z2 > 0)
    e_g2s = e_g2 + U_BF16 * A(g2)
    bnd["W2"] = e_g2s.T @ A(h1) + A(g2).T @ e_h1 + e_g2s.T @ e_h1 + _gamma(B) * (A(g2).T @ A(h1))
    bnd["b2"] = e_g2s.sum(0) + _gamma(B) * A(g2).sum(0)
    # G1 = (G2 W2) [z1 > 0]
    q1 = g2 @ W2
    e_q1 = e_g2s @ A(W2) + _gamma(128) * (A(g2) @ A(W2))
    e_g1 = masked(q1, e_q1, z1, e_z1)
    g1 = q1 * (z1 > 0)
    e_g1s = e_g1 + U_BF16 * A(g1)
    bnd["W1"] = e_g1s.T @ A(X) + _gamma(B) * (A(g1).T @ A(X))
    bnd["b1"] = e_g1s.sum(0) + _gamma(B) * A(g1).sum(0)
    return ref_loss, ref, e_loss, bnd


@pytest.mark.parametrize("unfused", [False, True])
def test_gradients_match_reference(env, unfused):
    """The fused step (every product of a 128-row tile in one kernel, weight
    gradients accumulated in tensor memory) and the one-product-per-launch
    path both meet the derived elementwise bound."""
    torch, crmc = env
    mlp = W.random_mlp(seed=21, out_gain=1.0)
    rng = np.random.default_rng(3)
    X, t = _batch(rng, 1024)
    tr = crmc.Trainer(mlp, max_batch=1024, unfused=unfused)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    torch.cuda.synchronize()
    loss, g = tr.gradients(Xd.data_ptr(), td.data_ptr(), 1024)
    p = MO.params_from_bf16(mlp, W.bf16_to_f32)
    Xq = W.bf16_to_f32(W.to_bf16_bits(X)).astype(np.float64)
    ref_loss, ref, e_loss, bnd = _gradient_bounds(p, Xq, t.astype(np.float64))
    assert abs(loss - ref_loss) <= e_loss, (loss, ref_loss, e_loss)
    G = _split(g)
    for name in MO.NAMES:
        a = np.atleast_1d(np.asarray(G[name], np.float64)).ravel()
        b = np.atleast_1d(np.asarray(ref[name], np.float64)).ravel()
        e = np.atleast_1d(np.asarray(bnd[name], np.float64)).ravel()
        err = np.abs(a - b)
        assert np.all(err <= e), (name, float(np.max(err / np.maximum(e, 1e-300))), float(err.max()))
        nb = np.linalg.norm(b)
        if nb > 0:  # the bound is not vacuous: the gradient is resolved
            assert float(a @ b / (np.linalg.norm(a) * nb)) > 0.999, name


def _adam_bounds(p64, m64, v64, grads, lr, beta1, beta2, eps):
    """Elementwise bounds on |GPU - float64 reference| of the masters and both
    Adam moments after each of the given gradient steps, for the FP32 update
    m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    p -= lr (m / c1) / (sqrt(v / c2) + eps): each FP32 operation rounds with
    relative error <= 2^-24, the hyperparameters and the bias corrections are
    rounded to FP32 once, and the errors of earlier steps carry over (scaled by
    b1, b2).  Returns a list of (bound_p, bound_m, bound_v), one per step."""
    u = U_F32
    e1 = abs(float(np.float32(beta1)) - beta1)
    e2 = abs(float(np.float32(beta2)) - beta2)
    n = len(p64)
    dm = np.zeros(n); dv = np.zeros(n); dp = np.zeros(n)
    m = m64.copy(); v = v64.copy(); p = p64.copy()
    out = []
    for k, g in enumerate(grads, start=1):
        g = g.astype(np.float64)
        a_m = beta1 * np.abs(m) + (1 - beta1) * np.abs(g)
        a_v = beta2 * v + (1 - beta2) * g * g
        dm = beta1 * dm + e1 * (np.abs(m) + np.abs(g)) + 4 * u * a_m
        dv = beta2 * dv + e2 * (v + g * g) + 6 * u * a_v
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        c1, c2 = 1 - beta1 ** k, 1 - beta2 ** k
        sv = np.sqrt(v / c2)
        den = sv + eps
        r = (m / c1) / den
        # error of the ratio from the moments' errors and its own roundings
        d_sv = np.where(sv > 0, (dv / c2) / (2 * np.maximum(sv, 1e-300)), np.sqrt(dv / c2))
        dr = (dm / c1) / den + np.abs(m / c1) * d_sv / den ** 2 + 10 * u * np.abs(r)
        p = p - lr * r
        dp = dp + lr * dr + 2 * u * lr * np.abs(r) + u * np.abs(p)
        out.append((dp.copy(), dm.copy(), dv.copy()))
    return out


def test_adam_update_matches_reference_elementwise(env):
    """cr_train_apply with given gradients against oracle adam_step: every
    FP32 master and both moments, after the first step and after ten."""
    torch, crmc = env
    lr, beta1, beta2, eps = 1e-3, 0.9, 0.999, 1e-8
    tr = crmc.Trainer(W.random_mlp(seed=31, gain=0.5), max_batch=128, lr=lr, beta1=beta1, beta2=beta2, eps=eps)
    P0, _ = tr.get()
    n = len(P0)
    rng = np.random.default_rng(8)
    mag = 10.0 ** rng.uniform(-5.0, 1.0, n)  # per-parameter gradient scale over six decades
    grads = []
    for k in range(10):
        g = (rng.normal(size=n) * mag).astype(np.float32)
        g[k::97] = 0.0  # some exact zeros
        if k == 3:
            g[::5] *= -1.0  # sign changes between steps
        grads.append(g)
    p = _split(P0.astype(np.float64))
    st = MO.adam_init(p)
    bounds = _adam_bounds(P0.astype(np.float64), np.zeros(n), np.zeros(n), grads, lr, beta1, beta2, eps)
    flat = lambda d: np.concatenate([np.atleast_1d(np.asarray(d[k], np.float64)).ravel() for k in MO.NAMES])
    for k, g in enumerate(grads, start=1):
        tr.apply(g)
        p = MO.adam_step(p, _split(g.astype(np.float64)), st, lr=lr, beta1=beta1, beta2=beta2, eps=eps)
        if k not in (1, 10):
            continue
        Pg, _ = tr.get()
        mg, vg = tr.moments()
        bp, bm, bv = bounds[k - 1]
        for name, got, want, b in (("params", Pg, flat(p), bp), ("m", mg, flat(st["m"]), bm),
                                   ("v", vg, flat(st["v"]), bv)):
            err = np.abs(got.astype(np.float64) - want)
            assert np.all(err <= b), (k, name, float(np.max(err / np.maximum(b, 1e-300))))
        # the update is resolved: the masters moved by about lr per step
        assert np.median(np.abs(Pg.astype(np.float64) - P0)) > 0.5 * lr
    steps, _ = tr.stats()
    assert steps == 10


def test_adam_steps_reduce_the_loss_like_the_reference(env):
    torch, crmc = env
    mlp = W.random_mlp(seed=22, gain=0.5, out_gain=1.0)
    rng = np.random.default_rng(4)
    X, t = _batch(rng, 512, scale=0.0)
    tr = crmc.Trainer(mlp, max_batch=512, lr=3e-3)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    torch.cuda.synchronize()
    p = MO.params_from_bf16(mlp, W.bf16_to_f32)
    st = MO.adam_init(p)
    Xq = W.bf16_to_f32(W.to_bf16_bits(X)).astype(np.float64)
    losses, ref_losses = [], []
    for k in range(150):
        losses.append(tr.step(Xd.data_ptr(), td.data_ptr(), 512, want_loss=(k % 10 == 0 or k == 149)))
        l, g = MO.loss_and_grads(p, Xq, t.astype(np.float64))
        ref_losses.append(l)
        p = MO.adam_step(p, g, st, lr=3e-3)
    l0, l_end = losses[0], losses[-1]
    assert l_end < 0.1 * l0, (l0, l_end)
    assert abs(l0 - ref_losses[0]) <= 2e-2 * ref_losses[0]
    assert l_end <= 3.0 * ref_losses[-1] + 1e-3, (l_end, ref_losses[-1])
    steps, launches = tr.stats()
    assert steps == 150 and launches == 150 * 2  # the fused step; the partials' sum with Adam and the BF16 copies


def test_trained_surrogate_keeps_da_parity(env):
    """Features and pair energies recorded by logged DA sweeps train the
    surrogate; the exported weights then drive a DA sweep that matches the
    oracle trial by trial."""
    torch, crmc = env
    w = W.config2(seed=6, scale=0.5)
    g = crmc.Context(w)
    g.set_surrogate(W.random_mlp(seed=23, out_gain=0.0))
    n = g.trials_per_sweep * 4
    r = g.sweep_da(n, 17, log=True, features=True)
    ok = (r["da"]["stage"] > 0) & np.isfinite(r["da"]["lnA2"])
    X = r["features"][ok]
    y = (r["da"]["dE_sur"][ok].astype(np.float64) - r["da"]["lnA2"][ok]).astype(np.float32)
    B = (len(X) // 128) * 128
    X = np.concatenate([X[:B], -X[:B]])  # the surrogate is antisymmetrised: train on both signs
    y = np.concatenate([y[:B], -y[:B]])
    tr = crmc.Trainer(W.random_mlp(seed=24, gain=0.5), max_batch=len(X), lr=2e-3)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    torch.cuda.synchronize()
    l0 = tr.step(Xd.data_ptr(), yd.data_ptr(), len(X), want_loss=True)
    for _ in range(100):
        l1 = tr.step(Xd.data_ptr(), yd.data_ptr(), len(X), want_loss=True)
    assert l1 < l0
    _, mlp = tr.get()
    w2 = W.config2(seed=7, scale=0.5)
    h = crmc.Context(w2)
    h.set_surrogate(mlp)
    m = h.trials_per_sweep * 2
    r2 = h.sweep_da(m, 19, log=True, features=True)
    o, lo, do, ties = compare_logs_da(w2, mlp, r2["log"], r2["da"], r2["features"], m, 19)
    compare_states(h, o, w2.n_sites)


def test_fused_step_over_many_tiles_per_cta(env):
    """A batch of more 128-row tiles than SMs (each CTA accumulates several
    tiles' weight gradients in tensor memory) gives the one-product-per-launch
    gradients within the sum of both paths' rounding (the derived bound
    against float64, applied to each)."""
    torch, crmc = env
    mlp = W.random_mlp(seed=25, out_gain=1.0)
    rng = np.random.default_rng(9)
    B = 128 * 400
    X, t = _batch(rng, B)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    torch.cuda.synchronize()
    p = MO.params_from_bf16(mlp, W.bf16_to_f32)
    Xq = W.bf16_to_f32(W.to_bf16_bits(X)).astype(np.float64)
    ref_loss, ref, e_loss, bnd = _gradient_bounds(p, Xq, t.astype(np.float64))
    for unfused in (False, True):
        tr = crmc.Trainer(mlp, max_batch=B, unfused=unfused)
        loss, g = tr.gradients(Xd.data_ptr(), td.data_ptr(), B)
        assert abs(loss - ref_loss) <= e_loss
        G = _split(g)
        for name in MO.NAMES:
            a = np.atleast_1d(np.asarray(G[name], np.float64)).ravel()
            b = np.atleast_1d(np.asarray(ref[name], np.float64)).ravel()
            e = np.atleast_1d(np.asarray(bnd[name], np.float64)).ravel()
            assert np.all(np.abs(a - b) <= e), (unfused, name)
        tr.close()
