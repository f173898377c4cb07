"""Surrogate training on the tensor cores against the float64 reference
(oracle/mlp_oracle.py), through the C ABI.

  * the tcgen05 product D = A B^T equals the float64 product of the same BF16
    operands within FP32 accumulation error (tiles, a ragged M, a K that is not
    a multiple of the 64-wide stage, split-K accumulation, N = 48 and 128);
  * the loss and every gradient tensor match the reference within the BF16
    bound (activations are stored in BF16 between the products): cosine
    similarity > 0.999 and relative L2 error < 3e-2;
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


def test_gradients_match_reference(env):
    torch, crmc = env
    mlp = W.random_mlp(seed=21, out_gain=1.0)
    rng = np.random.default_rng(3)
    X, t = _batch(rng, 1024)
    tr = crmc.Trainer(mlp, max_batch=1024)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    torch.cuda.synchronize()
    loss, g = tr.gradients(Xd.data_ptr(), td.data_ptr(), 1024)
    p = MO.params_from_bf16(mlp, W.bf16_to_f32)
    Xq = W.bf16_to_f32(W.to_bf16_bits(X)).astype(np.float64)
    ref_loss, ref = MO.loss_and_grads(p, Xq, t.astype(np.float64))
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss + 1e-6, (loss, ref_loss)
    G = _split(g)
    for name in MO.NAMES:
        a = np.atleast_1d(np.asarray(G[name], np.float64)).ravel()
        b = np.atleast_1d(np.asarray(ref[name], np.float64)).ravel()
        nb = np.linalg.norm(b)
        if nb == 0:
            assert np.linalg.norm(a) <= 1e-6
            continue
        cos = float(a @ b / (np.linalg.norm(a) * nb + 1e-300))
        rel = float(np.linalg.norm(a - b) / nb)
        assert cos > 0.999 and rel < 3e-2, (name, cos, rel)


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
    assert steps == 150 and launches == 150 * 14


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
