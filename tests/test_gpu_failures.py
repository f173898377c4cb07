"""Failure detection on the GPU without a GPU fault (through the C ABI).

  * the bounded mbarrier waits of the tensor-core product run out when an
    operand copy is withheld (cr_selftest_mma_timeout): the call returns
    CR_ERR_TIMEOUT, the output is untouched, and the next product on the same
    stream is correct -- the CTA freed its tensor memory and the context
    stayed usable;
  * the bounded dependency waits of the persistent batch sweep run out when
    one replica withholds its colour-0 completion
    (cr_batch_selftest_wait_timeout): CR_ERR_TIMEOUT within about the given
    limit, and the device runs a following batch sweep exactly;
  * a FENE bond stretched to R0 by a loaded configuration is reported as
    CR_ERR_BOND_BROKEN by the next force evaluation (the error word of the
    force kernel), not as a NaN force.
"""
import numpy as np
import pytest

from paper_2109_07527_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CR_ERR_TIMEOUT = -5
CR_ERR_BOND_BROKEN = -6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_07527_gb300 import crmc
    crmc._lib()
    return torch, crmc


def _bf16(torch, a):
    bits = W.to_bf16_bits(np.asarray(a, np.float32))
    return torch.from_numpy(bits.view(np.int16).copy()).cuda(), W.bf16_to_f32(bits).astype(np.float64)


def test_mma_bounded_wait_expires_and_the_context_recovers(env):
    torch, crmc = env
    rng = np.random.default_rng(1)
    A, Af = _bf16(torch, rng.normal(size=(128, 64)))
    B, Bf = _bf16(torch, rng.normal(size=(128, 64)))
    D = torch.full((128, 128), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    for polls in (1 << 12, 1 << 16):  # twice in a row, two limits
        assert crmc.selftest_mma_timeout(A.data_ptr(), B.data_ptr(), D.data_ptr(), polls) == CR_ERR_TIMEOUT
        assert torch.isnan(D).all().item()  # the timed-out CTA wrote nothing
    # the same product without the withheld copy
    crmc.mma_bf16(A.data_ptr(), B.data_ptr(), D.data_ptr(), 128, 128, 64)
    got = D.cpu().numpy().astype(np.float64)
    ref = Af @ Bf.T
    assert np.all(np.abs(got - ref) <= 2e-6 * (np.abs(Af) @ np.abs(Bf).T) + 1e-6)


def test_stretched_bond_is_reported(env):
    torch, crmc = env
    w = W.config1(seed=4)
    g = crmc.Context(w)
    st = g.state()
    i, j = [int(x) for x in w.bonds[0]]
    xyz = st["xyz"].copy()
    L = float(w.params["box_L"])
    d = xyz[j].astype(np.float64) - xyz[i]
    d -= L * np.round(d / L)
    # move j along the bond to 1.6 sigma from i (R0 = 1.5)
    xyz[j] = np.mod(xyz[i] + d / np.linalg.norm(d) * 1.6, L).astype(np.float32)
    g.load(len(st["id"]), xyz, st["vel"], st["type"], st["cls"], st["state"])
    with pytest.raises(crmc.CrError) as e:
        g.md_forces()
    assert e.value.code == CR_ERR_BOND_BROKEN
    g.close()
    h = crmc.Context(w)  # the device is fine: a new context evaluates forces
    h.md_forces()
    assert np.isfinite(h.state()["force"]).all()
    h.close()


def test_persistent_sweep_wait_expires_and_the_device_recovers(env):
    import time

    import oracle
    from parity_util import compare_states
    torch, crmc = env
    ws = [W.config2(seed=13, scale=0.5, pH=p) for p in (3.0, 5.0, 7.0)]
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    t0 = time.perf_counter()
    assert b.selftest_wait_timeout(1, 50.0) == CR_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0  # one bounded wait, then the rest skipped
    with pytest.raises(crmc.CrError) as e:
        ctxs[1].check()
    assert e.value.code == CR_ERR_TIMEOUT
    b.close()
    # a new batch on the same device runs the oracle's chain
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(2, 8)
    for r, (w, g) in enumerate(zip(ws, ctxs)):
        o = oracle.Oracle(w)
        o.sweep(o.trials_per_sweep * 2, 8 ^ (r << 32))
        compare_states(g, o, w.n_sites)
    b.close()
