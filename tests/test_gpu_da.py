"""GPU delayed-acceptance path (through the C ABI) against the oracle, trial by trial.

Features and the surrogate dE~ must be bit-exact, stage decisions identical up
to ties (see parity_util.compare_logs_da), dE within the parity tolerance, and
the final charge states identical.  Also: every DA launch shape gives the same
chain, unlogged DA sweeps (which skip the exact sum after a stage-1 rejection)
give the same chain as logged ones, and a batch of replicas equals independent
oracle runs.
"""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W
from parity_util import compare_logs_da, compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def _da_parity(crmc, w, mlp, sweeps, seed, **kw):
    g = crmc.Context(w, **kw)
    g.set_surrogate(mlp)
    n = g.trials_per_sweep * sweeps
    r = g.sweep_da(n, seed, log=True, features=True)
    okw = {k: v for k, v in kw.items() if k in ("schedule", "trials_per_domain", "domain_cells")}
    o, lo, do, ties = compare_logs_da(w, mlp, r["log"], r["da"], r["features"], n, seed, okw)
    compare_states(g, o, w.n_sites)
    return g, r, do, ties


@pytest.mark.parametrize("out_gain", [2.0, 0.0])
def test_da_parity_chain(crmc, out_gain):
    w = W.config1(seed=7)
    g, r, do, ties = _da_parity(crmc, w, W.random_mlp(seed=11, out_gain=out_gain), 6, 21)
    st = r["da"]["stage"]
    assert (st == 1).sum() > 0 and (st == 2).sum() > 0  # both stage outcomes occur
    assert ties <= 2


def test_da_parity_polyelectrolyte_half_box(crmc):
    w = W.config2(seed=2, scale=0.5)
    _da_parity(crmc, w, W.random_mlp(seed=12, out_gain=1.5), 2, 5)


def test_da_parity_nanoparticles(crmc):
    w = W.config3(separation=12.0, seed=1, n_sites=200)
    _da_parity(crmc, w, W.random_mlp(seed=13, out_gain=1.0), 1, 8)


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_da_launch_shapes_give_the_same_chain(crmc, threads):
    w = W.config2(seed=3, scale=0.5)
    mlp = W.random_mlp(seed=14, out_gain=1.5)
    ref = crmc.Context(w)
    ref.set_surrogate(mlp)
    ref.set_launch_shape(128, 0)
    n = ref.trials_per_sweep * 2
    a = ref.sweep_da(n, 33, log=True, features=True)
    g = crmc.Context(w)
    g.set_surrogate(mlp)
    g.set_launch_shape(threads, 0)
    b = g.sweep_da(n, 33, log=True, features=True)
    for f in ("flags", "id_a", "id_b"):
        assert np.array_equal(a["log"][f], b["log"][f])
    assert np.array_equal(a["da"]["dE_sur"], b["da"]["dE_sur"])
    assert np.array_equal(a["features"], b["features"])
    assert np.array_equal(a["log"]["dE"], b["log"]["dE"])  # exact fixed-point sums


def test_unlogged_da_sweeps_follow_the_logged_chain(crmc):
    """Unlogged DA sweeps skip the exact sum after a stage-1 rejection; the
    chain must not change (states compared bitwise after several sweeps)."""
    w = W.config2(seed=4, scale=0.5)
    mlp = W.random_mlp(seed=15, out_gain=1.5)
    a = crmc.Context(w)
    a.set_surrogate(mlp)
    b = crmc.Context(w)
    b.set_surrogate(mlp)
    n = a.trials_per_sweep * 3
    ra = a.sweep_da(n, 44, stats=True)
    rb = b.sweep_da(n, 44, stats=True, log=True)
    sa, sb = a.state(), b.state()
    for k in ("id", "xyz", "type", "state"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(ra["stats"]["accepts"], rb["stats"]["accepts"])
    assert np.array_equal(ra["stats"]["attempts"], rb["stats"]["attempts"])


def test_da_batch_matches_independent_oracle_runs(crmc):
    ws = [W.config2(seed=5, scale=0.5, pH=pH) for pH in (3.5, 5.5)]
    mlps = [W.random_mlp(seed=16 + i, out_gain=1.5) for i in range(2)]
    ctxs = [crmc.Context(w) for w in ws]
    for c, m in zip(ctxs, mlps):
        c.set_surrogate(m)
    b = crmc.Batch(ctxs)
    b.sweep_da(2, 77)
    for r, (w, m, c) in enumerate(zip(ws, mlps, ctxs)):
        o = oracle.Oracle(w)
        o.set_surrogate(m)
        o.set_da(True)
        o.sweep(o.trials_per_sweep * 2, 77 ^ (r << 32))
        compare_states(c, o, w.n_sites)


def test_da_rejects_unsupported_geometry(crmc):
    w = W.config1(seed=1, schedule=1, trials_per_domain=64)  # global schedule
    g = crmc.Context(w)
    with pytest.raises(crmc.CrError):
        g.set_surrogate(W.random_mlp(seed=1))
    g2 = crmc.Context(W.config1(seed=1))
    with pytest.raises(crmc.CrError):
        g2.sweep_da(g2.trials_per_sweep, 1)  # no surrogate loaded


def test_da_parity_with_lists_beyond_shared_memory(crmc):
    w = W.config2(seed=9, scale=0.5)
    _da_parity(crmc, w, W.random_mlp(seed=18, out_gain=1.5), 2, 13, list_capacity=8, halo_capacity=64)


def test_da_parity_config5_full_size(crmc):
    """The large delayed-acceptance system at full size (100 chains x 200, L =
    250, ~70 000 particles), one sweep of one trial per domain (8000 trials):
    features, dE~, stage decisions and charge states against the oracle."""
    w = W.config5(seed=3)
    w.params["trials_per_domain"] = 1
    g, r, do, ties = _da_parity(crmc, w, W.random_mlp(seed=31, out_gain=1.0), 1, 5)
    st = r["da"]["stage"]
    assert (st == 1).sum() > 0 and (st == 2).sum() > 0
    assert ties <= 2
