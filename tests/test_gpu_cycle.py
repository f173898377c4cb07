"""The MD step split around CR-MC calls (one force evaluation per MD/CR-MC
cycle), through the C ABI, against the oracle's split step.

  * md_begin + md_end with nothing in between equals md_step, bitwise;
  * cycles begin -> CR-MC sweeps -> end match the oracle: the trials decision
    by decision (the oracle is synchronised to the GPU positions after the
    drift, where MD has rounded differently), then positions and velocities
    within the MD tolerances after the closing kick;
  * a batch of replicas equals the same calls on each context alone.
"""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W
from parity_util import STRUCT_FLAGS, de_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def _wrapdiff(a, b, L):
    d = a.astype(np.float64) - b.astype(np.float64)
    return d - L * np.round(d / L)


def test_split_step_equals_md_step(crmc):
    w = W.config1(seed=9, n_pairs=16)
    a, b = crmc.Context(w), crmc.Context(w)
    a.sweep(a.trials_per_sweep, 3)
    b.sweep(b.trials_per_sweep, 3)
    for s in range(3):
        a.md_step(1, 0.005, 1.0, 77)
        b.md_begin(0.005, 1.0, 77)
        b.md_end(0.005, 1.0, 77)
    sa, sb = a.state(), b.state()
    for k in ("id", "xyz", "vel"):
        assert np.array_equal(sa[k], sb[k]), k


def test_cycles_match_oracle(crmc):
    w = W.config1(seed=6, n_pairs=32)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    L = float(np.float32(w.params["box_L"]))
    n = g.trials_per_sweep * 2
    inserted = 0
    for cyc in range(5):
        g.md_begin(0.005, 1.0, 77)
        o.md_begin(0.005, 1.0, 77)
        sg, so = g.state(), o.particles()
        assert np.array_equal(sg["id"], so["id"])
        assert np.abs(_wrapdiff(sg["xyz"], so["xyz"], L)).max() < 2e-5
        assert np.abs(sg["vel"] - so["vel"]).max() < 2e-4
        o.set_positions(sg["id"], sg["xyz"], sg["vel"])
        lg = g.sweep(n, 10 + cyc, log=True)["log"]
        lo = o.sweep(n, 10 + cyc, log=True)["log"]
        assert np.array_equal(lg["move"], lo["move"])
        assert np.array_equal(lg["flags"] & STRUCT_FLAGS, lo["flags"] & STRUCT_FLAGS)
        assert np.array_equal(lg["flags"], lo["flags"]), np.flatnonzero(lg["flags"] != lo["flags"])[:4]
        assert np.array_equal(lg["id_a"], lo["id_a"]) and np.array_equal(lg["id_b"], lo["id_b"])
        ok = (lo["flags"] & STRUCT_FLAGS) == 0
        assert np.all(np.abs(lg["dE"][ok] - lo["dE"][ok]) <= de_tol(lo[ok]))
        inserted += int(np.sum((lg["flags"] & oracle.F_ACC) != 0))
        g.md_end(0.005, 1.0, 77)
        o.md_end(0.005, 1.0, 77)
        sg, so = g.state(), o.particles()
        assert np.array_equal(sg["id"], so["id"])
        assert np.abs(_wrapdiff(sg["xyz"], so["xyz"], L)).max() < 2e-5
        assert np.abs(sg["vel"] - so["vel"]).max() < 2e-4  # includes inserted ions' drawn velocities
    assert inserted > 0


def test_batch_split_step_equals_single_contexts(crmc):
    ws = [W.config2(seed=8, scale=0.5, pH=pH) for pH in (3.0, 6.0)]
    single = [crmc.Context(w) for w in ws]
    batched = [crmc.Context(w) for w in ws]
    b = crmc.Batch(batched)
    for cyc in range(3):
        b.md_begin(0.005, 1.0, 40 + cyc)
        b.sweep(1, 50 + cyc)
        b.md_end(0.005, 1.0, 40 + cyc)
        for r, c in enumerate(single):
            c.md_begin(0.005, 1.0, (40 + cyc) ^ (r << 32))
            c.sweep(c.trials_per_sweep, (50 + cyc) ^ (r << 32))
            c.md_end(0.005, 1.0, (40 + cyc) ^ (r << 32))
    for c1, c2 in zip(single, batched):
        s1, s2 = c1.state(), c2.state()
        for k in ("id", "xyz", "vel", "state"):
            assert np.array_equal(s1[k], s2[k]), k


@pytest.mark.parametrize("mode", [0, 1])
def test_graph_cycle_equals_calls(crmc, mode):
    """cr_batch_cycle (one CUDA graph launch per step once tuned, the step's
    seeds and counters read from device memory) equals the same cycles made
    call by call -- md_begin, sweep, md_end with seeds seed0 + s -- bit for
    bit, for per-colour and persistent sweeps, and across two calls (the graph
    reused with new seeds)."""
    ws = [W.config2(seed=14, scale=0.5, pH=p) for p in (3.0, 4.5, 6.0)]
    runs = []
    for graph in (True, False):
        ctxs = [crmc.Context(w) for w in ws]
        b = crmc.Batch(ctxs)
        b.set_persistent(mode)
        b.set_launch_shape(64, 0)
        if graph:
            b.cycle(2, 0.005, 1.0, 100, 500)  # the first step runs call by call (no forces yet)
            ctxs[0].timing(reset=True)
            b.cycle(4, 0.005, 1.0, 102, 502)
            assert ctxs[0].timing(reset=True)["launches"] > 0  # the graph's kernels are counted
        else:
            for s in range(6):
                b.md_begin(0.005, 1.0, 500 + s)
                b.sweep(1, 100 + s)
                b.md_end(0.005, 1.0, 500 + s)
        for g in ctxs:
            g.check()
        runs.append([g.state() for g in ctxs])
        b.close()
    for a, c in zip(*runs):
        for k in ("id", "xyz", "vel", "state"):
            assert np.array_equal(a[k], c[k]), k


@pytest.mark.parametrize("mode,da", [(0, False), (1, False), (0, True)])
def test_graph_cycle_after_a_load_equals_calls(crmc, mode, da):
    """A cycle whose forces are stale (every replica just loaded, as in a
    coupling that uploads the configuration each step) runs its first step
    from the graph that evaluates the forces first, then the step's own graph:
    bit for bit the calls md_begin (which evaluates them), sweep, md_end; also
    with delayed-acceptance sweeps."""
    ws = [W.config2(seed=15, scale=0.5, pH=p) for p in (3.5, 5.0)]
    runs = []
    for graph in (True, False):
        ctxs = [crmc.Context(w) for w in ws]
        if da:
            for g in ctxs:
                g.set_surrogate(W.random_mlp(seed=16, out_gain=1.5))
        b = crmc.Batch(ctxs)
        b.set_persistent(mode)
        b.set_launch_shape(128 if da else 64, 0)  # a shape of both sets: no tuning, so the graphs run
        step = 0
        for it in range(3):
            for g in ctxs:  # reload each replica's own state: the forces become stale
                st = g.state()
                g.load(st["n"], *[np.ascontiguousarray(st[k]) for k in ("xyz", "vel", "type", "cls", "state")])
            if graph:
                ctxs[0].timing(reset=True)
                b.cycle(2, 0.005, 1.0, 100 + step, 500 + step, da=da)
                assert ctxs[0].timing(reset=True)["launches"] > 0
            else:
                for s in range(2):
                    b.md_begin(0.005, 1.0, 500 + step + s)
                    if da:
                        b.sweep_da(1, 100 + step + s)
                    else:
                        b.sweep(1, 100 + step + s)
                    b.md_end(0.005, 1.0, 500 + step + s)
            step += 2
        for g in ctxs:
            g.check()
        runs.append([g.state() for g in ctxs])
        b.close()
    for a, c in zip(*runs):
        for k in ("id", "xyz", "vel", "state"):
            assert np.array_equal(a[k], c[k]), k
