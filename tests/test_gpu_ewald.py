"""Ewald electrostatics on the GPU (the paper's PPPM energy model, Sec. III.A,
evaluated as a direct Ewald sum) under the global schedule, trial by trial
against the oracle: moves, chosen ids and decisions identical, Delta E within
1e-6 of the gross term sum (the reciprocal part's FP32 terms and structure-
factor updates included), final states identical; batches of replicas equal
the per-replica oracle runs; the MD forces (real-space erfc plus reciprocal
part) equal the oracle's and MD/CR-MC cycles follow it; delayed acceptance,
the coloured schedule and the captured cycle are refused with Ewald."""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W
from parity_util import compare_logs, compare_states

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def _replica_seed(seed, r):
    return seed ^ (r << 32)


def _electrolyte(n_acid=30, L=20.0, rc=8.0, alpha=0.4, kmax=6, m=50, seed=3, pH=7.0):
    w = W.weak_acid_electrolyte(n_acid=n_acid, L=L, pH=pH, pKa=6.5, pIS=2.0, rc=rc, seed=seed,
                                trials_per_domain=m, alpha=alpha)
    w.params["ewald_kmax"] = kmax
    return w


@pytest.mark.parametrize("kmax,threads", [(6, 128), (6, 512), (12, 256)])
def test_ewald_trials_match_the_oracle(crmc, kmax, threads):
    w = _electrolyte(kmax=kmax)
    g = crmc.Context(w)
    g.set_launch_shape(threads, 0)
    n = g.trials_per_sweep * 8
    lg = g.sweep(n, 41, log=True)["log"]
    o, lo, ties = compare_logs(w, lg, n, 41)
    compare_states(g, o, w.n_sites)
    acc = (lo["flags"] & oracle.F_ACC) != 0
    assert acc.sum() > 20 and ties <= 2


def test_ewald_paper_electrolyte_box(crmc):
    """The method comparison's weak-acid electrolyte (500 acids, L = 50 l_B,
    r_c = 10 l_B) with a reciprocal sum over |n| <= 10."""
    w = _electrolyte(n_acid=500, L=100.0, rc=20.0, alpha=0.16, kmax=10, m=200, seed=1)
    g = crmc.Context(w)
    n = g.trials_per_sweep * 3
    lg = g.sweep(n, 5, log=True)["log"]
    o, lo, ties = compare_logs(w, lg, n, 5)
    compare_states(g, o, w.n_sites)


def test_ewald_batch_matches_oracle(crmc):
    ws = [_electrolyte(seed=s, pH=pH) for s, pH in ((5, 5.0), (6, 7.0), (7, 9.0))]
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(5, 88)
    for r, (w, g) in enumerate(zip(ws, ctxs)):
        o = oracle.Oracle(w)
        o.sweep(o.trials_per_sweep * 5, _replica_seed(88, r))
        compare_states(g, o, w.n_sites)
    b.close()


def test_ewald_refusals(crmc):
    w = _electrolyte()
    with pytest.raises(crmc.CrError) as e:
        crmc.Context(w, schedule=crmc.SCHED_COLOURED)
    assert e.value.code == -1
    g = crmc.Context(w)
    for f in (lambda: g.set_surrogate(W.random_mlp(seed=1)),):
        with pytest.raises(crmc.CrError) as e:
            f()
        assert e.value.code == -1
    b = crmc.Batch([g])
    with pytest.raises(crmc.CrError) as e:
        b.cycle(1, 0.005, 1.0, 1, 2)
    assert e.value.code == -1
    b.close()
    g.sweep(g.trials_per_sweep, 3)  # the context still works
    g.close()


F_REL = 4e-6  # FP32 force terms against FP64, relative to the gross sum of the terms


@pytest.mark.parametrize("box", ["small", "paper"])
def test_ewald_md_forces_match_oracle(crmc, box):
    if box == "small":
        w = _electrolyte()
    else:  # the method comparison's box, |n| <= 10
        w = _electrolyte(n_acid=500, L=100.0, rc=20.0, alpha=0.16, kmax=10, m=50, seed=1)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    n = g.trials_per_sweep * 6
    lg = g.sweep(n, 9, log=True)["log"]
    lo = o.sweep(n, 9, log=True)["log"]
    assert np.array_equal(lg["flags"], lo["flags"])
    g.md_forces()
    st = g.state()
    ids, F, S = o.forces()
    assert np.array_equal(st["id"], ids)
    err = np.abs(st["force"].astype(np.float64) - F)
    assert np.all(err <= F_REL * S + 2e-6), (np.argmax(err - F_REL * S), err.max())
    assert np.abs(F).max() > 0.05  # not vacuous


def _wrapdiff(a, b, L):
    d = a.astype(np.float64) - b.astype(np.float64)
    return d - L * np.round(d / L)


def test_ewald_md_cycles_match_oracle(crmc):
    """md_begin -> sweep -> md_end under Ewald: positions and velocities within the
    MD tolerances, the trials decision by decision (the oracle synchronised to the
    GPU's positions after the drift)."""
    w = _electrolyte(seed=4)
    w.vel = np.random.default_rng(4).normal(size=(w.n, 3)).astype(np.float32)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    L = float(np.float32(w.params["box_L"]))
    n = g.trials_per_sweep * 2
    for cyc in range(5):
        g.md_begin(0.005, 1.0, 31)
        o.md_begin(0.005, 1.0, 31)
        sg, so = g.state(), o.particles()
        assert np.array_equal(sg["id"], so["id"])
        assert np.abs(_wrapdiff(sg["xyz"], so["xyz"], L)).max() < 2e-5
        assert np.abs(sg["vel"] - so["vel"]).max() < 2e-4
        o.set_positions(sg["id"], sg["xyz"], sg["vel"])
        lg = g.sweep(n, 60 + cyc, log=True)["log"]
        lo = o.sweep(n, 60 + cyc, log=True)["log"]
        assert np.array_equal(lg["flags"], lo["flags"]) and np.array_equal(lg["id_a"], lo["id_a"])
        g.md_end(0.005, 1.0, 31)
        o.md_end(0.005, 1.0, 31)
        sg, so = g.state(), o.particles()
        assert np.array_equal(sg["id"], so["id"])
        assert np.abs(_wrapdiff(sg["xyz"], so["xyz"], L)).max() < 2e-5
        assert np.abs(sg["vel"] - so["vel"]).max() < 2e-4
    g.check()


def test_ewald_with_invocations_and_a_pH_change(crmc):
    """Grand-reaction invocations (salt ions as their own types) and a new
    reservoir pH between sweeps, under Ewald: trial by trial vs the oracle."""
    from paper_2109_07527_gb300 import methods
    w = _electrolyte(m=100)
    g = crmc.Context(w)
    n = g.trials_per_sweep * 2
    inv = methods.grand_reaction_invocations(7.0, 2.0, 2.0, reactions=1)
    steps = [(inv[0][0], 7.0), (inv[1][0], 7.0), (inv[2][0], 5.5), (inv[3][0], 5.5)]
    done = []
    for k, (args, pH) in enumerate(steps):
        seed = 70 + k
        g.set_pH(pH)
        g.set_invocation(*args)
        lg = g.sweep(n, seed, log=True)["log"]

        def prep(o, done=tuple(done), args=args, pH=pH):
            for (a, p), sd in done:
                o.set_pH(p)
                o.set_invocation(*a)
                o.sweep(n, sd)
            o.set_pH(pH)
            o.set_invocation(*args)
        o, lo, ties = compare_logs(w, lg, n, seed, prep=prep)
        compare_states(g, o, w.n_sites)
        done.append(((args, pH), seed))
    g.close()


def test_ewald_checkpoint_and_bound_buffers_continue_the_chain(crmc):
    """A checkpoint restored into a fresh context, and a context whose
    configuration lives in caller-owned device memory, both continue the
    unsplit Ewald chain bit for bit (S(k) is rebuilt from the state at every
    sweep)."""
    import torch
    w = _electrolyte(m=100)
    a, b = crmc.Context(w), crmc.Context(w)
    for s in range(3):
        a.sweep(a.trials_per_sweep, 10 + s)
        b.sweep(b.trials_per_sweep, 10 + s)
    ck = b.checkpoint()
    c = crmc.Context(w)
    c.restore(ck)
    i = c.info
    ncell, nslot = i["nc"] ** 3, i["nc"] ** 3 * i["cap"]
    t = dict(cnt=torch.zeros(ncell, dtype=torch.int32, device="cuda"),
             pos=torch.zeros(4 * nslot, dtype=torch.float32, device="cuda"),
             vel=torch.zeros(4 * nslot, dtype=torch.float32, device="cuda"),
             id=torch.zeros(nslot, dtype=torch.int64, device="cuda"),
             info=torch.zeros(nslot, dtype=torch.int32, device="cuda"))
    c.bind_device_buffers(t["cnt"].data_ptr(), t["pos"].data_ptr(), t["vel"].data_ptr(), t["id"].data_ptr(),
                          t["info"].data_ptr(), ncell, nslot)
    for s in range(3, 6):
        a.sweep(a.trials_per_sweep, 10 + s)
        c.sweep(c.trials_per_sweep, 10 + s)
    sa, sc = a.state(), c.state()
    for k in ("id", "xyz", "type", "state", "site_state"):
        assert np.array_equal(sa[k], sc[k]), k
    for g in (a, b, c):
        g.close()
