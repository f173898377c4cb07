"""Reservoir chemistry on the GPU path against the oracle, through the C ABI.

  * the conventional reaction ensemble (RxMC, pI_X+ = pH and pI_X- = pOH
    given explicitly; App. B) on interacting sites with explicit ions, trial by
    trial;
  * a time-dependent pH (App. B): sweeps at one pH, cr_set_pH, sweeps at
    another -- trial by trial against the oracle doing the same, for one
    context and for a batch whose replicas change pH between sweeps;
  * the ungrouped subspecies fractions (Sec. II.D) equal the oracle's, and
    their expected numbers follow the context's ion counts.
"""
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


def _rxmc(w):
    pH = float(w.params["pH"])
    w.params.update(pIX_explicit=1, pIX_plus=pH, pIX_minus=float(w.params["pKw"]) - pH)
    return w


def test_parity_rxmc_explicit_ion_chemical_potentials(crmc):
    """RxMC as the special case of CR-MC with pI_X+ = pH, pI_X- = pOH: the
    polyacid chain with interacting ions, both schedules."""
    for schedule, m in ((0, 10), (1, 400)):
        w = _rxmc(W.config1(seed=2, schedule=schedule, trials_per_domain=m))
        g = crmc.Context(w)
        n = g.trials_per_sweep * (12 if schedule == 0 else 15)
        lg = g.sweep(n, 21, log=True)["log"]
        o, lo, ties = compare_logs(w, lg, n, 21, dict(schedule=schedule, trials_per_domain=m))
        compare_states(g, o, w.n_sites)
        assert (lg["flags"] & 1).sum() > 20
        g.close()


def test_parity_ph_changed_between_sweeps(crmc):
    """pH 3.5 -> 6.0 -> 4.5 between sweeps of the half-size polyelectrolyte box
    (acids and, through pIXgen, both reservoir ions change), trial by trial."""
    w = W.config2(seed=9, scale=0.5, pH=3.5)
    g = crmc.Context(w)
    n = g.trials_per_sweep * 2
    done = []  # (pH, seed) of the segments already compared

    def prep(o):
        for pH, sd in done:
            o.set_pH(pH)
            o.sweep(n, sd)

    for k, pH in enumerate((3.5, 6.0, 4.5)):
        if k:
            g.set_pH(pH)
        lg = g.sweep(n, 40 + k, log=True)["log"]
        cur = pH

        def prep_k(o, cur=cur):
            prep(o)
            o.set_pH(cur)

        o, lo, ties = compare_logs(w, lg, n, 40 + k, prep=prep_k)
        done.append((pH, 40 + k))
    compare_states(g, o, w.n_sites)
    g.close()


def test_batch_follows_ph_changes_of_its_contexts(crmc):
    """Replicas of a batch change pH between batch sweeps (cr_set_pH on the
    contexts); each replica equals the oracle run with its key and pH
    schedule."""
    ws = [W.config2(seed=10, scale=0.5, pH=p) for p in (3.0, 5.0)]
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    os_ = [oracle.Oracle(w) for w in ws]
    sched = [(3.0, 5.0), (6.5, 4.0)]
    for k in range(2):
        for r, (g, o) in enumerate(zip(ctxs, os_)):
            if k:
                g.set_pH(sched[k][r])
                o.set_pH(sched[k][r])
        b.sweep(2, 70 + k)
        for r, o in enumerate(os_):
            o.sweep(o.trials_per_sweep * 2, (70 + k) ^ (r << 32))
    for w, g, o in zip(ws, ctxs, os_):
        compare_states(g, o, w.n_sites)
    b.close()


@pytest.mark.parametrize("pH", [3.0, 7.0, 9.5])
def test_ungrouped_fractions(crmc, pH):
    w = W.config1(seed=3)
    w.params["pH"] = pH
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    g.sweep(g.trials_per_sweep * 4, 5)
    u, uo, c = g.ungroup(), o.ungroup(), g.counts()
    for a, b in (("p_S_plus", "p_Sp"), ("p_H", "p_H"), ("p_S_minus", "p_Sm"), ("p_OH", "p_OH")):
        assert abs(u[a] - uo[b]) <= 1e-12 * max(1.0, abs(uo[b])), (a, u[a], uo[b])
    assert u["n_H"] == pytest.approx(u["p_H"] * c["n_Xp"], rel=1e-15)
    assert u["n_OH"] == pytest.approx(u["p_OH"] * c["n_Xm"], rel=1e-15)
    g.set_pH(pH + 1.0)
    o.set_pH(pH + 1.0)
    u, uo = g.ungroup(), o.ungroup()
    assert abs(u["p_H"] - uo["p_H"]) <= 1e-12 and abs(u["p_OH"] - uo["p_OH"]) <= 1e-12
    g.close()
