"""Grand-reaction invocations on the GPU path against the oracle, through the
C ABI (cr_set_invocation; App. B: the scheme invoked repeatedly with
different types of ions; Sec. II.B: applied separately to dissociated and
salt ions, the grand-reaction ensemble):

  * a cycle of the four invocations -- (H+, OH-) acid and salt moves,
    (S+, S-) acid and salt moves, (H+, S-) and (S+, OH-) salt moves -- on the
    polyacid chain with interacting ions, trial by trial, both schedules;
  * a batch whose replicas run different invocations between batch sweeps
    ends in the states of the oracle runs with the same keys and invocations;
  * the salt ions of the other invocations stay as interacting bystanders:
    an RxMC invocation after them leaves their number unchanged;
  * bad invocation arguments are refused before anything runs.
"""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W
from parity_util import compare_logs, compare_states

pytestmark = pytest.mark.gpu

CR_ERR_INVALID_ARG = -1


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def invocations(w):
    """(cation, anion, pI_cation, pI_anion, reactions) of one grand-reaction cycle."""
    pH = float(w.params["pH"])
    pOH = float(w.params["pKw"]) - pH
    pSp, pSm = float(w.params["pIS_plus"]), float(w.params["pIS_minus"])
    return [(W.XP, W.XM, pH, pOH, 5), (W.SP, W.SM, pSp, pSm, 5), (W.XP, W.SM, pH, pSm, 4),
            (W.SP, W.XM, pSp, pOH, 4)]


@pytest.mark.parametrize("schedule,m", [(0, 10), (1, 400)])
def test_parity_grand_reaction_cycle(crmc, schedule, m):
    w = W.config1(seed=3, schedule=schedule, trials_per_domain=m)
    # a lower pI_S makes salt insertions frequent enough to populate S+- quickly
    w.params.update(pIS_plus=1.0, pIS_minus=1.0)
    g = crmc.Context(w)
    n = g.trials_per_sweep * (6 if schedule == 0 else 8)
    inv = invocations(w)
    done = []  # (invocation, seed) of the segments already compared

    def prep_to(k):
        def prep(o):
            for (c, a, pc, pa, r), sd in done:
                o.set_invocation(c, a, pc, pa, r)
                o.sweep(n, sd)
            o.set_invocation(*inv[k])
        return prep

    for cycle in range(2):
        for k in range(4):
            seed = 60 + 4 * cycle + k
            g.set_invocation(*inv[k])
            lg = g.sweep(n, seed, log=True)["log"]
            o, lo, ties = compare_logs(w, lg, n, seed, dict(schedule=schedule, trials_per_domain=m), prep=prep_to(k))
            compare_states(g, o, w.n_sites)
            done.append((inv[k], seed))
    c = g.counts()
    # salt ions were inserted, and the starting X+- (H+ and OH- under these
    # invocations, scarce in the reservoir at pH 5) were removed
    assert c["n_Sp"] > 0 and c["n_Sm"] > 0 and c["n_Xp"] < 64 and c["n_Xm"] < 64
    g.close()


def test_batch_replicas_follow_their_invocations(crmc):
    ws = [W.config2(seed=21, scale=0.5, pH=p) for p in (3.0, 5.0, 6.5)]
    for w in ws:
        w.params.update(pIS_plus=1.5, pIS_minus=1.5)
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    os_ = [oracle.Oracle(w) for w in ws]
    invs = [invocations(w) for w in ws]
    for k in range(4):
        for r, (g, o) in enumerate(zip(ctxs, os_)):
            j = (k + r) % 4  # the replicas are at different invocations
            g.set_invocation(*invs[r][j])
            o.set_invocation(*invs[r][j])
        b.sweep(2, 90 + k)
        for r, o in enumerate(os_):
            o.sweep(o.trials_per_sweep * 2, (90 + k) ^ (r << 32))
    for w, g, o in zip(ws, ctxs, os_):
        compare_states(g, o, w.n_sites)
    assert sum(g.counts()["n_Sp"] for g in ctxs) > 0
    b.close()


def test_bystander_salt_ions_are_kept_by_rxmc(crmc):
    w = W.config1(seed=5)
    w.params.update(pIS_plus=1.0, pIS_minus=1.0)
    g = crmc.Context(w)
    inv = invocations(w)
    g.set_invocation(*inv[1])  # (S+, S-): inserts salt ions
    g.sweep(g.trials_per_sweep * 6, 1)
    c0 = g.counts()
    assert c0["n_Sp"] > 0
    g.set_invocation(*inv[0])  # RxMC: H+ / OH- only
    g.sweep(g.trials_per_sweep * 6, 2)
    c1 = g.counts()
    assert (c1["n_Sp"], c1["n_Sm"]) == (c0["n_Sp"], c0["n_Sm"])
    assert c1["net_charge"] == 0
    g.close()


def test_invocation_arguments_are_refused(crmc):
    w = W.config1(seed=2)
    g = crmc.Context(w)
    for args in ((W.ACID, W.XM, 2.0, 2.0, 7), (W.XP, W.SP, 2.0, 2.0, 7), (W.XP, W.XM, float("inf"), 2.0, 7),
                 (W.XP, W.XM, 2.0, 2.0, 0), (W.XP, W.XM, 2.0, 2.0, 2), (W.XP, W.XM, 2.0, 2.0, 8)):
        with pytest.raises(crmc.CrError) as e:
            g.set_invocation(*args)
        assert e.value.code == CR_ERR_INVALID_ARG
    # the context still runs the default chain of the oracle
    g.sweep(g.trials_per_sweep * 2, 7)
    o = oracle.Oracle(w)
    o.sweep(o.trials_per_sweep * 2, 7)
    compare_states(g, o, w.n_sites)
    g.close()


def test_method_comparison_reproduces_fig2_qualitatively(crmc):
    """Sec. III.A / Fig. 2 on the weak-acid electrolyte (500 acids, pKa 6.5,
    pH 7, pI_S = 2, L = 50 l_B), the same random starts for every method:
    CR-MC and the grand-reaction ensemble reach the same degree of
    dissociation, CR-MC several times sooner (most grand-reaction moves
    involve the nearly absent H+ or OH- and are rejected), and RxMC stays far
    from it (without salt ions at pH 7)."""
    from paper_2109_07527_gb300 import methods
    r = methods.compare_convergence(crmc, n_rep=32, blocks=16, m=250, seed=1)
    cr, gr, rx = (np.array(r[k]) for k in ("crmc", "grxmc", "rxmc"))
    final = cr[-6:].mean()
    assert 0.3 < final < 0.95
    assert abs(gr[-6:].mean() - final) < 0.02, (gr[-6:], final)
    assert rx[-6:].mean() < 0.2 * final, rx[-6:]
    # after 2 blocks (3000 trials per replica)
    assert cr[1] > 0.9 * final and gr[1] < 0.8 * final, (cr[:4], gr[:4], final)
