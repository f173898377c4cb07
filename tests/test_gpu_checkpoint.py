"""Checkpoint / resume through the C ABI: a run split by cr_checkpoint and
cr_restore into a fresh context continues the unsplit chain bit for bit --
particle ids (inserted ions >= 2^32), positions, velocities, charge states --
whether the split falls between MD/CR-MC cycles (the integrator's forces carry
over) or inside an MD step, after its drift (no forces yet)."""
import numpy as np
import pytest

from paper_2109_07527_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DT, GAMMA = 0.005, 1.0


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def _cycle(g, s):
    g.md_begin(DT, GAMMA, 500 + s)
    g.sweep(g.trials_per_sweep, 100 + s)
    g.md_end(DT, GAMMA, 500 + s)


def _same(a, b):
    for k in ("id", "xyz", "vel", "type", "state", "cls", "site_state"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("n", "n_Am", "n_Xp", "n_Xm"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("split", ["between_cycles", "inside_md_step"])
def test_split_run_equals_unsplit(crmc, split):
    w = W.config2(seed=4, scale=0.5)
    a = crmc.Context(w)  # unsplit
    b = crmc.Context(w)  # runs to the split and is checkpointed
    for s in range(3):
        _cycle(a, s)
        _cycle(b, s)
    if split == "inside_md_step":
        a.md_begin(DT, GAMMA, 900)
        b.md_begin(DT, GAMMA, 900)
    ck = b.checkpoint()
    assert ck["forces_valid"] == (1 if split == "between_cycles" else 0)
    assert ck["sweep"] == 3 and (ck["id"] >= 2 ** 32).any()  # inserted ions are in it
    _same(b.state(), a.state())
    b.close()
    c = crmc.Context(w)
    c.restore(ck)
    _same(c.state(), a.state())
    if split == "inside_md_step":
        for g in (a, c):
            g.sweep(g.trials_per_sweep, 901)
            g.md_end(DT, GAMMA, 900)
    for s in range(3, 6):
        _cycle(a, s)
        _cycle(c, s)
    _same(c.state(), a.state())
    a.close()
    c.close()


def test_restore_rejects_inconsistent_ids(crmc):
    w = W.config1(seed=2)
    g = crmc.Context(w)
    g.sweep(g.trials_per_sweep * 2, 3)
    ck = g.checkpoint()
    h = crmc.Context(w)
    bad = dict(ck)
    bad["id"] = ck["id"].copy()
    bad["id"][1] = bad["id"][0]  # a duplicate id, and particle 1 missing
    with pytest.raises(crmc.CrError):
        h.restore(bad)
    h.restore(ck)  # the consistent checkpoint is accepted
    assert np.array_equal(h.state()["id"], ck["id"])
    g.close()
    h.close()
