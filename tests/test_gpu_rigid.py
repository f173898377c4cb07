"""Rigid bodies on the GPU (cr_set_rigid_bodies): the nanoparticles of the
two-nanoparticle system move as rigid bodies, against the oracle.

  * the body setup (centre, principal frame, moments, momenta) equals the
    oracle's;
  * MD/CR-MC cycles (md_begin -> sweep -> md_end) match the oracle: body
    states and member positions within the MD tolerances after each half of
    the step, the trials decision by decision (the oracle is synchronised to
    the GPU's positions and bodies after the drift), also at the full size of
    the system (2 x 1000 sites, L = 100);
  * md_step equals md_begin + md_end bit for bit; members keep their
    distances over many steps and the orientations stay orthonormal;
  * bad declarations and calls that would lose the bodies are refused.
"""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W
from parity_util import STRUCT_FLAGS, de_tol

pytestmark = pytest.mark.gpu

DT, GAMMA = 0.005, 0.05  # Sec. IV.B: Langevin damping time 20 tau


@pytest.fixture(scope="module")
def crmc():
    from paper_2109_07527_gb300 import crmc as m
    m._lib()
    return m


def _wrapdiff(a, b, L):
    d = a.astype(np.float64) - b.astype(np.float64)
    return d - L * np.round(d / L)


def _pair(seed=2, n_sites=40, L=40.0, R=3.0, separation=9.0):
    w = W.config3(separation=separation, n_sites=n_sites, L=L, R=R, seed=seed)
    sites = np.flatnonzero((w.type == W.ACID) | (w.type == W.BASE))
    w.state[sites[w.type[sites] == W.ACID][::2]] = 1
    w.state[sites[w.type[sites] == W.BASE][::2]] = 1
    rng = np.random.default_rng(seed)
    w.vel = (rng.normal(size=(w.n, 3)) * 0.7).astype(np.float32)
    return w


def _same_bodies(bg, bo, L):
    assert bg.shape == bo.shape
    assert np.all(np.abs(_wrapdiff(bg[:, 0:3], bo[:, 0:3], L)) < 2e-5)
    assert np.allclose(bg[:, 3:6], bo[:, 3:6], atol=1e-5)
    assert np.allclose(bg[:, 6:15], bo[:, 6:15], atol=1e-6)
    assert np.allclose(bg[:, 15:18], bo[:, 15:18], atol=1e-4 * np.abs(bo[:, 15:18]).max() + 1e-6)
    assert np.allclose(bg[:, 18:22], bo[:, 18:22], rtol=1e-9)


def _same_particles(sg, so, L):
    assert np.array_equal(sg["id"], so["id"])
    assert np.abs(_wrapdiff(sg["xyz"], so["xyz"], L)).max() < 2e-5
    assert np.abs(sg["vel"] - so["vel"]).max() < 2e-4


def test_setup_matches_oracle(crmc):
    w = _pair()
    g, o = crmc.Context(w), oracle.Oracle(w)
    first, count = w.meta["bodies"]
    g.set_rigid_bodies(first, count)
    o.set_bodies(first, count)
    L = float(np.float32(w.params["box_L"]))
    bg, bo = g.rigid_body_state(), o.body_state()
    _same_bodies(bg, bo, L)
    assert np.all(bo[:, 21] == count)
    _same_particles(g.state(), o.particles(), L)  # members now move rigidly on both sides


def _cycles(crmc, w, n_cyc, trials_mult=2):
    g, o = crmc.Context(w), oracle.Oracle(w)
    first, count = w.meta["bodies"]
    g.set_rigid_bodies(first, count)
    o.set_bodies(first, count)
    L = float(np.float32(w.params["box_L"]))
    n = g.trials_per_sweep * trials_mult
    x0 = g.rigid_body_state()[:, 0:3]
    acc = 0
    for cyc in range(n_cyc):
        g.md_begin(DT, GAMMA, 77)
        o.md_begin(DT, GAMMA, 77)
        _same_bodies(g.rigid_body_state(), o.body_state(), L)
        sg = g.state()
        _same_particles(sg, o.particles(), L)
        o.set_positions(sg["id"], sg["xyz"], sg["vel"])
        o.set_body_state(g.rigid_body_state())
        lg = g.sweep(n, 10 + cyc, log=True)["log"]
        lo = o.sweep(n, 10 + cyc, log=True)["log"]
        assert np.array_equal(lg["move"], lo["move"])
        assert np.array_equal(lg["flags"], lo["flags"]), np.flatnonzero(lg["flags"] != lo["flags"])[:4]
        assert np.array_equal(lg["id_a"], lo["id_a"]) and np.array_equal(lg["id_b"], lo["id_b"])
        ok = (lo["flags"] & STRUCT_FLAGS) == 0
        assert np.all(np.abs(lg["dE"][ok] - lo["dE"][ok]) <= de_tol(lo[ok]))
        acc += int(np.sum((lg["flags"] & oracle.F_ACC) != 0))
        g.md_end(DT, GAMMA, 77)
        o.md_end(DT, GAMMA, 77)
        _same_bodies(g.rigid_body_state(), o.body_state(), L)
        _same_particles(g.state(), o.particles(), L)
    assert acc > 0
    moved = np.abs(_wrapdiff(g.rigid_body_state()[:, 0:3], x0, L)).max()
    assert moved > 0.0
    g.check()
    g.close()


def test_cycles_match_oracle(crmc):
    _cycles(crmc, _pair(), 5)


def test_cycles_match_oracle_full_size(crmc):
    """The two-nanoparticle system at its full size: 2 x 1000 sites, R = 5, L = 100."""
    w = W.config3(separation=12.0, seed=3)
    sites = np.flatnonzero((w.type == W.ACID) | (w.type == W.BASE))
    w.state[sites[w.type[sites] == W.ACID][::4]] = 1
    w.state[sites[w.type[sites] == W.BASE][::4]] = 1
    w.vel = (np.random.default_rng(3).normal(size=(w.n, 3))).astype(np.float32)
    _cycles(crmc, w, 2, trials_mult=1)


def test_cycles_match_oracle_across_the_periodic_boundary(crmc):
    """The first nanoparticle centred on the box corner, so that it straddles
    all three periodic boundaries."""
    w = _pair(seed=7)
    L = float(w.params["box_L"])
    x = np.mod(w.xyz.astype(np.float64) + [L / 2 + 4.5, L / 2, L / 2], L).astype(np.float32)
    x[x >= np.float32(L)] = 0.0
    w.xyz = x
    first, count = w.meta["bodies"]
    nb = x[first[0]:first[0] + count[0]]
    assert np.all(nb.min(0) < 2.0) and np.all(nb.max(0) > L - 2.0)  # split by every boundary
    _cycles(crmc, w, 4)


def test_cycles_match_oracle_with_ewald(crmc):
    """The same cycles under Ewald electrostatics (global schedule, |n| <= 6):
    the bodies feel the reciprocal-space forces too."""
    w = _pair(seed=6)
    w.params.update(schedule=1, ewald_kmax=6, trials_per_domain=100)
    _cycles(crmc, w, 4)


def test_md_step_equals_begin_end_and_bodies_stay_rigid(crmc):
    w = _pair(seed=4)
    first, count = w.meta["bodies"]
    a, b = crmc.Context(w), crmc.Context(w)
    for g in (a, b):
        g.set_rigid_bodies(first, count)
    s0 = a.state()
    for s in range(20):
        a.md_step(1, DT, GAMMA, 50 + s)
        b.md_begin(DT, GAMMA, 50 + s)
        b.md_end(DT, GAMMA, 50 + s)
    sa, sb = a.state(), b.state()
    for k in ("id", "xyz", "vel"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(a.rigid_body_state(), b.rigid_body_state())
    a.md_step(400, DT, GAMMA, 99)
    s1 = a.state()
    L = float(np.float32(w.params["box_L"]))
    for f, c in zip(first, count):
        i0 = np.searchsorted(s0["id"], np.arange(f, f + c))
        i1 = np.searchsorted(s1["id"], np.arange(f, f + c))
        d0 = _wrapdiff(s0["xyz"][i0][:, None], s0["xyz"][i0][None], L)
        d1 = _wrapdiff(s1["xyz"][i1][:, None], s1["xyz"][i1][None], L)
        assert np.abs(np.linalg.norm(d0, axis=-1) - np.linalg.norm(d1, axis=-1)).max() < 5e-5
    bs = a.rigid_body_state()
    R = bs[:, 6:15].reshape(-1, 3, 3)
    assert np.allclose(np.einsum("bij,bik->bjk", R, R), np.eye(3), atol=1e-12)
    a.check()


def test_refusals(crmc):
    w = _pair(seed=5)
    first, count = w.meta["bodies"]
    g = crmc.Context(w)
    before = g.state()
    n_ion = int(np.flatnonzero((w.type == W.XP) | (w.type == W.XM))[0])
    for f, c in (([0, 30], [41, 41]), ([0], [1]), ([n_ion - 1], [2]), ([w.n - 1], [5]), ([-1], [3])):
        with pytest.raises(crmc.CrError):
            g.set_rigid_bodies(f, c)
    st = g.state()
    for k in ("id", "xyz", "vel"):
        assert np.array_equal(st[k], before[k]), k  # nothing changed
    g.set_rigid_bodies(first, count)
    with pytest.raises(crmc.CrError):
        crmc.Batch([g])
    st = g.state()
    arrs = [np.ascontiguousarray(st[k]) for k in ("xyz", "vel", "type", "cls", "state")]
    with pytest.raises(crmc.CrError):
        g.load(st["n"], *arrs)
    g.set_rigid_bodies([], [])  # removed: a load and a batch are fine again
    assert g.rigid_body_state().shape == (0, 22)
    b = crmc.Batch([g])
    b.close()
    g.close()
