"""Pins of the oracle's rigid bodies (Sec. IV.B: the nanoparticles carry their
sites rigidly and are thermostatted as a whole), against facts that do not
come from the oracle's own formulas:

* the body frame is the principal frame of the inertia tensor that the test
  forms itself from the positions (numpy's symmetric eigen-solver);
* a free symmetric top: its figure axis precesses about the fixed angular
  momentum L at the rate |L| / I_perp (closed form), L and the rotational
  energy stay fixed, the centre of mass moves on a straight line;
* rigidity: member distances do not change;
* with friction and noise every translational and rotational degree of
  freedom of a body holds kT = 1 (equipartition);
* an interacting system (two charged nanoparticles and their ions, gamma = 0)
  keeps its total energy, kinetic (free particles and bodies) plus potential,
  and its total momentum;
* planted mistakes (torque sign, no rotational noise) fail these pins.
"""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W


def _beads(xyz, vel=None, L=40.0):
    n = len(xyz)
    params = W.default_params(box_L=L, rc=10.0, lB=0.0, schedule=1, wca_on=[0] * 16)
    return W.Workload(name="beads", xyz=np.asarray(xyz, np.float32), type=np.zeros(n, np.int32),
                      cls=np.full(n, W.CLS_NONE, np.int32), state=np.zeros(n, np.int8), pK=np.zeros(n),
                      bonds=np.zeros((0, 2), np.int32),
                      vel=None if vel is None else np.asarray(vel, np.float32), params=params, capacity=n + 16)


def _top(a=1.0, b=2.0, omega=(0.3, 0.1, 0.5), V=(0.1, 0.0, 0.0), c=(20.0, 20.0, 20.0)):
    d = np.array([[a, 0, 0], [-a, 0, 0], [0, a, 0], [0, -a, 0], [0, 0, b], [0, 0, -b]], float)
    xyz = (np.array(c) + d).astype(np.float32)
    d = xyz.astype(np.float64) - xyz.astype(np.float64).mean(0)
    return _beads(xyz, np.array(V) + np.cross(np.array(omega), d))


def _rot(k, th, v):
    return v * np.cos(th) + np.cross(k, v) * np.sin(th) + k * np.dot(k, v) * (1 - np.cos(th))


def test_body_frame_is_the_principal_frame():
    rng = np.random.default_rng(4)
    d = rng.normal(size=(9, 3)) * [1.0, 1.6, 0.7]
    xyz = (np.array([39.0, 1.0, 20.0]) + d) % 40.0  # across the periodic boundary
    w = _beads(xyz, rng.normal(size=(9, 3)))
    o = oracle.Oracle(w)
    o.set_bodies([0], [9])
    s = o.body_state()[0]
    R = s[6:15].reshape(3, 3)
    x = w.xyz.astype(np.float64)
    dd = x - x[0]
    dd -= 40.0 * np.round(dd / 40.0)
    com = dd.mean(0)
    r = dd - com
    I = (r * r).sum() * np.eye(3) - r.T @ r
    ev = np.linalg.eigh(I)[0]
    assert np.allclose(s[18:21], ev, rtol=1e-12, atol=1e-12)
    assert np.allclose(R.T @ I @ R, np.diag(ev), atol=1e-10)
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-13) and abs(np.linalg.det(R) - 1.0) < 1e-13
    assert np.allclose((s[0:3] - (x[0] + com) + 20.0) % 40.0 - 20.0, 0.0, atol=1e-12)
    v = w.vel.astype(np.float64)
    assert np.allclose(s[3:6], v.mean(0), atol=1e-12)
    L = np.cross(r, v).sum(0)
    assert np.allclose(R @ s[15:18], L, atol=1e-12)
    assert s[21] == 9.0


def test_free_symmetric_top_precesses_at_the_closed_form_rate():
    o = oracle.Oracle(_top())
    o.set_bodies([0], [6])
    s0 = o.body_state()[0]
    assert np.allclose(s0[18:21], [4.0, 10.0, 10.0])  # I_sym = 4 a^2, I_perp = 2 a^2 + 2 b^2
    R0 = s0[6:15].reshape(3, 3)
    L = R0 @ s0[15:18]
    dt, steps = 0.002, 2000
    o.md_step(steps, dt, 0.0, 1)
    s = o.body_state()[0]
    R = s[6:15].reshape(3, 3)
    t = steps * dt
    ang = np.linalg.norm(L) * t / 10.0
    assert ang > 1.0  # the axis has turned far
    assert np.abs(R[:, 0] - _rot(L / np.linalg.norm(L), ang, R0[:, 0])).max() < 1e-6
    assert np.abs(R @ s[15:18] - L).max() < 1e-12
    assert np.abs(s[0:3] - (s0[0:3] + s0[3:6] * t)).max() < 1e-10
    e0 = 0.5 * np.sum(s0[15:18] ** 2 / s0[18:21])
    e1 = 0.5 * np.sum(s[15:18] ** 2 / s[18:21])
    assert abs(e1 - e0) < 1e-6 * e0
    # rigidity: the members keep their distances, at FP32 rounding of positions
    x = o.particles()["xyz"].astype(np.float64)
    x0 = _top().xyz.astype(np.float64)
    D = lambda y: np.linalg.norm(y[:, None] - y[None], axis=-1)
    assert np.abs(D(x) - D(x0)).max() < 2e-5


def test_planted_torque_sign_is_caught_by_energy_conservation():
    """An interacting system with gamma = 0 keeps kinetic + potential energy;
    with the torque's sign planted wrong it does not."""
    drift = {}
    for plant in ("none", "rigid_torque_sign"):
        oracle.plant(plant)
        w = _charged_pair()
        o = oracle.Oracle(w)
        o.set_bodies(*w.meta["bodies"])
        o.md_step(1, 0.002, 0.0, 1)
        e0, p0 = _energy(o), _momentum(o)
        o.md_step(300, 0.002, 0.0, 1)
        e1, p1 = _energy(o), _momentum(o)
        drift[plant] = abs(e1 - e0)
        if plant == "none":
            assert np.abs(p1 - p0).max() < 1e-9 * len(w.xyz)
    oracle.plant("none")
    # velocity Verlet at dt = 0.002: an O(dt^2) error far below 1e-4 kT here
    assert drift["none"] < 1e-4, drift
    assert drift["rigid_torque_sign"] > 1e-3, drift


def _charged_pair(seed=2):
    w = W.config3(separation=9.0, n_sites=40, L=40.0, R=3.0, seed=seed)
    sites = np.flatnonzero((w.type == W.ACID) | (w.type == W.BASE))
    acids = sites[w.type[sites] == W.ACID][::2]
    bases = sites[w.type[sites] == W.BASE][::2]
    w.state[acids] = 1
    w.state[bases] = 1
    rng = np.random.default_rng(seed)
    w.vel = (rng.normal(size=(w.n, 3)) * 0.7).astype(np.float32)
    return w


def _energy(o):
    p = o.particles()
    s = o.body_state()
    ids = p["id"]
    members = np.zeros(len(ids), bool)
    first, count = o.bodies
    for f, c in zip(first, count):
        members |= (ids >= f) & (ids < f + c)
    v = p["vel"][~members]
    ke = 0.5 * float((v * v).sum())
    ke += float(np.sum(0.5 * s[:, 21] * np.sum(s[:, 3:6] ** 2, 1)))
    ke += float(np.sum(0.5 * s[:, 15:18] ** 2 / s[:, 18:21]))
    return ke + o.energy()


def _momentum(o):
    p = o.particles()
    s = o.body_state()
    first, count = o.bodies
    members = np.zeros(len(p["id"]), bool)
    for f, c in zip(first, count):
        members |= (p["id"] >= f) & (p["id"] < f + c)
    return p["vel"][~members].sum(0) + (s[:, 21:22] * s[:, 3:6]).sum(0)


def _gas():
    base = np.array([[1.0, 0, 0], [-1.0, 0, 0], [0, 1.5, 0], [0, -1.5, 0], [0, 0, 0.7], [0, 0, -0.7],
                     [0.4, 0.4, 0.4]])
    xyz = np.concatenate([np.array([5.0 + 10 * (b % 4), 10.0 + 20 * (b // 4), 20.0]) + base for b in range(8)])
    return _beads(xyz)


@pytest.mark.parametrize("plant", ["none", "rigid_no_rot_noise"])
def test_thermostat_gives_equipartition(plant):
    oracle.plant(plant)
    try:
        o = oracle.Oracle(_gas())
        o.set_bodies(np.arange(8) * 7, [7] * 8)
        o.md_step(2000, 0.005, 1.0, 5)
        kt, kr = [], []
        for blk in range(500):
            o.md_step(100, 0.005, 1.0, 6 + blk)
            s = o.body_state()
            kt.append((s[:, 21:22] * s[:, 3:6] ** 2).mean())
            kr.append((s[:, 15:18] ** 2 / s[:, 18:21]).mean(0))
    finally:
        oracle.plant("none")
    kt, kr = np.mean(kt), np.mean(kr, 0)
    if plant == "none":
        assert abs(kt - 1.0) < 0.05, kt
        assert np.all(np.abs(kr - 1.0) < 0.08), kr
    else:
        assert np.all(kr < 0.1), kr  # friction alone drains the rotation


def test_bodies_refused():
    w = _charged_pair()
    o = oracle.Oracle(w)
    first, count = w.meta["bodies"]
    n_ion = int(np.flatnonzero((w.type == W.XP) | (w.type == W.XM))[0])
    for f, c in (([0, 30], [41, 41]),  # overlapping
                 ([0], [1]),  # one member
                 ([n_ion - 1], [2]),  # an ion member
                 ([w.n - 1], [5]),  # beyond the permanent ids
                 ([-1], [3])):
        with pytest.raises(ValueError):
            o.set_bodies(f, c)
    line = _beads(np.array([[10.0, 10, 10], [11.0, 10, 10], [12.0, 10, 10]]))
    with pytest.raises(ValueError):  # collinear: no moment about the line
        oracle.Oracle(line).set_bodies([0], [3])
    o.set_bodies(first, count)
    assert len(o.body_state()) == 2
