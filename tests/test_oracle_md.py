"""Pins for the oracle's MD part (forces and the Langevin velocity-Verlet step).

* Conservative forces are minus the gradient of the brute-force total energy
  (pairs + FENE bonds), checked by central finite differences.
* Newton's third law: the forces sum to zero.
* With gamma = 0 the velocity-Verlet step conserves total energy to O(dt^2).
* With the Langevin terms an ideal gas equilibrates to kT = 1 (<v^2> = 3).
"""
import math

import numpy as np

import oracle
from paper_2109_07527_gb300 import workloads as W


def _total_energy(o):
    return o.energy() + o.bond_energy()


def test_forces_are_minus_energy_gradient():
    w = W.config1(seed=5, n_pairs=12)
    o = oracle.Oracle(w)
    # ionise some sites so that Coulomb forces are present
    o.sweep(o.trials_per_sweep * 20, 3)
    ids, F, S = o.forces()
    p = o.particles()
    xyz = p["xyz"].copy()
    rng = np.random.default_rng(0)
    picks = rng.choice(len(ids), size=12, replace=False)
    h = 1e-3
    for i in picks:
        for c in range(3):
            xp = xyz.copy(); xm = xyz.copy()
            xp[i, c] = np.float32(xyz[i, c] + h)
            xm[i, c] = np.float32(xyz[i, c] - h)
            hh = float(xp[i, c]) - float(xm[i, c])
            o.set_positions(p["id"], xp); ep = _total_energy(o)
            o.set_positions(p["id"], xm); em = _total_energy(o)
            fd = -(ep - em) / hh
            assert abs(fd - F[i, c]) < 2e-4 * max(1.0, S[i, c]), (i, c, fd, F[i, c], S[i, c])
    o.set_positions(p["id"], xyz)


def test_forces_sum_to_zero():
    w = W.config1(seed=6)
    o = oracle.Oracle(w)
    o.sweep(o.trials_per_sweep * 10, 4)
    _, F, S = o.forces()
    assert np.all(np.abs(F.sum(0)) < 1e-9 * max(1.0, S.sum()))


def test_nve_energy_conservation():
    w = W.config1(seed=7, n_pairs=16)
    w.vel[:] = (np.random.default_rng(1).normal(size=w.vel.shape) * 0.5).astype(np.float32)
    o = oracle.Oracle(w)
    o.md_step(1, 0.002, 0.0, 1)  # initial force evaluation

    def etot():
        v = o.particles()["vel"]
        return _total_energy(o) + 0.5 * float((v * v).sum())

    e0 = etot()
    o.md_step(200, 0.002, 0.0, 1)
    e1 = etot()
    assert abs(e1 - e0) / w.n < 2e-3, (e0, e1)


def test_langevin_thermalises_ideal_gas():
    w = W.ideal(n_sites=0, n_pairs=150, seed=3, L=40.0)
    w.vel = np.zeros((w.n, 3), np.float32)
    o = oracle.Oracle(w)
    o.md_step(400, 0.005, 1.0, 42)
    ke = []
    for b in range(20):
        o.md_step(50, 0.005, 1.0, 42)
        v = o.particles()["vel"]
        ke.append(float((v * v).mean()))
    T = float(np.mean(ke))
    assert abs(T - 1.0) < 0.05, T


def test_split_step_equals_md_step():
    """md_begin + md_end with nothing in between is exactly one md_step."""
    w = W.config1(seed=9, n_pairs=16)
    a, b = oracle.Oracle(w), oracle.Oracle(w)
    for s in range(3):
        a.md_step(1, 0.005, 1.0, 77)
        b.md_begin(0.005, 1.0, 77)
        b.md_end(0.005, 1.0, 77)
    pa, pb = a.particles(), b.particles()
    assert np.array_equal(pa["xyz"], pb["xyz"]) and np.array_equal(pa["vel"], pb["vel"])


def test_cycles_with_trials_inside_the_step_keep_the_temperature():
    """CR-MC trials between the drift and the force evaluation (one force
    evaluation per cycle) leave the Langevin temperature at kT = 1."""
    w = W.config1(seed=10, n_pairs=24)
    o = oracle.Oracle(w, trials_per_domain=2)
    n = o.trials_per_sweep
    for s in range(150):
        o.md_begin(0.005, 1.0, 5)
        o.sweep(n, 100 + s)
        o.md_end(0.005, 1.0, 5)
    ke = []
    for s in range(300):
        o.md_begin(0.005, 1.0, 5)
        o.sweep(n, 1000 + s)
        o.md_end(0.005, 1.0, 5)
        if s % 10 == 0:
            v = o.particles()["vel"]
            ke.append(float((v * v).mean()))
    T = float(np.mean(ke))
    assert abs(T - 1.0) < 0.08, T
