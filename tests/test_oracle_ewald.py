"""Pins of the oracle's Ewald electrostatics (the paper's energy model is PPPM,
Sec. III.A, a mesh evaluation of the Ewald sum).  The oracle's Ewald energy is
checked against values that do not come from its own formula:

* the Madelung constants of the rock-salt (NaCl) and caesium-chloride
  structures, 1.747564594633 and 1.762674773070 for the nearest-neighbour
  distance d (textbook values): E / N = -M l_B / (2 d);
* the independence of the total energy from the splitting parameter alpha
  (the real-space, reciprocal and self parts each change with alpha; only a
  correct balance of the three keeps the sum fixed);
* Delta E = E_after - E_before for every accepted trial of a CR-MC run under
  the global schedule (the trials' reciprocal part is an update of S(k), the
  energy a recomputation from scratch);
* planted mistakes (half the reciprocal part, no self term) fail these pins;
* the MD forces (real-space erfc pair forces plus the reciprocal-space forces)
  are minus the gradient of the Ewald energy (central finite differences),
  sum to zero, and keep kinetic plus potential energy in a run without the
  thermostat; a reciprocal force of the wrong sign fails the gradient pin.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W

M_NACL = 1.747564594633182
M_CSCL = 1.762674773070988


def _ions_workload(xyz, q, L, rc, alpha, kmax, lB=1.0):
    n = len(q)
    t = np.where(np.asarray(q) > 0, W.XP, W.XM).astype(np.int32)
    params = W.default_params(box_L=L, rc=rc, lB=lB, alpha=alpha, schedule=1, trials_per_domain=1,
                              wca_on=[0] * 16, ewald_kmax=kmax)
    return W.Workload(name="lattice", xyz=np.asarray(xyz, np.float32), type=t, cls=np.zeros(n, np.int32),
                      state=np.zeros(n, np.int8), pK=np.zeros(n), bonds=np.zeros((0, 2), np.int32), vel=None,
                      params=params, capacity=n + 16)


def _rock_salt(n=8, d=1.0, shift=0.25):
    g = np.arange(n)
    ix, iy, iz = np.meshgrid(g, g, g, indexing="ij")
    xyz = (np.stack([ix, iy, iz], -1).reshape(-1, 3) + shift) * d
    q = np.where((ix + iy + iz).reshape(-1) % 2 == 0, 1, -1)
    return xyz, q, n * d


def _caesium_chloride(n=6, a=1.0, shift=0.1):
    g = np.arange(n)
    ix, iy, iz = np.meshgrid(g, g, g, indexing="ij")
    corners = (np.stack([ix, iy, iz], -1).reshape(-1, 3) + shift) * a
    centres = corners + 0.5 * a
    xyz = np.concatenate([corners, centres])
    q = np.concatenate([np.ones(len(corners), int), -np.ones(len(centres), int)])
    return xyz, q, n * a


def test_rock_salt_madelung_constant():
    xyz, q, L = _rock_salt()
    o = oracle.Oracle(_ions_workload(xyz, q, L, rc=4.0, alpha=1.0, kmax=12))
    e = o.energy() / len(q)
    assert abs(e + M_NACL / 2.0) < 1e-7 * M_NACL


def test_caesium_chloride_madelung_constant():
    xyz, q, L = _caesium_chloride()
    d = math.sqrt(3.0) / 2.0
    o = oracle.Oracle(_ions_workload(xyz, q, L, rc=3.0, alpha=1.3, kmax=13))
    e = o.energy() / len(q)
    assert abs(e + M_CSCL / (2.0 * d)) < 1e-7 * M_CSCL


def _random_electrolyte(n_pairs=40, L=10.0, seed=5):
    rng = np.random.default_rng(seed)
    xyz = rng.random((2 * n_pairs, 3)) * L
    q = np.tile([1, -1], n_pairs)
    return xyz, q, L


def test_total_energy_does_not_depend_on_alpha():
    xyz, q, L = _random_electrolyte()
    parts = []
    for alpha, kmax in ((0.9, 13), (1.1, 16)):
        o = oracle.Oracle(_ions_workload(xyz, q, L, rc=5.0, alpha=alpha, kmax=kmax))
        parts.append(o.ewald_parts())
        assert abs(sum(parts[-1]) - o.energy()) < 1e-12 * sum(abs(v) for v in parts[-1])
    (r1, k1, s1), (r2, k2, s2) = parts
    scale = max(abs(r1) + abs(k1) + abs(s1), abs(r2) + abs(k2) + abs(s2))
    assert abs(s1 - s2) > 0.1 * abs(s1)  # the parts do change with alpha
    assert abs((r1 + k1 + s1) - (r2 + k2 + s2)) < 1e-7 * scale


def _cr_system(seed=3):
    w = W.weak_acid_electrolyte(n_acid=30, L=20.0, pH=7.0, pKa=6.5, pIS=2.0, rc=8.0, seed=seed,
                                trials_per_domain=1, alpha=0.4)
    w.params["ewald_kmax"] = 6
    return w


def test_trial_dE_is_the_energy_difference():
    o = oracle.Oracle(_cr_system())
    assert o.ewald_nk == sum(1 for x in range(-6, 7) for y in range(-6, 7) for z in range(-6, 7)
                             if 0 < x * x + y * y + z * z <= 36)
    acc = 0
    for t in range(400):
        e0 = o.energy()
        rec = o.sweep(1, 900 + t, log=True)["log"][0]
        e1 = o.energy()
        if rec["flags"] & oracle.F_ACC:
            acc += 1
            assert abs((e1 - e0) - rec["dE"]) < 1e-9 * max(1.0, rec["S"]), t
        else:
            assert e1 == e0
    assert acc > 20


def test_sweep_dE_sum_is_the_energy_difference():
    """Within a sweep S(k) is carried from trial to trial by the accepted
    changes: the accepted dE of a 25-trial sweep add up to its energy change."""
    w = _cr_system(seed=4)
    w.params["trials_per_domain"] = 25
    o = oracle.Oracle(w)
    n_acc = 0
    for s in range(20):
        e0 = o.energy()
        log = o.sweep(25, 300 + s, log=True)["log"]
        e1 = o.energy()
        acc = (log["flags"] & oracle.F_ACC) != 0
        n_acc += int(acc.sum())
        assert abs((e1 - e0) - log["dE"][acc].sum()) < 1e-9 * max(1.0, log["S"].sum()), s
    assert n_acc > 20


@pytest.mark.parametrize("kind", ["ewald_half_recip", "drop_self"])
def test_planted_mistakes_fail_the_madelung_pin(kind):
    oracle.plant(kind)
    xyz, q, L = _rock_salt()
    o = oracle.Oracle(_ions_workload(xyz, q, L, rc=4.0, alpha=1.0, kmax=12))
    assert abs(o.energy() / len(q) + M_NACL / 2.0) > 100 * 1e-7 * M_NACL  # far outside the pin's tolerance


def test_planted_half_reciprocal_breaks_alpha_independence():
    oracle.plant("ewald_half_recip")
    xyz, q, L = _random_electrolyte()
    e = [oracle.Oracle(_ions_workload(xyz, q, L, rc=5.0, alpha=a, kmax=k)).energy() for a, k in ((0.9, 13), (1.1, 16))]
    assert abs(e[0] - e[1]) > 1e-3 * abs(e[0])


def test_ewald_needs_the_global_schedule():
    w = _cr_system()
    with pytest.raises(ValueError):
        oracle.Oracle(w, schedule=0)


def _ionised(seed=3):
    w = _cr_system(seed)
    o = oracle.Oracle(w)
    o.sweep(o.trials_per_sweep * 30, 11)  # ionise acids, insert ions
    return o


def _fd_errors(o, n_pick=10, h=1e-3):
    ids, F, S = o.forces()
    p = o.particles()
    xyz = p["xyz"].copy()
    charged = np.flatnonzero(np.isin(p["type"], (W.XP, W.XM)) | (p["state"] == 1))
    picks = np.random.default_rng(0).choice(charged, size=n_pick, replace=False)
    worst = 0.0
    for i in picks:
        for c in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[i, c] = np.float32(xyz[i, c] + h)
            xm[i, c] = np.float32(xyz[i, c] - h)
            hh = float(xp[i, c]) - float(xm[i, c])
            o.set_positions(p["id"], xp)
            ep = o.energy()
            o.set_positions(p["id"], xm)
            em = o.energy()
            worst = max(worst, abs(-(ep - em) / hh - F[i, c]) / max(1.0, S[i, c]))
    o.set_positions(p["id"], xyz)
    return worst, F, S


def test_ewald_forces_are_minus_energy_gradient():
    o = _ionised()
    worst, F, S = _fd_errors(o)
    assert worst < 2e-4, worst
    assert np.abs(F).max() > 0.1  # not vacuous
    assert np.all(np.abs(F.sum(0)) < 1e-9 * max(1.0, S.sum()))  # Newton's third law, reciprocal part included


def test_planted_reciprocal_force_sign_fails_the_gradient_pin():
    oracle.plant("ewald_force_sign")
    try:
        o = _ionised()
        worst, _, _ = _fd_errors(o)
    finally:
        oracle.plant("none")
    assert worst > 1e-2, worst


def test_ewald_md_conserves_energy():
    o = _ionised(seed=5)
    o.md_step(1, 0.002, 0.0, 1)

    def etot():
        v = o.particles()["vel"]
        return o.energy() + 0.5 * float((v * v).sum())

    e0 = etot()
    o.md_step(200, 0.002, 0.0, 1)
    e1 = etot()
    assert abs(e1 - e0) < 1e-4, (e0, e1)  # velocity Verlet at dt = 0.002 (1.5e-6 measured)
