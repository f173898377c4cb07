"""GPU CR-MC path (through the C ABI) against the FP64 oracle, trial by trial.

Decisions and charge states must be identical for the same seed, dE within
1e-6 of the oracle relative to max(|dE|, sum |pair changes|) (see
parity_util).  Cases cover several tiles and ragged domains, every move type,
acid and base sites, ghost and interacting ions, the global and the coloured
schedule, expanded WCA, and the full-size polyelectrolyte workload.
"""
import math

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


def _parity(crmc, w, sweeps, seed, **kw):
    g = crmc.Context(w, **kw)
    n = g.trials_per_sweep * sweeps
    lg = g.sweep(n, seed, log=True)["log"]
    okw = {k: v for k, v in kw.items() if k in ("schedule", "trials_per_domain", "domain_cells")}
    o, lo, ties = compare_logs(w, lg, n, seed, okw)
    compare_states(g, o, w.n_sites)
    return g, o, lg, lo, ties


def test_philox_device_matches_oracle(crmc):
    out = crmc.philox(0, 7, 11, 3, 0xDEADBEEF, 0x12345678, 4096)
    for i in range(4096):  # every block of the range, bit for bit
        assert out[i].tolist() == oracle.philox([i, 7, 11, 3], [0xDEADBEEF, 0x12345678]).tolist()
    hi = crmc.philox(0xFFFFF000, 0xFFFFFFFF, 0x80000000, 6, 0xFFFFFFFF, 0, 4096)  # counter words near overflow
    for i in range(0, 4096, 7):
        assert hi[i].tolist() == oracle.philox([0xFFFFF000 + i, 0xFFFFFFFF, 0x80000000, 6], [0xFFFFFFFF, 0]).tolist()
    kat = crmc.philox(0, 0, 0, 0, 0, 0, 1)[0]
    assert kat.tolist() == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


@pytest.mark.parametrize("schedule,m", [(0, 4), (1, 256)])
def test_parity_ideal_ghost_ions(crmc, schedule, m):
    w = W.ideal(n_sites=50, pH=5.0, pKa=5.0, n_pairs=20, seed=11, schedule=schedule, trials_per_domain=m)
    _, _, lg, _, ties = _parity(crmc, w, 20, 5)
    assert (lg["flags"] & 1).sum() > 100


@pytest.mark.parametrize("n_base", [0, 3])
def test_parity_interacting_sites(crmc, n_base):
    w = W.enum_sites(n_sites=8, n_base=n_base, seed=3, schedule=1, trials_per_domain=256)
    if n_base:
        w.params["pH"] = 7.0
        w.pK[:] = 7.0
    _parity(crmc, w, 20, 9)


@pytest.mark.parametrize("schedule,m,sweeps", [(0, 10, 16), (1, 500, 20)])
def test_parity_config1_polyacid(crmc, schedule, m, sweeps):
    w = W.config1(seed=1, schedule=schedule, trials_per_domain=m)
    g, o, lg, lo, ties = _parity(crmc, w, sweeps, 1)
    acc = lg["flags"] & 1
    assert acc.sum() > 50
    moves = set(np.unique(lg["move"][acc == 1]).tolist())
    assert {0, 1, 4, 5} <= moves  # acid and salt, both directions


def test_parity_config2_half_box(crmc):
    """16 chains x 200 at 1/8 of the volume: several domains per colour, ragged cell occupancy."""
    w = W.config2(seed=2, scale=0.5)
    _parity(crmc, w, 6, 3)


def test_parity_config3_nanoparticles(crmc):
    """Acid and base sites on two nanoparticle shells, expanded WCA cores (Delta = R - r)."""
    w = W.config3(separation=12.0, seed=1, L=60.0, n_sites=300)
    _parity(crmc, w, 8, 4)


def test_parity_config3_full_size_nanoparticles(crmc):
    """The nanoparticle pair at full size: two R = 5 cores with 1000 surface
    sites each (acids on one, bases on the other), L = 100, 20 mM salt, at the
    closest separation of the sweep (10.5: the cores' surfaces 0.5 sigma
    apart), trial by trial."""
    w = W.config3(separation=10.5, seed=2)
    assert w.n_sites == 2000 and float(w.params["box_L"]) == 100.0
    g, o, lg, lo, ties = _parity(crmc, w, 3, 6)
    acc = lg["flags"] & 1
    moves = set(np.unique(lg["move"][acc == 1]).tolist())
    assert {0, 2} <= moves  # acid and base sites both ionise (from all-neutral shells)


def test_parity_full_size_polyelectrolyte(crmc):
    """The benchmark workload itself (L = 120, 3200 sites, ~4000 ion pairs), two sweeps."""
    w = W.config2(seed=1)
    g, o, lg, lo, ties = _parity(crmc, w, 2, 1)
    assert len(lg) == 20000
    assert ties <= 2


def test_repeated_calls_continue_the_chain(crmc):
    """Two calls of n trials give the same chain as the oracle's two calls."""
    w = W.config1(seed=4)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    n = g.trials_per_sweep * 3
    for seed in (7, 7, 8):
        lg = g.sweep(n, seed, log=True)["log"]
        lo = o.sweep(n, seed, log=True)["log"]
        assert np.array_equal(lg["flags"], lo["flags"])
    compare_states(g, o, w.n_sites)


def test_no_sites_only_salt_moves(crmc):
    w = W.ideal(n_sites=0, n_pairs=30, seed=2)
    w.params["ion_coupling"] = 1
    w.params["lB"] = 2.0
    _parity(crmc, w, 10, 2)


def test_empty_box(crmc):
    w = W.ideal(n_sites=0, n_pairs=0, seed=2)
    _parity(crmc, w, 5, 1)


def test_stats_count_every_trial(crmc):
    w = W.config1(seed=5)
    g = crmc.Context(w)
    n = g.trials_per_sweep * 4
    st = g.sweep(n, 3, stats=True)["stats"]
    assert st["trials"] == n and st["attempts"].sum() == n
    assert 0 < st["accepts"].sum() < n


def test_errors(crmc):
    w = W.config1(seed=1)
    g = crmc.Context(w)
    with pytest.raises(crmc.CrError) as e:
        g.sweep(g.trials_per_sweep + 1, 1)
    assert e.value.code == -1
    bad = W.config1(seed=1)
    bad.state[0] = 1  # one ionised acid without a counterion
    with pytest.raises(crmc.CrError) as e:
        crmc.Context(bad)
    assert e.value.code == -2
    small = W.config1(seed=1)
    small.params["rc"] = 25.0  # rc > L/2
    with pytest.raises(crmc.CrError) as e:
        crmc.Context(small)
    assert e.value.code == -1


def test_cell_overflow_is_reported(crmc):
    w = W.ideal(n_sites=40, n_pairs=200, seed=1, pIS=0.0)
    g = crmc.Context(w, cell_capacity=8)
    with pytest.raises(crmc.CrError) as e:
        for s in range(50):
            g.sweep(g.trials_per_sweep * 4, s, stats=True)
    assert e.value.code == -3


def test_gpu_titration_matches_exact_closed_form(crmc):
    """GPU alpha of ideal acids at three pH values within 0.005 of the exact
    finite-box result (Eq. QQ with E = 0)."""
    from scipy.special import gammaln, ive
    n, L = 50, 40.0
    for pH in (4.0, 5.0, 6.0):
        w = W.ideal(n_sites=n, L=L, pH=pH, pKa=5.0, n_pairs=20, seed=11, trials_per_domain=8)
        g = crmc.Context(w)
        ln10 = math.log(10.0)
        pIX = -math.log10(10 ** -2.0 + 10 ** -min(pH, 14 - pH))
        lnz = math.log(0.602214076 * (L * 0.355) ** 3) - ln10 * pIX
        k = np.arange(n + 1)
        logP = gammaln(n + 1) - gammaln(k + 1) - gammaln(n - k + 1) + k * ln10 * (pH - 5.0) + np.log(ive(k, 2 * math.exp(lnz)))
        P = np.exp(logP - logP.max())
        P /= P.sum()
        exact = float((k * P).sum() / n)
        tps = g.trials_per_sweep
        g.sweep(tps * 50, 1)
        vals = []
        for b in range(400):
            g.sweep(tps * 4, 2 + b)
            vals.append(g.counts()["n_Am"] / n)
        assert abs(np.mean(vals) - exact) < 0.005, (pH, np.mean(vals), exact)


# ------------------------------------------------------------------ MD part
F_REL = 4e-6  # FP32 force terms against FP64: relative to the gross magnitude of the summed terms


def _wrapdiff(a, b, L):
    d = a.astype(np.float64) - b.astype(np.float64)
    return d - L * np.round(d / L)


def test_md_forces_match_oracle(crmc):
    w = W.config1(seed=5)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    n = g.trials_per_sweep * 4
    g.sweep(n, 3)
    o.sweep(n, 3)
    g.md_forces()
    st = g.state()
    ids, F, S = o.forces()
    assert np.array_equal(st["id"], ids)
    err = np.abs(st["force"].astype(np.float64) - F)
    tol = F_REL * S + 2e-6
    assert np.all(err <= tol), (np.argmax(err / tol), err.max())
    assert np.abs(F).max() > 1.0  # the check is not vacuous


def test_asymmetric_wca_table_refused(crmc):
    """A pair potential's class table is symmetric; the force kernel evaluates
    each pair once and relies on it, so an asymmetric table is refused."""
    w = W.config1(seed=5)
    w.params["wca_del"] = list(w.params["wca_del"])
    w.params["wca_del"][0 * 4 + 1] = 0.5  # (0, 1) but not (1, 0)
    with pytest.raises(crmc.CrError) as e:
        crmc.Context(w)
    assert e.value.code == -1


def test_md_forces_full_size_sampled(crmc):
    """Forces of the full polyelectrolyte box: every particle vs the oracle's brute-force sum."""
    w = W.config2(seed=1)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    g.md_forces()
    st = g.state()
    ids, F, S = o.forces()
    assert np.array_equal(st["id"], ids)
    err = np.abs(st["force"].astype(np.float64) - F)
    assert np.all(err <= F_REL * S + 2e-6)


def test_md_step_and_interleaved_cycles(crmc):
    """CR-MC sweeps (bit-exact) alternating with MD steps (FP32 vs FP64 within
    tolerance); the oracle is re-synchronised to the GPU positions after each MD step."""
    w = W.config1(seed=6, n_pairs=32)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    L = float(np.float32(w.params["box_L"]))
    n = g.trials_per_sweep * 2
    for cyc in range(4):
        lg = g.sweep(n, 10 + cyc, log=True)["log"]
        lo = o.sweep(n, 10 + cyc, log=True)["log"]
        assert np.array_equal(lg["flags"], lo["flags"]) and np.array_equal(lg["id_a"], lo["id_a"])
        g.md_step(1, 0.005, 1.0, 77)
        o.md_step(1, 0.005, 1.0, 77)
        sg, so = g.state(), o.particles()
        assert np.array_equal(sg["id"], so["id"])
        assert np.abs(_wrapdiff(sg["xyz"], so["xyz"], L)).max() < 2e-5
        assert np.abs(sg["vel"] - so["vel"]).max() < 2e-4
        o.set_positions(sg["id"], sg["xyz"], sg["vel"])
    g.md_step(20, 0.005, 1.0, 78)
    g.check()


@pytest.mark.parametrize("threads,regs", [(32, 0), (64, 0), (128, 0), (128, 4), (256, 0), (256, 2), (512, 0), (512, 1)])
def test_launch_shape_does_not_change_the_chain(crmc, threads, regs):
    """Every (threads, halo registers) shape the autotuner may pick gives the
    oracle's chain: halo in registers or shared memory, single-warp domains."""
    w = W.config2(seed=2, scale=0.5)
    g = crmc.Context(w)
    g.set_launch_shape(threads, regs)
    assert g.launch_shape() == (threads, regs)
    n = g.trials_per_sweep * 3
    lg = g.sweep(n, 3, log=True)["log"]
    o, lo, ties = compare_logs(w, lg, n, 3)
    compare_states(g, o, w.n_sites)


def test_autotuner_keeps_the_chain(crmc):
    """Unlogged sweeps used for tuning (one shape per sweep, with full and
    compact shared-memory capacities) continue the same chain."""
    w = W.config2(seed=3, scale=0.5)
    g = crmc.Context(w)
    o = oracle.Oracle(w)
    n = g.trials_per_sweep * 14
    g.sweep(n, 5)
    o.sweep(n, 5)
    compare_states(g, o, w.n_sites)
    assert g.launch_shape()[0] in (32, 64, 128, 256, 512)


# ------------------------------------------------------------------ batches of replicas
def _replica_seed(seed, r):
    return seed ^ (r << 32)


def test_batch_matches_independent_oracle_runs(crmc):
    """A batch of replicas (different pH, different box sizes) advanced by
    one launch per colour equals, replica by replica, the oracle run with the
    replica's key."""
    ws = [W.config2(seed=5, scale=0.5, pH=pH) for pH in (3.0, 4.5, 6.0)]
    ws += W.config4(seed=2, n_rep=2, hi=300)
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(4, 77)
    for r, (w, g) in enumerate(zip(ws, ctxs)):
        o = oracle.Oracle(w)
        o.sweep(o.trials_per_sweep * 4, _replica_seed(77, r))
        compare_states(g, o, w.n_sites)


def test_batch_of_64_uneven_replicas_matches_oracle(crmc):
    """The batched titration at full size: 64 replicas with chain lengths
    log-uniform in [50, 1000], pH uniform in [2, 10] and boxes from 36.8 to
    100 sigma (1 to 64 domains per colour) advanced together, one launch per
    colour; every replica's final state equals the oracle run with its key."""
    ws = W.config4(seed=1)
    assert len(ws) == 64
    ctxs = [crmc.Context(w) for w in ws]
    nact = sorted({g.info["nd"] ** 3 // 8 for g in ctxs})
    assert nact[0] == 1 and nact[-1] == 64
    b = crmc.Batch(ctxs)
    b.sweep(3, 91)
    for r, (w, g) in enumerate(zip(ws, ctxs)):
        o = oracle.Oracle(w)
        o.sweep(o.trials_per_sweep * 3, _replica_seed(91, r))
        compare_states(g, o, w.n_sites)
    b.close()


@pytest.mark.parametrize("threads,regs,cap", [(64, 0, 0), (128, 4, 0), (256, 0, 0), (64, 0, 8)])
def test_persistent_sweep_equals_colour_launches(crmc, threads, regs, cap):
    """The persistent batch sweep (a domain starts when its neighbours of
    lower colours are done, so colours overlap within and across replicas)
    and one launch per colour give the same states bit for bit, and both the
    oracle's; cap = 8 puts dense domains' lists in the global scratch, one
    region per (colour, domain), while domains of several colours run."""
    ws = [W.config2(seed=12, scale=0.5, pH=p) for p in (3.0, 4.5, 6.0)] + W.config4(seed=3, n_rep=3, hi=400)
    kw = dict(list_capacity=cap, halo_capacity=64) if cap else {}
    runs = []
    for persistent in (True, False):
        ctxs = [crmc.Context(w, **kw) for w in ws]
        b = crmc.Batch(ctxs)
        b.set_persistent(persistent)
        b.set_launch_shape(threads, regs)
        b.sweep(3, 55)
        runs.append([g.state() for g in ctxs])
        if persistent:
            for r, (w, g) in enumerate(zip(ws, ctxs)):
                o = oracle.Oracle(w)
                o.sweep(o.trials_per_sweep * 3, _replica_seed(55, r))
                compare_states(g, o, w.n_sites)
        b.close()
    for a, c in zip(*runs):
        for k in ("id", "xyz", "vel", "state"):
            assert np.array_equal(a[k], c[k]), k


def test_batch_md_equals_per_context_md(crmc):
    ws = [W.config2(seed=7, scale=0.5, pH=pH) for pH in (3.0, 5.0)]
    a = [crmc.Context(w) for w in ws]
    c = [crmc.Context(w) for w in ws]
    b = crmc.Batch(a)
    b.sweep(2, 9)
    b.md_step(3, 0.005, 1.0, 11)
    for r, g in enumerate(c):
        g.sweep(g.trials_per_sweep * 2, _replica_seed(9, r))
        g.md_step(3, 0.005, 1.0, _replica_seed(11, r))
    for x, y in zip(a, c):
        sx, sy = x.state(), y.state()
        assert np.array_equal(sx["id"], sy["id"])
        assert np.array_equal(sx["xyz"], sy["xyz"]) and np.array_equal(sx["vel"], sy["vel"])


@pytest.mark.parametrize("list_capacity,halo_capacity", [(8, 64), (4, 32)])
def test_parity_with_lists_and_halos_beyond_shared_memory(crmc, list_capacity, halo_capacity):
    """Small on-chip capacities force the global-memory paths: domain lists in
    the global scratch region and halo particles read from global memory."""
    w = W.config2(seed=3, scale=0.5)
    _parity(crmc, w, 2, 31, list_capacity=list_capacity, halo_capacity=halo_capacity)


@pytest.mark.parametrize("threads,regs", [(64, 0), (128, 4), (512, 1)])
def test_flat_frame_full_box_launch_shapes(crmc, threads, regs):
    """In the full-size box (L = 120, regions of 36 sigma) the halo is compared
    in the region's flat frame, held in shared memory or in registers; regions
    that wrap around the periodic boundary along one to three axes occur every
    sweep.  The chain equals the oracle's trial by trial."""
    w = W.config2(seed=11)
    g = crmc.Context(w)
    g.set_launch_shape(threads, regs)
    n = g.trials_per_sweep
    lg = g.sweep(n, 13, log=True)["log"]
    o, lo, ties = compare_logs(w, lg, n, 13)
    compare_states(g, o, w.n_sites)
