"""The parity comparator itself, on CPU: fed a log that the oracle wrote
(standing in for a device log), it must pass an exact copy and fail each kind
of planted disagreement -- a move, a chosen particle, a decision outside the
tie band, a dE beyond its tolerance, a final state."""
import numpy as np
import pytest

import oracle
from paper_2109_07527_gb300 import workloads as W
from parity_util import compare_logs, compare_states, de_tol

SEED = 77


@pytest.fixture(scope="module")
def run():
    w = W.config1(seed=1, trials_per_domain=4)
    o = oracle.Oracle(w)
    lo = o.sweep(12 * o.trials_per_sweep, SEED, log=True)["log"]
    return w, lo


def _accepted_finite(lo):
    ok = (lo["flags"] & (oracle.F_NOELIG | oracle.F_EDGE | oracle.F_OVERLAP)) == 0
    return np.flatnonzero(ok & ((lo["flags"] & oracle.F_ACC) != 0) & np.isfinite(lo["dE"]))


def test_exact_copy_passes(run):
    w, lo = run
    _, lo2, ties = compare_logs(w, lo.copy(), len(lo), SEED)
    assert ties == 0
    assert np.array_equal(lo2["flags"], lo["flags"])


def test_planted_move_fails(run):
    w, lo = run
    lg = lo.copy()
    lg["move"][len(lo) // 2] ^= 1
    with pytest.raises(AssertionError, match="move"):
        compare_logs(w, lg, len(lo), SEED)


def test_planted_particle_choice_fails(run):
    w, lo = run
    lg = lo.copy()
    i = _accepted_finite(lo)[3]
    lg["id_a"][i] += 1
    with pytest.raises(AssertionError, match=f"trial {i}"):
        compare_logs(w, lg, len(lo), SEED)


def test_planted_decision_outside_tie_band_fails(run):
    w, lo = run
    lg = lo.copy()
    tau = 1e-6 * lo["S"] + 1e-12
    far = np.flatnonzero(np.abs(lo["lnu"] - lo["lnA"]) > 1e3 * tau)
    i = int(far[len(far) // 3])
    lg["flags"][i] ^= oracle.F_ACC
    with pytest.raises(AssertionError, match=f"trial {i}"):
        compare_logs(w, lg, len(lo), SEED)


def test_planted_dE_beyond_tolerance_fails(run):
    w, lo = run
    lg = lo.copy()
    i = _accepted_finite(lo)[5]
    lg["dE"][i] += 3.0 * de_tol(lo[i:i + 1])[0]
    with pytest.raises(AssertionError, match="dE out of tolerance"):
        compare_logs(w, lg, len(lo), SEED)
    # a NaN or an infinity fails too
    for bad in (np.nan, np.inf):
        lg["dE"][i] = bad
        with pytest.raises(AssertionError, match="dE out of tolerance"):
            compare_logs(w, lg, len(lo), SEED)
    # within the tolerance it passes
    lg["dE"][i] = lo["dE"][i] + 0.5 * de_tol(lo[i:i + 1])[0]
    compare_logs(w, lg, len(lo), SEED)


class _FakeContext:
    """Returns a state read from an oracle, optionally with one site flipped."""

    def __init__(self, o, n_sites, flip=None):
        p = o.particles()
        self.s = dict(p)
        self.s["site_state"] = o.site_states(n_sites).copy()
        if flip is not None:
            self.s["site_state"][flip] ^= 1
        self.s.update(o.counts())
        self.s["net_charge"] = 0

    def state(self):
        return self.s


def test_compare_states_detects_a_flipped_site(run):
    w, _ = run
    o = oracle.Oracle(w)
    o.sweep(4 * o.trials_per_sweep, SEED)
    n_sites = w.n_sites
    compare_states(_FakeContext(o, n_sites), o, n_sites)
    with pytest.raises(AssertionError):
        compare_states(_FakeContext(o, n_sites, flip=0), o, n_sites)
