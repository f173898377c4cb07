"""GPU-vs-oracle comparison helpers for the parity tests.

Protocol (tolerances written here, used by every parity test):
  * moves, chosen particle ids, no-eligible / edge / overlap flags: bit-exact;
  * dE: |dE_gpu - dE_oracle| <= 1e-6 * S + 1e-9, where S >= |dE| is the gross
    magnitude of the summed terms (sum over pair terms of the absolute values
    of their components), the condition scale of FP32 pair terms;
  * accept decisions: identical, except a "tie" where |ln u - lnA_oracle| is
    within tau = 1e-6 * S + 1e-12; the oracle is then re-run with the GPU's
    decision forced at that trial and the comparison continues;
  * the final charge states, ids and positions: identical.
"""
import numpy as np

import oracle

DE_REL = 1e-6
STRUCT_FLAGS = oracle.F_NOELIG | oracle.F_EDGE | oracle.F_OVERLAP


def de_tol(lo):
    """1e-6 relative to S, the gross magnitude of the summed pair terms
    (S >= |dE|; pair terms cancel internally near the cutoffs)."""
    return DE_REL * lo["S"] + 1e-9


def compare_logs(w, lg, n_trials, seed, oracle_kw=None, max_ties=8, prep=None):
    """Run the oracle over the same trials (forcing tie decisions) and
    compare with the GPU trial log.  prep (optional) brings every fresh
    oracle to the state the GPU log starts from (earlier calls, a pH change).
    Returns (oracle, oracle log, ties)."""
    oracle_kw = oracle_kw or {}
    forced = np.full(n_trials, -1, np.int8)
    ties = 0
    while True:
        o = oracle.Oracle(w, **oracle_kw)
        if prep is not None:
            prep(o)
        lo = o.sweep(n_trials, seed, log=True, forced=forced)["log"]
        assert np.array_equal(lg["move"], lo["move"]), _first(lg, lo, "move")
        bad = np.flatnonzero((lg["flags"] & STRUCT_FLAGS) != (lo["flags"] & STRUCT_FLAGS))
        dec = np.flatnonzero((lg["flags"] & oracle.F_ACC) != (lo["flags"] & oracle.F_ACC))
        ids = np.flatnonzero((lg["id_a"] != lo["id_a"]) | (lg["id_b"] != lo["id_b"]))
        first = min([x[0] for x in (bad, dec, ids) if len(x)] or [n_trials])
        if first == n_trials:
            break
        if len(dec) and dec[0] == first and not (len(bad) and bad[0] == first) and not (len(ids) and ids[0] == first):
            tau = 1e-6 * lo["S"][first] + 1e-12
            if abs(lo["lnu"][first] - lo["lnA"][first]) <= tau and ties < max_ties:
                forced[first] = 1 if (lg["flags"][first] & oracle.F_ACC) else 0
                ties += 1
                continue
        raise AssertionError(f"trial {first}: gpu {lg[first]} oracle {lo[first]}")
    ok = (lo["flags"] & (oracle.F_NOELIG | oracle.F_EDGE | oracle.F_OVERLAP)) == 0
    with np.errstate(invalid="ignore"):
        err = np.abs(lg["dE"] - lo["dE"])
    tol = de_tol(lo)
    # written as "not within" so that a NaN or an infinity where the oracle
    # has a finite value (every counted trial) fails
    badi = np.flatnonzero(ok & ~(err <= tol))
    assert len(badi) == 0, "dE out of tolerance:\n" + "\n".join(
        f"  trial {i}: move {lo['move'][i]} gpu dE {lg['dE'][i]!r} oracle dE {lo['dE'][i]!r} S {lo['S'][i]!r} "
        f"gpu S {lg['S'][i]!r} err {err[i]:.3e} tol {tol[i]:.3e}" for i in badi[:8])
    with np.errstate(invalid="ignore"):
        lt = np.abs(lg["lnA"] - lo["lnA"])
    ltol = tol + 1e-12 * np.abs(lo["lnA"])
    badl = np.flatnonzero(ok & ~(lt <= ltol))
    assert len(badl) == 0, "lnA out of tolerance:\n" + "\n".join(
        f"  trial {i}: move {lo['move'][i]} gpu lnA {lg['lnA'][i]!r} oracle lnA {lo['lnA'][i]!r} "
        f"dE {lg['dE'][i]!r}/{lo['dE'][i]!r} tol {ltol[i]:.3e}" for i in badl[:8])
    assert np.array_equal(lg["lnu"], lo["lnu"]) or np.allclose(lg["lnu"], lo["lnu"], rtol=1e-15, atol=0)
    return o, lo, ties


def _first(lg, lo, field):
    i = int(np.flatnonzero(lg[field] != lo[field])[0])
    return f"{field} differs first at trial {i}: gpu {lg[i]} oracle {lo[i]}"


def compare_states(g, o, n_sites):
    sg = g.state()
    so = o.particles()
    assert np.array_equal(sg["id"], so["id"]), "particle ids differ"
    assert np.array_equal(sg["xyz"], so["xyz"]), "positions differ"
    assert np.array_equal(sg["type"], so["type"])
    assert np.array_equal(sg["state"], so["state"])
    assert np.array_equal(sg["site_state"], o.site_states(n_sites))
    co = o.counts()
    for k in ("n", "n_Am", "n_Bp", "n_Xp", "n_Xm", "n_Sp", "n_Sm"):
        assert sg[k] == co[k], (k, sg[k], co[k])
    assert sg["net_charge"] == 0
    return sg, so


def compare_logs_da(w, mlp, lg, dg, fg, n_trials, seed, oracle_kw=None, max_ties=8):
    """Delayed-acceptance run: the oracle with the same surrogate over the same
    trials.  Moves, ids, structural flags, features and the surrogate dE~ are
    bit-exact (the same FP32 operations in the same order on both sides);
    stage-1 decisions may differ only in a tie |ln u - lnA1| <= 1e-9 (the two
    sides round the chemical constants differently), stage-2 decisions only in
    a tie |ln u2 - lnA2| <= 1e-6 S + 1e-12 (the dE tolerance); the oracle is
    re-run with the GPU's stage decision forced there.  dE and lnA as in
    compare_logs.  Returns (oracle, oracle log, oracle DA records, ties)."""
    oracle_kw = oracle_kw or {}
    forced = np.full(n_trials, -1, np.int8)
    ties = 0
    while True:
        o = oracle.Oracle(w, **oracle_kw)
        o.set_surrogate(mlp)
        o.set_da(True)
        r = o.sweep(n_trials, seed, log=True, forced=forced, da_log=True, features=True)
        lo, do, fo = r["log"], r["da"], r["features"]
        assert np.array_equal(lg["move"], lo["move"]), _first(lg, lo, "move")
        bad = np.flatnonzero(((lg["flags"] & STRUCT_FLAGS) != (lo["flags"] & STRUCT_FLAGS)) |
                             (lg["id_a"] != lo["id_a"]) | (lg["id_b"] != lo["id_b"]) |
                             np.any(fg != fo, axis=1) |
                             (dg["dE_sur"].view(np.uint32) != do["dE_sur"].view(np.uint32)))
        st1 = np.flatnonzero(dg["stage"] != do["stage"])
        dec = np.flatnonzero((lg["flags"] & oracle.F_ACC) != (lo["flags"] & oracle.F_ACC))
        first = min([x[0] for x in (bad, st1, dec) if len(x)] or [n_trials])
        if first == n_trials:
            break
        if not (len(bad) and bad[0] == first) and ties < max_ties:
            if len(st1) and st1[0] == first:
                if abs(lo["lnu"][first] - lo["lnA"][first]) <= 1e-9:
                    forced[first] = 2 | (1 if dg["stage"][first] == 2 else 0)
                    ties += 1
                    continue
            elif len(dec) and dec[0] == first:
                tau = 1e-6 * lo["S"][first] + 1e-12
                if abs(do["lnu2"][first] - do["lnA2"][first]) <= tau:
                    f1 = forced[first] if forced[first] >= 0 else 0
                    forced[first] = (f1 & 3) | 8 | (4 if (lg["flags"][first] & oracle.F_ACC) else 0)
                    ties += 1
                    continue
        raise AssertionError(f"trial {first}: gpu {lg[first]} {dg[first]} oracle {lo[first]} {do[first]}\n"
                             f"features gpu {fg[first]} oracle {fo[first]}")
    ok = (lo["flags"] & (oracle.F_NOELIG | oracle.F_EDGE)) == 0
    fin = ok & np.isfinite(lo["dE"])
    assert np.array_equal(np.isfinite(lg["dE"][ok]), np.isfinite(lo["dE"][ok]))
    err = np.abs(lg["dE"][fin] - lo["dE"][fin])
    tol = de_tol(lo[fin])
    assert np.all(err <= tol), ("dE out of tolerance", np.flatnonzero(fin)[err > tol][:8])
    lt = np.abs(lg["lnA"][ok] - lo["lnA"][ok])
    assert np.all(lt <= 1e-9 + 1e-12 * np.abs(lo["lnA"][ok])), ("lnA1 out of tolerance", lt.max())
    l2 = np.abs(dg["lnA2"][fin] - do["lnA2"][fin])
    assert np.all(l2 <= tol + 1e-12 * np.abs(do["lnA2"][fin])), ("lnA2 out of tolerance", l2.max())
    assert np.array_equal(np.isnan(dg["lnu2"]), np.isnan(do["lnu2"]))
    m = ~np.isnan(do["lnu2"])
    assert np.allclose(dg["lnu2"][m], do["lnu2"][m], rtol=1e-15, atol=0)
    return o, lo, do, ties
