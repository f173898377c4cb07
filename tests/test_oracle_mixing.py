"""How fast the chain decorrelates per trial under the paper's global rule and
under the domain-local coloured schedule (the oracle, config 1: one 50-site
chain with 64 ion pairs in L = 40, pure CR-MC without MD).

Domain-local moves keep every domain's net charge; only the per-sweep shift of
the domain grid moves charge between domains.  On this dilute system that
makes the degree of ionisation decorrelate much more slowly per trial with
domains of two half-cutoff cells than with the global rule, and domains of
four cells (2 r_c, one per colour) recover most of the difference.  Both
schedules sample the same distribution (pinned elsewhere); this test records
the cost in trials, which a trials/s figure does not show.  (With an MD step
after every sweep, as in the hybrid cycle, the chains' relaxation under MD is
slower still and sets the pace for both schedules; tau_trials(md=True) measures
that, too slowly for this suite.)"""
import math

import numpy as np

import oracle
from paper_2109_07527_gb300 import workloads as W


def tau_trials(schedule, m, domain_cells=None, samples=1500, every=512, workload=None, md=False):
    """Integrated autocorrelation time of the ionised-site count, in trials
    (FFT autocorrelation, self-consistent window of five times tau), for
    config 1 or the given workload.  The half-size polyelectrolyte figures
    quoted beside this test's come from workload=W.config2(seed=2, scale=0.5),
    samples=1200, every=640 (1.3 x 10^6 trials each, a few minutes).  md=True
    adds one velocity-Verlet/Langevin step (dt 0.005, gamma 1) after every
    sweep, as in the hybrid MD/CR-MC cycle."""
    w = workload if workload is not None else W.config1(seed=1)
    o = oracle.Oracle(w, schedule=schedule, trials_per_domain=m, domain_cells=domain_cells)
    tps = o.trials_per_sweep
    reps = max(1, every // tps)
    if md:
        for i in range(max(1, 200000 // tps)):
            o.sweep(tps, 1 + i)
            o.md_step(1, 0.005, 1.0, 7 + i)
    else:
        o.sweep(tps * max(1, 200000 // tps), 1)
    x = []
    for i in range(samples):
        for r in range(reps):
            o.sweep(tps, 1000 + 100 * i + r)
            if md:
                o.md_step(1, 0.005, 1.0, 50000 + 100 * i + r)
        x.append(o.counts()["n_Am"])
    x = np.asarray(x, float) - np.mean(x)
    n = len(x)
    f = np.fft.rfft(x, 2 * n)
    ac = np.fft.irfft(f * np.conj(f))[:n]
    ac /= ac[0]
    tau = 1.0
    for k in range(1, n):
        tau += 2.0 * ac[k]
        if k >= 5.0 * tau:
            break
    return max(tau, 1.0) * tps * reps


def test_domain_local_schedule_mixing_cost():
    t_global = tau_trials(1, 512)
    t_two = tau_trials(0, 1)                    # 64 domains of 2^3 half-cutoff cells
    t_four = tau_trials(0, 8, domain_cells=4)   # 8 domains of 4^3 cells (2 r_c wide)
    assert t_two > 4.0 * t_global, (t_global, t_two, t_four)
    assert t_four < 0.5 * t_two, (t_global, t_two, t_four)
    assert math.isfinite(t_four)
