#!/usr/bin/env python
"""Benchmark of the CR-MC hot path on GB300 (prints one JSON line).

Workload: the polyelectrolyte solution the metric is quoted on -- 16 chains x
200 acid beads (pKa 4.5), L = 120 sigma, ~4000 ion pairs, r_c = 12 sigma,
l_B = 2 sigma -- titrated at pH 2.0, 2.5, ..., 8.0: 13 replicas advanced as one
batch (one phase launch per colour covers all of them), synthetic seeded
coordinates.  One step = one MD/CR-MC cycle of every replica: one
velocity-Verlet/Langevin MD step (dt = 0.005, gamma = 1) with 10^4 CR-MC trials
(one sweep of 1000 domains x 10 trials) between its drift and its force
evaluation, so that one force evaluation serves both; the full job is 100 steps
(10^6 trials per replica).
The single-replica (pH 4.5) plain path is reported beside it, and the
surrogate delayed-acceptance path ("surrogate_da"): training pairs recorded by
logged DA sweeps, the MLP trained on the tensor cores (throughput against the
BF16 tensor peak), then the same batched cycle with DA sweeps.  Inputs are
resident in HBM; L2 is flushed (256 MB write) between timed steps.

--impl reference times the CPU oracle on the same workload (rank 0 only).
Under torchrun each rank runs its own 13-replica batch of the same workload
with its own seeded structure (no collective on the data path; scaling
"weak"); the timed regions are bracketed by barriers and the slowest rank's
time divides the units of all ranks.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CR-MC trials/s on 1 GB300 (plain vs surrogate-DA/batched) at |Δα|≤0.005"
WORKLOAD = ("polyelectrolyte solution, pH swept 2..8 in steps of 0.5 (13 replicas in one batch): 16 chains x 200 "
            "acid beads (pKa 4.5), L=120 sigma, ~4000 ion pairs, rc=12, lB=2, DSF alpha=0.2; step = 1e4 CR-MC trials "
            "per replica (1000 domains x 10) inside 1 MD step (dt 0.005, gamma 1; the trials run between the drift "
            "and the force evaluation, one force evaluation per step) per replica")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-da", action="store_true")
    ap.add_argument("--no-config4", action="store_true")
    ap.add_argument("--no-fig2", action="store_true")
    ap.add_argument("--no-config3", action="store_true")
    ap.add_argument("--train-only", action="store_true",
                    help="time only the surrogate's training step (batch 32,768, synthetic features) and exit")
    ap.add_argument("--mobile-only", action="store_true",
                    help="time only the MD/CR-MC cycles of the two rigid nanoparticles and exit")
    ap.add_argument("--ewald-only", action="store_true",
                    help="time only CR-MC sweeps with Ewald electrostatics (the 500-acid box of the method "
                         "comparison, 64 replicas, |n| <= 16, global schedule) and exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device):
    """The largest value of x over all ranks (every rank must call it); x
    itself when no process group is initialised or it has one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed (each rank does the
    same fixed work, weak scaling) over the slowest rank's time."""
    return units_per_rank * world / seconds


def workload(rank):
    from paper_2109_07527_gb300 import workloads as W
    return W.config2(seed=1 + rank, pH=4.5, trials_per_domain=10)


def bytes_per_trial(L, rc, n_particles):
    """Algorithmic bytes of one trial: for each of the 2 changed particles the
    27-cell stencil at the reference cell side a = L / floor(L / rc), 16 B per
    particle (float4 position + charge), plus 64 B for the commit."""
    a = L / math.floor(L / rc)
    rho = n_particles / L ** 3
    return 2.0 * 27.0 * a ** 3 * rho * 16.0 + 64.0


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBps", "hbm"):
                if k in d:
                    return float(d[k]), "measured"
        except (OSError, ValueError):
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_sha():
    h = hashlib.sha256()
    for f in ("crmc_phase.cu", "crmc_device.cuh", "crmc_common.h"):
        h.update(open(os.path.join(ROOT, "paper_2109_07527_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the phase kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "cr_phase_polyelectrolyte_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("kernel_sha") != kernel_sha():
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of the SM clock and the throttle reasons every
    `period_ms`; stop() summarises the samples received inside [t0, t1]
    (host perf_counter times bracketing the timed region)."""

    def __init__(self, period_ms=50, smi="nvidia-smi"):
        self.proc = None
        self.rows = []
        self.period_ms = period_ms
        self.smi = smi

    def start(self, wait_s=5.0):
        """Start sampling and wait (at most wait_s) for the first sample, so
        that the sampler is live when the timed region begins."""
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen([self.smi, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.period_ms)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        end = time.perf_counter() + wait_s
        while not self.rows and time.perf_counter() < end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def stop(self, gpu_index, t0=None, t1=None, wait_s=2.0):
        if self.proc is None:
            return None
        # a timed region shorter than the period may hold no sample: wait (at
        # most wait_s) for the first one after its start
        end = time.perf_counter() + wait_s
        while (t0 is not None and not any(t >= t0 for t, _ in list(self.rows)) and time.perf_counter() < end
               and self.proc.poll() is None):
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        mine = [(t, r) for t, r in self.rows if len(r) >= 9 and r[0] == str(gpu_index)]
        inside = [r for t, r in mine if (t0 is None or t >= t0) and (t1 is None or t <= t1)]
        # a region shorter than the period: the first sample after its start
        after = [r for t, r in mine if t0 is not None and t >= t0][:1]
        rows = inside or after
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_in_region": len(inside),
                "period_ms": self.period_ms}


def host_cpu():
    """(model name, logical CPUs) of the host, from lscpu or /proc/cpuinfo."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return model or "unknown", os.cpu_count() or 1


def oracle_step(oracles, seed, md_seed, threads):
    """One step of the workload on the oracle: a sweep (10^4 trials at 10
    trials per domain, the GPU's chain) and one MD step of every replica, the
    replicas spread over `threads` host threads (each replica's chain is the
    sequential oracle's; the C calls release the GIL).  Returns the trials."""
    from concurrent.futures import ThreadPoolExecutor

    def one(o):
        o.sweep(o.trials_per_sweep, seed)
        o.md_step(1, 0.005, 1.0, md_seed)
        return o.trials_per_sweep

    if threads <= 1:
        return sum(one(o) for o in oracles)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return sum(ex.map(one, oracles))


def cpu_baseline(ws):
    """The oracle as it stands, on a bounded sample of the workload: one step
    (one 10^4-trial sweep at 10 trials per domain + one MD step) of the pH 4.5
    replica on one host thread, and one step of all 13 replicas with one
    replica per host thread."""
    import oracle
    model, ncpu = host_cpu()
    o1 = oracle.Oracle(ws[5])
    t0 = time.perf_counter()
    n1 = oracle_step([o1], 1000, 5, 1)
    dt1 = time.perf_counter() - t0
    threads = max(1, min(ncpu, len(ws)))
    os_ = [oracle.Oracle(w) for w in ws]
    t0 = time.perf_counter()
    n = oracle_step(os_, 1000, 5, threads)
    dt = time.perf_counter() - t0
    alphas = []  # every pH point's degree of ionisation after the step's sweep (MD leaves it alone)
    for o in os_:
        c = o.counts()
        alphas.append(c["n_Am"] / c["n_A"] if c["n_A"] > 0 else 0.0)
    return {"value": n / dt, "unit": "trials/s", "cores": threads, "kind": "oracle",
            "sample": f"one step of the 13-replica workload ({len(ws)} x {os_[0].trials_per_sweep} trials at 10 "
                      f"trials per domain + 1 MD step each, the GPU's chain), one replica per host thread, "
                      f"{dt:.1f} s",
            "cpu_model": model, "nproc": ncpu,
            "single_thread": {"value": n1 / dt1, "unit": "trials/s", "cores": 1,
                              "sample": f"one step of the pH {ws[5].params['pH']} replica ({n1} trials + 1 MD step), "
                                        f"{dt1:.1f} s"}}, alphas


def alpha_check(crmc, ws, alphas_o):
    """The metric's accuracy condition on the same sample, across the pH
    sweep: the GPU path runs the oracle's sweep of every pH point (same
    seed, same workload) and each degree of ionisation must be within 0.005
    of the oracle's (the chains are the same trial by trial, so the difference
    is 0 unless a decision fell within the tie band)."""
    ag = []
    for w in ws:
        g = crmc.Context(w)
        g.sweep(g.trials_per_sweep, 1000)
        ag.append(g.counts()["alpha"])
        g.close()
    d = [abs(a - b) for a, b in zip(ag, alphas_o)]
    return {"sample": f"every pH point ({len(ws)}), one sweep of {ws[0].params['trials_per_domain']} trials per "
                      f"domain, GPU vs oracle",
            "pH": [w.params["pH"] for w in ws], "alpha_gpu": ag, "alpha_oracle": alphas_o,
            "max_abs_diff": max(d), "bound": 0.005, "within": max(d) <= 0.005}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    ws = ph_sweep_workloads(0)
    model, ncpu = host_cpu()
    threads = max(1, min(ncpu, len(ws)))
    os_ = [oracle.Oracle(w) for w in ws]
    for s in range(args.warmup):
        oracle_step(os_, 7 + s, 3 + s, threads)
    t0 = time.perf_counter()
    n = 0
    for s in range(args.steps):
        n += oracle_step(os_, 100 + s, 5000 + s, threads)
    dt = time.perf_counter() - t0
    v = n / dt
    sample = (f"{args.steps} steps of the 13-replica workload, each a sweep of {os_[0].trials_per_sweep} trials "
              f"(10 per domain, the GPU's chain) + 1 MD step per replica, one replica per host thread "
              f"({threads} threads on {ncpu} CPUs, {model}), {dt:.1f} s")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "trials/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle", "replicas": len(ws)},
           "cpu_baseline": {"value": v, "unit": "trials/s", "cores": threads, "kind": "oracle", "sample": sample,
                            "cpu_model": model, "nproc": ncpu},
           "e2e": {"value": v, "unit": "trials/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def ph_sweep_workloads(rank):
    """The polyelectrolyte solution at pH 2.0, 2.5, ..., 8.0 (13 replicas of
    the same seeded starting structure)."""
    import copy
    base = workload(rank)
    out = []
    for i in range(13):
        w = copy.copy(base)
        w.params = dict(base.params)
        w.params["pH"] = 2.0 + 0.5 * i
        out.append(w)
    return out


def measured_tensor_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("bf16_tflops", "bf16_TFLOPs"):
                if k in d:
                    return float(d[k]), "measured"
        except (OSError, ValueError):
            pass
    return FALLBACK_BF16_TFLOPS, "fallback"


# unlogged sweeps that time every launch shape once: 12 plain shapes for a
# context; for a batch each of them also as a persistent sweep (24)
TUNE_SWEEPS = 26  # the context tuner: 12 shapes, two passes
BATCH_TUNE_SWEEPS = 50  # the batch tuner: 12 shapes in two launch forms, two passes

# exact (feature, pair energy) pairs recorded for the surrogate's training
TRAIN_PAIRS = 1_000_000

# floating-point operations of one training row (algorithmic, K = 48 input):
# forward 48x128 + 2 x 128x128, backward 4 x 128x128 + 128x48, 2 flops per MAC
TRAIN_FLOPS_PER_ROW = 2 * (48 * 128 + 2 * 128 * 128) + 2 * (4 * 128 * 128 + 128 * 48)


def run_da(crmc, torch, stream, flush, ws, dt, gamma, steps):
    """Surrogate delayed acceptance: record (feature, pair-energy) pairs with
    logged DA sweeps (zero surrogate: stage 1 is the chemistry alone), train the
    MLP on the tensor cores, then time the batched DA cycle with it."""
    from paper_2109_07527_gb300 import workloads as W
    rng = np.random.default_rng(0)
    gd = crmc.Context(ws[5])  # pH 4.5
    gd.set_surrogate(W.random_mlp(seed=5, out_gain=0.0))
    X, y = [], []
    n_rec, s = 0, 0
    while n_rec < TRAIN_PAIRS:  # exact (feature, pair dE) pairs of the polyelectrolyte box, one MD step between sweeps
        r = gd.sweep_da(gd.trials_per_sweep, 40 + s, log=True, features=True)
        ok = (r["da"]["stage"] > 0) & np.isfinite(r["da"]["lnA2"])
        X.append(r["features"][ok])
        y.append(r["da"]["dE_sur"][ok].astype(np.float64) - r["da"]["lnA2"][ok])
        n_rec += int(ok.sum())
        gd.md_step(1, dt, gamma, 60 + s)
        s += 1
    X = np.concatenate(X)
    y = np.concatenate(y).astype(np.float32)
    n_hold = len(X) // 10
    Xh, yh = X[:n_hold], y[:n_hold]
    X, y = np.concatenate([X[n_hold:], -X[n_hold:]]), np.concatenate([y[n_hold:], -y[n_hold:]])
    perm = rng.permutation(len(X))
    X, y = X[perm], y[perm]
    Bt = 32768 if len(X) >= 2 * 32768 else 8192
    nb = len(X) // Bt
    Xd = torch.from_numpy(np.ascontiguousarray(X[:nb * Bt])).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y[:nb * Bt])).cuda()
    tr = crmc.Trainer(W.random_mlp(seed=6, gain=0.5), max_batch=Bt, lr=1e-3, target_clip=20.0)
    loss0 = tr.step(Xd.data_ptr(), yd.data_ptr(), Bt, want_loss=True)
    n_train = 300
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(n_train):
        b = k % nb
        tr.step(Xd.data_ptr() + b * Bt * 48 * 4, yd.data_ptr() + b * Bt * 4, Bt)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    loss_end = tr.step(Xd.data_ptr(), yd.data_ptr(), Bt, want_loss=True)
    _, mlp = tr.get()
    tpeak, tkind = measured_tensor_peak()
    tflops = n_train * Bt * TRAIN_FLOPS_PER_ROW / (t_ms / 1e3) / 1e12
    # held-out error of the antisymmetrised surrogate (oracle-free: the library's own DA records)
    gd.set_surrogate(mlp)
    r = gd.sweep_da(gd.trials_per_sweep, 999, log=True, features=False)
    ev = r["da"]["stage"] > 0
    stage1_reject = float(np.mean(r["da"]["stage"][ev] == 1))
    fin = ev & np.isfinite(r["da"]["lnA2"])
    err = np.abs(r["da"]["lnA2"][fin])  # |dE~ - dE_pair|
    sur_err = {"median_kT": float(np.median(err)), "frac_within_1kT": float(np.mean(err < 1.0))}
    gd.close()
    # batched DA cycle, same step definition as the plain batch
    ctxs = [crmc.Context(w) for w in ws]
    for c in ctxs:
        c.set_surrogate(mlp)
    b = crmc.Batch(ctxs)
    b.sweep_da(22, 0xDA)  # launch-shape tuning of the DA variant (5 shapes in both launch forms, two passes)
    for s in range(3):
        b.cycle(1, dt, gamma, 1 + s, 1000 + s, da=True)

    def step(s):
        b.cycle(1, dt, gamma, 200 + s, 6000 + s, da=True)

    ms = time_steps(step, steps, stream, flush)
    for c in ctxs:
        c.check()
    per_step = ctxs[0].trials_per_sweep * len(ctxs)
    out = {"value": per_step * steps / (ms / 1e3), "unit": "trials/s", "steps": steps, "ms_per_step": ms / steps,
           "launch_shape": None, "stage1_reject_frac": stage1_reject, "surrogate_error": sur_err,
           "alpha_end": [round(c.counts()["alpha"], 4) for c in ctxs],
           "train": {"pairs_recorded": int(n_rec), "recording_sweeps": s, "rows": int(nb * Bt), "batch": Bt,
                     "steps": n_train, "ms": t_ms,
                     "rows_per_s": n_train * Bt / (t_ms / 1e3), "loss_first": loss0, "loss_end": loss_end,
                     "held_out_pairs": int(n_hold),
                     "roofline": {"bound": "tensor", "achieved": tflops, "peak": tpeak, "unit": "TFLOP/s",
                                  "frac": tflops / tpeak, "peak_source": tkind,
                                  "flops_per_row": TRAIN_FLOPS_PER_ROW}}}
    b.close()
    for c in ctxs:
        c.close()
    out["config5"] = run_config5(crmc, torch, stream, flush, mlp, steps)
    return out


def run_config5(crmc, torch, stream, flush, mlp, steps):
    """The large box of the learned stage: 100 x 200 acid beads (pKa 4.5, pH
    4.5), L = 250, ~25,000 ion pairs, with the surrogate trained on the
    polyelectrolyte pairs: plain sweeps against delayed-acceptance sweeps,
    each timed after its own launch-shape tuning (L2 flushed between
    sweeps), and the stage-1 rejection rate of a logged DA sweep."""
    from paper_2109_07527_gb300 import workloads as W
    w5 = W.config5(seed=1)
    g = crmc.Context(w5)
    tps = g.trials_per_sweep
    g.sweep(tps * TUNE_SWEEPS, 0x55)
    ms_plain = time_steps(lambda s: g.sweep(tps, 300 + s), steps, stream, flush)
    a_plain = g.counts()["alpha"]
    g.close()
    h = crmc.Context(w5)
    h.set_surrogate(mlp)
    h.sweep_da(tps * 11, 0x55)  # DA shapes (5, two passes)
    ms_da = time_steps(lambda s: h.sweep_da(tps, 300 + s), steps, stream, flush)
    a_da = h.counts()["alpha"]
    r = h.sweep_da(tps, 999, log=True, features=False)
    ev = r["da"]["stage"] > 0
    rej = float(np.mean(r["da"]["stage"][ev] == 1))
    counted = float(np.mean(ev))
    h.close()
    v_plain, v_da = tps * steps / (ms_plain / 1e3), tps * steps / (ms_da / 1e3)
    return {"workload": f"100 x 200 acid beads, L=250, {w5.n} particles, {w5.n_sites} sites, pH 4.5; "
                        f"{tps} trials per sweep", "steps": steps,
            "plain": {"value": v_plain, "unit": "trials/s", "ms_per_sweep": ms_plain / steps, "alpha_end": a_plain},
            "surrogate_da": {"value": v_da, "unit": "trials/s", "ms_per_sweep": ms_da / steps, "alpha_end": a_da,
                             "stage1_reject_frac": rej, "evaluated_frac": counted},
            "da_over_plain": v_da / v_plain}


def run_method_comparison(crmc, n_rep=128, blocks=40, m=250, ewald_kmax=0):
    """Sec. III.A / Fig. 2: alpha(trials) of the weak-acid electrolyte under
    CR-MC, the grand-reaction ensemble and RxMC (the same random starts), and
    the trials each needs to come within 5 % of CR-MC's plateau; with
    ewald_kmax > 0 under Ewald electrostatics (the paper's energy model) with
    the trials/s of each method's batch sweeps."""
    import time
    from paper_2109_07527_gb300 import methods
    t0 = time.perf_counter()
    r = methods.compare_convergence(crmc, n_rep=n_rep, blocks=blocks, m=m, seed=1, ewald_kmax=ewald_kmax)
    plateau = float(np.mean(r["crmc"][blocks // 2:]))
    t95 = {}
    for k in ("crmc", "grxmc", "rxmc"):
        a = np.asarray(r[k])
        hit = np.flatnonzero(np.abs(a - plateau) <= 0.05 * plateau)
        t95[k] = int(r["trials"][hit[0]]) if len(hit) else None
    energy = (f"Ewald: real space r_c = 10 l_B, alpha = 0.15/sigma, reciprocal |n| <= {ewald_kmax}" if ewald_kmax
              else "DSF r_c = 10 l_B")
    trials = n_rep * (r["trials"][-1] - r["trials"][blocks // 2 - 1])  # the timed second half of the blocks
    return {"workload": f"500 acid groups (pKa 6.5), L = 50 l_B, pH 7, pI_S = 2, {energy}, "
                        "global schedule, no ions at the start",
            "replicas_per_method": n_rep, "trials": r["trials"],
            "trials_per_s": {k: trials / r[k + "_sweep_s"] for k in ("crmc", "grxmc", "rxmc")},
            "alpha": {k: [round(x, 4) for x in r[k]] for k in ("crmc", "grxmc", "rxmc")},
            "alpha_plateau_crmc": plateau,
            "alpha_plateau_grxmc": float(np.mean(r["grxmc"][blocks // 2:])),
            "alpha_plateau_rxmc": float(np.mean(r["rxmc"][blocks // 2:])),
            "trials_to_within_5pct": t95, "wall_s": time.perf_counter() - t0}


def run_train_only(args):
    """The surrogate's training step alone, at the DA leg's batch (32,768 rows
    of 48 integer features; the targets a fixed linear map of them), timed
    with CUDA events after warm-up: a short program for profiling the fused
    training kernel."""
    import torch
    from paper_2109_07527_gb300 import crmc, workloads as W
    B = 32768
    rng = np.random.default_rng(0)
    X = rng.integers(-6, 7, (4 * B, 48)).astype(np.float32)
    y = (0.1 * X[:, 0] - 0.05 * X[:, 8]).astype(np.float32)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    tr = crmc.Trainer(W.random_mlp(seed=6, gain=0.5), max_batch=B, lr=1e-3, target_clip=20.0)
    stream = torch.cuda.current_stream()

    def step(k):
        b = k % 4
        tr.step(Xd.data_ptr() + b * B * 48 * 4, yd.data_ptr() + b * B * 4, B)

    for k in range(max(3, args.warmup)):
        step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    tpeak, tkind = measured_tensor_peak()
    tflops = B * TRAIN_FLOPS_PER_ROW / (ms / 1e3) / 1e12
    print(json.dumps({"metric": "surrogate training rows/s (fused tcgen05 step, batch 32768)",
                      "value": B / (ms / 1e3), "unit": "rows/s", "steps": args.steps, "ms_per_step": ms,
                      "roofline": {"bound": "tensor", "achieved": tflops, "peak": tpeak, "unit": "TFLOP/s",
                                   "frac": tflops / tpeak, "peak_source": tkind}}), flush=True)
    tr.close()


def run_ewald_only(args):
    """CR-MC sweeps of the method comparison's weak-acid electrolyte under
    Ewald electrostatics (|n| <= 16, alpha = 0.15/sigma, r_c = 10 l_B; global
    schedule): 64 replicas in one batch, the launch shape tuned first, then
    `steps` sweeps of 250 trials per replica timed with CUDA events between
    profiler start / stop (a short program for profiling the Ewald trials)."""
    import torch
    from paper_2109_07527_gb300 import crmc, workloads as W
    n_rep, m = 64, 250
    ws = [W.weak_acid_electrolyte(n_acid=500, seed=1 + r, trials_per_domain=m) for r in range(n_rep)]
    for w in ws:
        w.params["ewald_kmax"] = 16
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(BATCH_TUNE_SWEEPS + max(3, args.warmup), 11)  # the tuner's sweeps and the warm-up
    ctxs[0].check()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.profiler.start()
    e0.record(stream)
    b.sweep(args.steps, 12)
    e1.record(stream)
    torch.cuda.profiler.stop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ctxs[0].check()
    print(json.dumps({"metric": "CR-MC trials/s with Ewald electrostatics (global schedule)",
                      "value": n_rep * m / (ms / 1e3), "unit": "trials/s", "steps": args.steps,
                      "ms_per_sweep": ms, "replicas": n_rep, "trials_per_sweep": m,
                      "launch_shape": list(b.launch_shape()),
                      "alpha_end": float(np.mean([c.counts()["alpha"] for c in ctxs]))}), flush=True)
    b.close()
    for c in ctxs:
        c.close()


def run_mobile_only(args):
    """The two-nanoparticle system with rigid bodies (the bench leg
    `mobile_nanoparticles`) alone: the tuner's and warm-up steps, then `steps`
    MD/CR-MC cycles timed with CUDA events between profiler start / stop (a
    short program for profiling the rigid-body cycle)."""
    import torch
    from paper_2109_07527_gb300 import crmc
    crmc._lib()
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def bracket(fn, steps, stream_, flush_):
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        ms = time_steps(fn, steps, stream_, flush_)
        torch.cuda.profiler.stop()
        return ms

    out = run_config3_mobile(crmc, torch, stream, flush, args.steps, timer=bracket)
    print(json.dumps({"metric": "MD/CR-MC cycles/s, two rigid nanoparticles", **out}), flush=True)


def run_config4(crmc, torch, stream, flush, steps):
    """The batched titration: 64 replicas, chain lengths log-uniform in
    [50, 1000], pH uniform in [2, 10], boxes at 10^-3 monomers per sigma^3
    (36.8 to 100 sigma), one batch; each step one MD/CR-MC cycle of every
    replica (one sweep inside one MD step), through the captured cycle."""
    from paper_2109_07527_gb300 import workloads as W
    ws = W.config4(seed=1)
    ctxs = [crmc.Context(w) for w in ws]
    b = crmc.Batch(ctxs)
    b.sweep(BATCH_TUNE_SWEEPS, 0x44)
    g0 = ctxs[0]
    g0.set_timing(True)
    for s in range(3):
        b.cycle(1, 0.005, 1.0, 1 + s, 1000 + s)
    g0.timing(reset=True)
    ms = time_steps(lambda s: b.cycle(1, 0.005, 1.0, 100 + s, 5000 + s), steps, stream, flush)
    tm = g0.timing(reset=True)
    for g in ctxs:
        g.check()
    per_step = sum(g.trials_per_sweep for g in ctxs)
    out = {"workload": "64 replicas, N log-uniform in [50, 1000], pH uniform in [2, 10], pKa 5, "
                       "1e-3 monomers per sigma^3, 10 mM", "replicas": len(ctxs), "trials_per_step": per_step,
           "value": per_step * steps / (ms / 1e3), "unit": "trials/s", "steps": steps, "ms_per_step": ms / steps,
           "sweep_launches_per_step": tm["phase_launches"] / steps,
           "sweep_kernel_ms_per_step": tm["phase_ms"] / steps, "launch_shape": list(b.launch_shape())}
    b.close()
    for g in ctxs:
        g.close()
    return out


def run_config3_mobile(crmc, torch, stream, flush, steps, timer=None):
    """The two-nanoparticle system as a full MD run with mobile rigid
    nanoparticles: 2 x 1000 sites (acids pKa 4 on one, bases pKb 4 on the
    other) on spheres of radius 5 at 12 sigma, L = 100, 20 mM salt, pH 7; each
    nanoparticle (core and sites) one rigid body; each step one MD step
    (dt 0.005, Langevin damping time 20) around one CR-MC sweep."""
    from paper_2109_07527_gb300 import workloads as W
    w = W.config3(separation=12.0, seed=1)
    g = crmc.Context(w)
    g.set_rigid_bodies(*w.meta["bodies"])
    dt, gamma = 0.005, 0.05
    n = g.trials_per_sweep

    def step(s):
        g.md_begin(dt, gamma, 7000 + s)
        g.sweep(n, 9000 + s)
        g.md_end(dt, gamma, 7000 + s)

    for s in range(TUNE_SWEEPS + 4):  # the launch-shape tuner's sweeps and a warm-up
        step(s)
    b0 = g.rigid_body_state()
    ms = (timer or time_steps)(lambda s: step(100 + s), steps, stream, flush)
    b1 = g.rigid_body_state()
    g.check()
    st = g.state()
    out = {"workload": "two nanoparticles (R 5, 1000 sites each) as rigid bodies at 12 sigma, L=100, "
                       "20 mM, pH 7, l_B 0.7, r_c 12", "particles": int(st["n"]), "trials_per_step": n,
           "md_cr_cycles_per_s": steps / (ms / 1e3), "trials_per_s": n * steps / (ms / 1e3),
           "ms_per_step": ms / steps, "steps": steps,
           "body_displacement": float(np.abs(b1[:, 0:3] - b0[:, 0:3]).max()),
           "alpha_end": float(st["alpha"])}
    g.close()
    return out


def run_ewald_md(crmc, torch, stream, flush, steps):
    """MD/CR-MC cycles of the method comparison's weak-acid electrolyte (500
    acids, L = 100, pH 7) under Ewald electrostatics (alpha 0.15, r_c 20,
    |n| <= 16, global schedule) against the same box with the DSF energy
    (r_c 20): each step one MD step (dt 0.005, gamma 1) around one sweep of
    250 trials; the force evaluations timed by CUDA events."""
    from paper_2109_07527_gb300 import workloads as W
    out = {"workload": "weak-acid electrolyte, 500 acids, L=100, pH 7, alpha 0.15, r_c 20, global schedule, "
                       "one MD step around 250 trials per step"}
    for name, kmax in (("ewald", 16), ("dsf", 0)):
        w = W.weak_acid_electrolyte(n_acid=500, L=100.0, pH=7.0, rc=20.0, seed=1, trials_per_domain=250)
        w.params["ewald_kmax"] = kmax
        g = crmc.Context(w)
        n = g.trials_per_sweep

        def step(s):
            g.md_begin(0.005, 1.0, 300 + s)
            g.sweep(n, 500 + s)
            g.md_end(0.005, 1.0, 300 + s)

        for s in range(40):  # ions appear, the launch-shape tuner settles
            step(s)
        g.set_timing(True)
        g.timing(reset=True)
        ms = time_steps(lambda s: step(1000 + s), steps, stream, flush)
        tm = g.timing(reset=True)
        g.check()
        st = g.state()
        out[name] = {"md_cr_cycles_per_s": steps / (ms / 1e3), "ms_per_step": ms / steps,
                     "md_force_ms_per_eval": tm["md_ms"] / max(1, tm["md_launches"]),
                     "particles": int(st["n"]), "alpha_end": float(st["alpha"])}
        g.close()
    return out


def time_steps(step_fn, steps, stream, flush):
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for s in range(steps):
        starts[s].record(stream)
        step_fn(s)
        ends[s].record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    return sum(starts[s].elapsed_time(ends[s]) for s in range(steps))


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    from paper_2109_07527_gb300 import crmc

    dt, gamma = 0.005, 1.0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peak()

    # ---- batched pH sweep (the timed workload)
    ws = ph_sweep_workloads(rank)
    ctxs = [crmc.Context(w) for w in ws]
    batch = crmc.Batch(ctxs)
    per_rep = ctxs[0].trials_per_sweep
    per_step = per_rep * len(ctxs)
    batch.sweep(BATCH_TUNE_SWEEPS, 0xABC)  # launch-shape tuning (one shape and launch form per sweep)
    g0 = ctxs[0]
    g0.set_timing(True)  # before the warm-up, so that the captured cycle already records the phase kernel's events
    for s in range(args.warmup):
        batch.cycle(1, dt, gamma, 1 + s, 1000 + s)
    for g in ctxs:
        g.check()
    clocks = ClockSampler(period_ms=20)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    g0.timing(reset=True)

    def step(s):  # one MD step with the replicas' trials between its drift and its force evaluation (one graph)
        batch.cycle(1, dt, gamma, 100 + s, 5000 + s)

    t_region0 = time.perf_counter()
    torch.cuda.profiler.start()  # (a profiler started with capture off records the timed region only)
    ms = time_steps(step, args.steps, stream, flush)
    torch.cuda.profiler.stop()
    t_region1 = time.perf_counter()
    if world > 1:
        torch.distributed.barrier()
    cl = clocks.stop(local, t_region0, t_region1)
    tm = g0.timing(reset=True)
    g0.set_timing(False)
    for g in ctxs:
        g.check()
    ms = max_over_ranks(ms, "cuda")
    value = job_rate(per_step * args.steps, world, ms / 1e3)
    counts = [g.counts() for g in ctxs]
    L = float(ws[0].params["box_L"])
    rc = float(ws[0].params["rc"])
    info = g0.info
    # the batch's sweep kernel: one persistent launch per sweep (every colour
    # of every replica), or one launch per colour
    launches_per_step = tm["phase_launches"] / args.steps
    trials_per_launch = per_rep / launches_per_step  # per replica
    bytes_launch = sum(trials_per_launch * bytes_per_trial(L, rc, c["n"]) for c in counts)
    avg_launch_s = tm["phase_ms"] / max(tm["phase_launches"], 1) / 1e3
    achieved = bytes_launch / avg_launch_s / 1e9
    kname = ("k_cr_sweep (persistent: all colours of the 13 replicas per launch)" if launches_per_step < 1.5
             else "k_cr_phase (one colour of the 13 replicas per launch)")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profiled_traffic(), "kernel": kname,
                "peak_source": peak_kind, "bytes_per_trial_mean": bytes_launch / (trials_per_launch * len(ctxs)),
                "trials_per_launch": trials_per_launch * len(ctxs), "launches_per_step": launches_per_step,
                "avg_launch_us": avg_launch_s * 1e6, "phase_share_of_step": tm["phase_ms"] / ms}

    # ---- plain path: one replica (pH 4.5), same step definition
    plain = None
    if rank == 0:
        w1 = workload(rank)
        g1 = crmc.Context(w1)
        g1.sweep(g1.trials_per_sweep * TUNE_SWEEPS, 0xABC)
        for s in range(3):
            g1.md_begin(dt, gamma, 1000 + s)
            g1.sweep(g1.trials_per_sweep, 1 + s)
            g1.md_end(dt, gamma, 1000 + s)
        g1.set_timing(True)
        g1.timing(reset=True)
        n_plain = max(10, min(args.steps, 50))

        def step1(s):
            g1.md_begin(dt, gamma, 7000 + s)
            g1.sweep(g1.trials_per_sweep, 300 + s)
            g1.md_end(dt, gamma, 7000 + s)

        ms1 = time_steps(step1, n_plain, stream, flush)
        tm1 = g1.timing(reset=True)
        g1.check()
        c1 = g1.counts()
        al = tm1["phase_ms"] / max(tm1["phase_launches"], 1) / 1e3
        tpl1 = g1.trials_per_sweep / (tm1["phase_launches"] / n_plain)
        ach1 = tpl1 * bytes_per_trial(L, rc, c1["n"]) / al / 1e9
        plain = {"value": g1.trials_per_sweep * n_plain / (ms1 / 1e3), "unit": "trials/s", "steps": n_plain,
                 "ms_per_step": ms1 / n_plain, "launch_shape": list(g1.launch_shape()),
                 "roofline": {"achieved": ach1, "frac": ach1 / peak, "avg_launch_us": al * 1e6},
                 "md_force_ms_per_step": tm1["md_ms"] / n_plain, "alpha_end": c1["alpha"]}
        g1.close()

    da = None
    if rank == 0 and not args.no_da:
        da = run_da(crmc, torch, stream, flush, ws, dt, gamma, max(10, min(args.steps, 50)))
    cfg4 = None
    if rank == 0 and not args.no_config4:
        cfg4 = run_config4(crmc, torch, stream, flush, max(10, min(args.steps, 50)))
    cfg3 = None
    if rank == 0 and not args.no_config3:
        cfg3 = run_config3_mobile(crmc, torch, stream, flush, max(10, min(args.steps, 50)))
    fig2 = fig2_ewald = None
    if rank == 0 and not args.no_fig2:
        fig2 = run_method_comparison(crmc)
        fig2_ewald = run_method_comparison(crmc, n_rep=64, blocks=20, ewald_kmax=16)
        fig2_ewald["md_cycles"] = run_ewald_md(crmc, torch, stream, flush, 20)

    # ---- end to end through the public API with host buffers: each step
    # uploads every replica's configuration from pinned host memory, runs the
    # batched cycle and reads every replica's state back
    e2e = None
    if not args.no_e2e:
        # the replicas' configurations live in packed pinned host arrays
        # (replica r from r * stride; allocated once, as a caller coupling the
        # library to its own host-side code would): cr_batch_load_packed
        # uploads them, the batched cycle runs, cr_batch_state_packed reads
        # every new configuration back into the same arrays
        R = len(ctxs)
        stride = max(g.capacity for g in ctxs)
        pk = dict(xyz=torch.empty((R * stride, 3), dtype=torch.float32).pin_memory(),
                  vel=torch.empty((R * stride, 3), dtype=torch.float32).pin_memory(),
                  id=torch.empty(R * stride, dtype=torch.int64).pin_memory(),
                  type=torch.empty(R * stride, dtype=torch.int32).pin_memory(),
                  state=torch.empty(R * stride, dtype=torch.int8).pin_memory(),
                  cls=torch.empty(R * stride, dtype=torch.int32).pin_memory())
        nbuf = torch.zeros(R, dtype=torch.int64).pin_memory()
        ptr = {k: v.data_ptr() for k, v in pk.items()}
        load_ptr = {k: ptr[k] for k in ("xyz", "vel", "type", "cls", "state")}
        batch.state_packed(stride, ptr, nbuf.data_ptr())
        # one untimed step: the cycle after a load has its own graph (forces first), captured here
        batch.load_packed(stride, load_ptr, nbuf.data_ptr())
        batch.cycle(1, dt, gamma, 8999, 9499)
        batch.state_packed(stride, ptr, nbuf.data_ptr())
        e2e_steps = 20
        h2d = d2h = 0
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for s in range(e2e_steps):
            batch.load_packed(stride, load_ptr, nbuf.data_ptr())
            h2d += R * stride * (12 + 12 + 4 + 4 + 1) + 8 * R
            batch.cycle(1, dt, gamma, 9000 + s, 9500 + s)
            batch.state_packed(stride, ptr, nbuf.data_ptr())
            d2h += R * stride * (12 + 12 + 8 + 4 + 1 + 4) + 12 * R
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, "cuda")
        e2e = {"value": job_rate(per_step * e2e_steps, world, te), "unit": "trials/s", "h2d_bytes_per_step": h2d // e2e_steps,
               "d2h_bytes_per_step": d2h // e2e_steps, "steps": e2e_steps,
               "note": "per step: cr_batch_load_packed of the 13 replicas from packed pinned host arrays + the batched "
                       "cycle (1e4 trials per replica inside one MD step) + cr_batch_state_packed readback of every "
                       "replica into the same arrays (whole replica blocks are copied each way)"}

    if rank != 0:
        return
    out = {"metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 pair terms / i64 fixed-point sums and exponent / f64 near ties",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "replicas": len(ctxs), "pH": [w.params["pH"] for w in ws],
                      "l2": "flushed (256 MB write) between timed steps", "trials_per_step": per_step,
                      "md_steps_per_step": 1, "domains_per_replica": info["nd"] ** 3,
                      "cell_side": info["cell_side"], "launch_shape": list(batch.launch_shape()),
                      "alpha_end": [round(c["alpha"], 4) for c in counts],
                      "particles_end": [c["n"] for c in counts],
                      "parallelism": f"{world} GPU(s), independent replica batches"},
           "roofline": roofline, "gpu_launches": tm["launches"],
           "graph_launches_per_step": 1, "kernels_per_step": tm["launches"] / args.steps,
           "clocks": cl, "e2e": e2e, "plain": plain,
           "surrogate_da": da, "batched_titration": cfg4, "method_comparison": fig2,
           "method_comparison_ewald": fig2_ewald, "mobile_nanoparticles": cfg3,
           "md_cr_cycles_per_s": job_rate(args.steps, world, ms / 1e3)}
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"], alphas_o = cpu_baseline(ph_sweep_workloads(0))
        out["alpha_check"] = alpha_check(crmc, ph_sweep_workloads(0), alphas_o)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.train_only:
        run_train_only(a)
    elif a.ewald_only:
        run_ewald_only(a)
    elif a.mobile_only:
        run_mobile_only(a)
    else:
        run_ours(a)
