"""Pins for the FP64 CPU oracle, against what the paper and mathematics fix.

Each test checks the oracle against something other than itself:
  * Philox4x32-10 known-answer vectors (tests/golden/philox4x32_10_kat.txt).
  * Properties of the DSF pair potential (phi(rc) = phi'(rc) = 0, alpha -> 0
    limit) and of the WCA potential (Eq. LJe: U(sigma) = eps, U(2^(1/6)
    sigma) = 0, expanded distance is a shift).
  * The exact finite-box titration curve of ideal acids/bases, derived from
    Eq. (QQ) with E = 0 and charge neutrality: P(k) ~ C(n,k) K^k (z+/z-)^(k/2)
    I_k(2 sqrt(z+ z-)), and its Henderson-Hasselbalch limit at high salt
    (the Gibbs-Donnan + HH model of App. C).
  * Exact enumeration of all 2^n charge states of n <= 10 interacting sites.
  * Delta E of every accepted trial = E_after - E_before from a brute-force
    total energy (the plain definition of Delta E in Eq. acidacc).
  * Flux symmetry of site-state transitions (detailed balance, Eq. accrat).
  * Charge neutrality after every move and the stationary distribution being
    independent of the schedule (global vs domain-coloured).
"""
import math
import os

import numpy as np
import pytest
from scipy.special import erfc, gammaln, ive

import oracle
from paper_2109_07527_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert out.tolist() == v[6:10]


def test_philox_counter_sensitivity():
    """Changing any counter or key word changes every output word."""
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert np.all(oracle.philox(c, [5, 6]) != base)
    assert np.all(oracle.philox([1, 2, 3, 4], [5, 7]) != base)


# ---------------------------------------------------------------- pair potentials
@pytest.mark.parametrize("alpha,rc", [(0.2, 10.0), (0.2, 12.0), (0.35, 8.0)])
def test_dsf_vanishes_smoothly_at_cutoff(alpha, rc):
    assert abs(oracle.dsf_phi(alpha, rc, rc)) < 1e-15
    assert abs(oracle.dsf_force(alpha, rc, rc)) < 1e-15
    h = 1e-4
    # force is -dphi/dr (central differences, well inside the cutoff)
    for r in (0.9, 1.5, 3.0, rc / 2, rc - 0.5):
        fd = -(oracle.dsf_phi(alpha, rc, r + h) - oracle.dsf_phi(alpha, rc, r - h)) / (2 * h)
        assert abs(fd - oracle.dsf_force(alpha, rc, r)) < 1e-7 * max(1.0, abs(fd))
    # phi(r) - erfc(alpha r)/r is a straight line in r (the shift and the force shift)
    rs = np.linspace(1.0, rc, 7)
    resid = np.array([oracle.dsf_phi(alpha, rc, r) - erfc(alpha * r) / r for r in rs])
    coef = np.polyfit(rs, resid, 1)
    assert np.max(np.abs(np.polyval(coef, rs) - resid)) < 1e-12


def test_dsf_alpha_zero_is_shifted_force_coulomb():
    """alpha -> 0: phi(r) = 1/r - 1/rc + (r - rc)/rc^2 (shifted-force Coulomb)."""
    rc = 10.0
    for r in (0.8, 2.0, 5.0, 9.9):
        sf = 1.0 / r - 1.0 / rc + (r - rc) / rc ** 2
        assert abs(oracle.dsf_phi(0.0, rc, r) - sf) < 1e-14


def test_wca_values():
    c = 2.0 ** (1.0 / 6.0)
    assert abs(oracle.wca_u(1.0, 1.0, 0.0, 1.0) - 1.0) < 1e-14        # U(sigma) = eps
    assert abs(oracle.wca_u(1.0, 1.0, 0.0, c - 1e-12)) < 1e-9          # continuous at the cutoff
    assert oracle.wca_u(1.0, 1.0, 0.0, c + 1e-9) == 0.0
    assert abs(oracle.wca_u(2.5, 1.0, 0.0, 1.0) - 2.5) < 1e-13
    # expanded WCA is the plain one shifted by Delta (Eq. LJe)
    for r in (1.0, 1.05, 1.1):
        assert abs(oracle.wca_u(1.0, 1.0, 4.5, r + 4.5) - oracle.wca_u(1.0, 1.0, 0.0, r)) < 1e-12
    # minimum of 4[(1/s)^12 - (1/s)^6] is -1 at 2^(1/6): with the +eps shift, U(c) = 0
    assert oracle.wca_u(1.0, 1.0, 0.0, 0.5) > 16000.0


def test_expanded_wca_shifts_follow_table_II():
    """The nanoparticle workload's expanded-WCA table against the stored Table
    II rules, and the oracle's potential with those shifts: U = eps at
    r = Delta + sigma, zero from r_c* = Delta + 2^(1/6) sigma on."""
    rows = [ln.split() for ln in open(os.path.join(GOLD, "table2_expanded_wca.txt"))
            if ln.strip() and not ln.startswith("#")]
    R, r_ion = 5.0, 0.5
    rule = {(a, b): eval(f, {"__builtins__": {}}, dict(R=R, r=r_ion)) for a, b, f in rows}
    w = W.config3(separation=12.0, seed=1, L=60.0, n_sites=50)
    p = w.params
    cls = {"ion": 0, "particle": 1}  # short-range classes of free ions and cores
    c = 2.0 ** (1.0 / 6.0)
    for (a, b), delta in rule.items():
        for i, j in ((cls[a], cls[b]), (cls[b], cls[a])):
            assert p["wca_del"][4 * i + j] == delta, (a, b)
            assert p["wca_on"][4 * i + j] == 1
            eps, sig = p["wca_eps"][4 * i + j], p["wca_sig"][4 * i + j]
            assert abs(oracle.wca_u(eps, sig, delta, delta + sig) - eps) < 1e-12
            assert oracle.wca_u(eps, sig, delta, delta + c * sig + 1e-9) == 0.0
            assert oracle.wca_u(eps, sig, delta, delta + c * sig - 1e-3) > 0.0
    assert rule[("particle", "particle")] == 9.0 and rule[("particle", "ion")] == 4.5


# ---------------------------------------------------------------- closed forms
def exact_alpha(n, lnK, ln_zp, ln_zm):
    """<k>/n for P(k) ~ C(n,k) K^k (zp/zm)^(k/2) I_k(2 sqrt(zp zm))."""
    k = np.arange(n + 1)
    s = 2.0 * math.exp(0.5 * (ln_zp + ln_zm))
    logP = (gammaln(n + 1) - gammaln(k + 1) - gammaln(n - k + 1) + k * lnK + 0.5 * k * (ln_zp - ln_zm)
            + np.log(ive(k, s)))
    P = np.exp(logP - logP.max())
    P /= P.sum()
    return float((k * P).sum() / n)


def run_alpha(o, n_sites, n_batches, per_batch, seed, kind="n_Am", burn=None):
    burn = per_batch * 5 if burn is None else burn
    tps = o.trials_per_sweep
    o.sweep(max(tps, (burn // tps) * tps), seed)
    vals = []
    for b in range(n_batches):
        acc = 0.0
        nrep = max(1, per_batch // tps)
        for _ in range(nrep):
            o.sweep(tps, seed + 1 + b)
            acc += o.counts()[kind]
        vals.append(acc / nrep / n_sites)
    vals = np.array(vals)
    return vals.mean(), vals.std(ddof=1) / math.sqrt(len(vals))


@pytest.mark.parametrize("pH,schedule", [(4.0, 1), (5.0, 1), (6.0, 1), (5.0, 0), (4.0, 0)])
def test_ideal_titration_matches_exact_finite_box(pH, schedule):
    n, L, pIS, sig = 50, 40.0, 2.0, 0.355
    w = W.ideal(n_sites=n, L=L, pH=pH, pKa=5.0, pIS=pIS, n_pairs=20, seed=11, schedule=schedule,
                trials_per_domain=4 if schedule == 0 else 256)
    o = oracle.Oracle(w)
    ch = o.chem()
    ln10 = math.log(10.0)
    lnV = math.log(0.602214076 * (L * sig) ** 3)
    a_ex = exact_alpha(n, ln10 * (pH - 5.0), lnV - ln10 * ch["pIX_plus"], lnV - ln10 * ch["pIX_minus"])
    mean, se = run_alpha(o, n, 40, 4096, seed=100 + int(pH * 10) + schedule)
    assert abs(mean - a_ex) <= max(4.0 * se, 0.002), (mean, se, a_ex)
    assert abs(mean - a_ex) <= 0.005


def test_ideal_base_titration_asymmetric_reservoir():
    """Bases at pH 9 (pOH 5) with pI_S+ != pI_S-: uses z+ != z-."""
    n, L, sig = 40, 40.0, 0.355
    w = W.ideal(n_sites=n, L=L, pH=9.0, pKa=5.0, pIS=2.0, n_pairs=20, seed=5, schedule=1, trials_per_domain=256,
                base=True)
    w.params["pIS_minus"] = 2.5
    o = oracle.Oracle(w)
    ch = o.chem()
    ln10 = math.log(10.0)
    lnV = math.log(0.602214076 * (L * sig) ** 3)
    # bases release X-: the roles of z+ and z- swap relative to the acid form
    a_ex = exact_alpha(n, ln10 * (14.0 - 9.0 - 5.0), lnV - ln10 * ch["pIX_minus"], lnV - ln10 * ch["pIX_plus"])
    mean, se = run_alpha(o, n, 40, 4096, seed=7, kind="n_Bp")
    assert abs(mean - a_ex) <= max(4.0 * se, 0.002), (mean, se, a_ex)


def test_henderson_hasselbalch_limit_at_high_salt():
    """At 1 M salt the Donnan correction nearly vanishes: the exact finite-box
    alpha is within 0.005 of Henderson-Hasselbalch 1/(1 + 10^(pKa - pH)), and
    the oracle samples it."""
    n, L, sig, pH, pKa = 50, 30.0, 0.355, 5.0, 5.0
    w = W.ideal(n_sites=n, L=L, pH=pH, pKa=pKa, pIS=0.0, n_pairs=700, seed=2, schedule=1, trials_per_domain=512)
    o = oracle.Oracle(w)
    hh = 1.0 / (1.0 + 10 ** (pKa - pH))
    ch = o.chem()
    ln10 = math.log(10.0)
    lnV = math.log(0.602214076 * (L * sig) ** 3)
    a_ex = exact_alpha(n, 0.0, lnV - ln10 * ch["pIX_plus"], lnV - ln10 * ch["pIX_minus"])
    assert abs(a_ex - hh) < 0.005
    mean, se = run_alpha(o, n, 40, 4096, seed=9, burn=8192)
    assert se < 0.005
    assert abs(mean - a_ex) <= 4.0 * se, (mean, se, a_ex)


def two_state_ratio(lnK, zp, zm, m_max=400):
    """P(ionised) / P(neutral) of one acid site with ideal reservoir ions,
    summed term by term from the grand-canonical weights of Eq. (QQ) with
    E = 0: K^k * sum over anion numbers m of zp^(m+k) zm^m / ((m+k)! m!),
    neutrality fixing the cation number at m + k."""
    def lse(k):
        t = [(m + k) * math.log(zp) + m * math.log(zm) - math.lgamma(m + k + 1) - math.lgamma(m + 1)
             for m in range(m_max)]
        mx = max(t)
        return mx + math.log(sum(math.exp(x - mx) for x in t))
    return math.exp(lnK + lse(1) - lse(0))


@pytest.mark.parametrize("pH,pIS_minus", [(5.0, 2.0), (4.5, 2.5), (5.5, 1.5)])
def test_one_site_two_state_ratio(pH, pIS_minus):
    """A single acid site with ghost ions: the time fraction spent ionised
    against the exact two-state ratio (the ion sums done term by term, not
    through a Bessel function), also with an asymmetric reservoir."""
    L, sig = 40.0, 0.355
    w = W.ideal(n_sites=1, L=L, pH=pH, pKa=5.0, pIS=2.0, n_pairs=20, seed=6, schedule=1, trials_per_domain=256)
    w.params["pIS_minus"] = pIS_minus
    o = oracle.Oracle(w)
    ch = o.chem()
    v = 0.602214076 * (L * sig) ** 3
    r = two_state_ratio(math.log(10.0) * (pH - 5.0), v * 10 ** -ch["pIX_plus"], v * 10 ** -ch["pIX_minus"])
    p_ex = r / (1.0 + r)
    tps = o.trials_per_sweep
    o.sweep(tps * 40, 1)
    B, per = 30, 16384
    f = []
    for b in range(B):
        h = o.sweep(tps * (per // tps), 500 + b, hist_n=1)["hist"]
        f.append(h[1] / h.sum())
    mean, se = float(np.mean(f)), float(np.std(f, ddof=1) / math.sqrt(B))
    assert abs(mean - p_ex) <= max(4.0 * se, 0.003), (mean, se, p_ex)
    assert abs(mean - p_ex) <= 0.01


@pytest.mark.parametrize("schedule", [1, 0])
def test_ideal_salt_pair_distribution(schedule):
    """A box of ghost ions without sites: only the salt moves (Eqs. MCsaltf,
    MCmetro2) act, and the pair number N follows P(N) ~ (z+ z-)^N / (N!)^2
    (Eq. QQ with E = 0 and N+ = N- = N), with an asymmetric reservoir.  Under
    the coloured schedule the domain-local rule must give the same global
    distribution."""
    L, sig = 40.0, 0.355
    w = W.ideal(n_sites=0, L=L, pH=7.0, pIS=2.0, n_pairs=10, seed=3, schedule=schedule,
                trials_per_domain=256 if schedule == 1 else 4)
    w.params["pIS_minus"] = 2.3
    o = oracle.Oracle(w)
    ch = o.chem()
    v = 0.602214076 * (L * sig) ** 3
    ln_zz = math.log(v * 10 ** -ch["pIX_plus"]) + math.log(v * 10 ** -ch["pIX_minus"])
    N = np.arange(80)
    logP = N * ln_zz - 2.0 * gammaln(N + 1)
    P = np.exp(logP - logP.max())
    P /= P.sum()
    tps = o.trials_per_sweep
    o.sweep(tps * 20, 1)
    B, per = 30, 16384
    H = []
    for b in range(B):
        c = []
        for r in range(per // tps):
            o.sweep(tps, 100 + 1000 * b + r)
            k = o.counts()
            assert k["n_Xp"] == k["n_Xm"]
            c.append(k["n_Xm"])
        H.append(np.bincount(c, minlength=len(N))[:len(N)] / len(c))
    H = np.array(H)
    mean_N = (H * N).sum(1)
    m, se = mean_N.mean(), mean_N.std(ddof=1) / math.sqrt(B)
    m_ex = float((P * N).sum())
    assert abs(m - m_ex) <= max(4.0 * se, 0.05), (m, se, m_ex)
    hm, hse = H.mean(0), H.std(0, ddof=1) / math.sqrt(B)
    big = P > 0.02
    z = np.abs(hm - P)[big] / np.maximum(hse[big], 2e-3)
    assert z.max() < 5.0, (z.max(), hm[big], P[big])


@pytest.mark.parametrize("pH,expect", [(1.0, 0.0), (10.0, 1.0)])
def test_titration_limits(pH, expect):
    w = W.ideal(n_sites=20, pH=pH, pKa=5.0, n_pairs=10, seed=4, schedule=1, trials_per_domain=256)
    o = oracle.Oracle(w)
    mean, _ = run_alpha(o, 20, 10, 2048, seed=3)
    assert abs(mean - expect) < 0.01


def test_pIX_grouping_formula():
    """Eq. (pIXgen): 10^-pI_X = 10^-pI_S + 10^-min(pH, pOH); explicit pI_X overrides it."""
    for pH in (2.0, 7.0, 11.0):
        w = W.ideal(n_sites=4, pH=pH, n_pairs=2, seed=1, schedule=1, trials_per_domain=4)
        ch = oracle.Oracle(w).chem()
        ref = -math.log10(10 ** -2.0 + 10 ** -min(pH, 14.0 - pH))
        assert abs(ch["pIX_plus"] - ref) < 1e-12 and abs(ch["pIX_minus"] - ref) < 1e-12
    w = W.ideal(n_sites=4, pH=7.0, n_pairs=2, seed=1, schedule=1, trials_per_domain=4)
    w.params.update(pIX_explicit=1, pIX_plus=7.0, pIX_minus=7.0)
    ch = oracle.Oracle(w).chem()
    assert ch["pIX_plus"] == 7.0 and ch["pIX_minus"] == 7.0


@pytest.mark.parametrize("pH,pIS", [(2.0, 2.0), (4.0, 1.0), (7.0, 2.0), (9.5, 3.0), (12.0, 1.5)])
def test_pIX_from_reservoir_species(pH, pIS):
    """The combined ion activities from the reservoir's species (App. C): salt
    S+/S- at 10^-pIS, H+ and OH- at 10^-pH and 10^-pOH, and the acid anion
    (or base cation) that the reservoir's neutrality requires at a
    non-neutral pH.  Grouping species into one type adds their activities
    (App. B, Eq. mux), so X+ = everything positive and X- = everything
    negative.  The oracle's pI_X+ and pI_X- must be those activities."""
    pOH = 14.0 - pH
    s, h, oh = 10 ** -pIS, 10 ** -pH, 10 ** -pOH
    extra_anion = max(h - oh, 0.0)   # e.g. Cl- of HCl at pH < 7
    extra_cation = max(oh - h, 0.0)  # e.g. Na+ of NaOH at pH > 7
    pos = [s, h, extra_cation]
    neg = [s, oh, extra_anion]
    assert abs(sum(pos) - sum(neg)) <= 1e-15 * sum(pos)  # the reservoir is neutral
    a_plus, a_minus = sum(pos), sum(neg)
    w = W.ideal(n_sites=4, pH=pH, pIS=pIS, n_pairs=2, seed=1, schedule=1, trials_per_domain=4)
    ch = oracle.Oracle(w).chem()
    assert abs(ch["pIX_plus"] + math.log10(a_plus)) < 1e-12
    assert abs(ch["pIX_minus"] + math.log10(a_minus)) < 1e-12


@pytest.mark.parametrize("pH,pIS", [(2.0, 2.0), (4.0, 1.0), (7.0, 2.0), (9.5, 3.0), (12.0, 1.5)])
def test_ungrouped_fractions_from_reservoir_species(pH, pIS):
    """Ungrouping (Sec. II.D): the share of a subspecies in its group is its
    activity over the group's summed activity (the reservoir species of App. C
    as in the test above); reached both at creation and through set_pH."""
    pOH = 14.0 - pH
    s, h, oh = 10 ** -pIS, 10 ** -pH, 10 ** -pOH
    a_plus = s + h + max(oh - h, 0.0)
    a_minus = s + oh + max(h - oh, 0.0)
    want = dict(p_Sp=s / a_plus, p_H=h / a_plus, p_Sm=s / a_minus, p_OH=oh / a_minus)
    w = W.ideal(n_sites=4, pH=pH, pIS=pIS, n_pairs=2, seed=1, schedule=1, trials_per_domain=4)
    o = oracle.Oracle(w)
    w2 = W.ideal(n_sites=4, pH=7.5 if pH != 7.5 else 3.0, pIS=pIS, n_pairs=2, seed=1, schedule=1,
                 trials_per_domain=4)
    o2 = oracle.Oracle(w2)
    o2.set_pH(pH)
    for u in (o.ungroup(), o2.ungroup()):
        for k, v in want.items():
            assert abs(u[k] - v) <= 1e-12 * v, (k, u[k], v)
        assert u["p_Sp"] + u["p_H"] <= 1.0 + 1e-12 and u["p_Sm"] + u["p_OH"] <= 1.0 + 1e-12


@pytest.mark.parametrize("pH0,pH1", [(3.0, 6.0), (6.5, 4.5)])
def test_set_pH_moves_the_titration_to_its_exact_value(pH0, pH1):
    """A time-dependent pH (App. B): an ideal box equilibrated at pH0 and then
    switched to pH1 titrates to the exact finite-box value at pH1 (and pI_X
    follows Eq. pIXgen at the new pH)."""
    n, L, pIS, sig = 50, 40.0, 2.0, 0.355
    w = W.ideal(n_sites=n, L=L, pH=pH0, pKa=5.0, pIS=pIS, n_pairs=20, seed=12, schedule=1, trials_per_domain=256)
    o = oracle.Oracle(w)
    o.sweep(o.trials_per_sweep * 40, 3)
    o.set_pH(pH1)
    ch = o.chem()
    ref = -math.log10(10 ** -pIS + 10 ** -min(pH1, 14.0 - pH1))
    assert abs(ch["pIX_plus"] - ref) < 1e-12 and abs(ch["pOH"] - (14.0 - pH1)) < 1e-12
    ln10 = math.log(10.0)
    lnV = math.log(0.602214076 * (L * sig) ** 3)
    a_ex = exact_alpha(n, ln10 * (pH1 - 5.0), lnV - ln10 * ch["pIX_plus"], lnV - ln10 * ch["pIX_minus"])
    mean, se = run_alpha(o, n, 40, 4096, seed=200 + int(10 * pH1))
    assert abs(mean - a_ex) <= max(4.0 * se, 0.002), (mean, se, a_ex)
    assert abs(mean - a_ex) <= 0.005


# ---------------------------------------------------------------- exact enumeration
def dsf_energy_states(w, n):
    """E(s) for all 2^n site states from the DSF definition (scipy erfc)."""
    p = w.params
    a, rc, lB = p["alpha"], p["rc"], p["lB"]
    c1 = erfc(a * rc) / rc
    c2 = erfc(a * rc) / rc ** 2 + 2 * a / math.sqrt(math.pi) * math.exp(-a * a * rc * rc) / rc
    self_c = -(erfc(a * rc) / (2 * rc) + a / math.sqrt(math.pi))
    L = np.float32(p["box_L"]).astype(np.float64)
    x = w.xyz[:n].astype(np.float64)
    qion = np.where(w.type[:n] == W.ACID, -1.0, 1.0)
    E = np.zeros(1 << n)
    for s in range(1 << n):
        q = np.array([qion[i] if (s >> i) & 1 else 0.0 for i in range(n)])
        e = lB * self_c * float(q @ q)
        for i in range(n):
            for j in range(i + 1, n):
                d = x[i] - x[j]
                d -= L * np.round(d / L)
                r = float(np.sqrt(d @ d))
                if r < rc and q[i] != 0 and q[j] != 0:
                    e += lB * q[i] * q[j] * (erfc(a * r) / r - c1 + c2 * (r - rc))
        E[s] = e
    return E


def enumeration_probs(w, n, chem):
    p = w.params
    ln10 = math.log(10.0)
    L = float(np.float32(p["box_L"]))
    lnV = math.log(0.602214076 * (L * p["sigma_nm"]) ** 3)
    ln_zp = lnV - ln10 * chem["pIX_plus"]
    ln_zm = lnV - ln10 * chem["pIX_minus"]
    pOH = p["pKw"] - p["pH"]
    E = dsf_energy_states(w, n)
    logw = np.zeros(1 << n)
    for s in range(1 << n):
        kA = kB = 0
        lw = 0.0
        for i in range(n):
            if (s >> i) & 1:
                if w.type[i] == W.ACID:
                    lw += ln10 * (p["pH"] - w.pK[i]); kA += 1
                else:
                    lw += ln10 * (pOH - w.pK[i]); kB += 1
        D = kA - kB
        lw += 0.5 * D * (ln_zp - ln_zm) + math.log(ive(abs(D), 2 * math.exp(0.5 * (ln_zp + ln_zm))))
        logw[s] = lw - E[s]
    P = np.exp(logw - logw.max())
    return P / P.sum()


@pytest.mark.parametrize("schedule,n_base", [(1, 0), (0, 0), (1, 2)])
def test_exact_enumeration_interacting_sites(schedule, n_base):
    n = 6
    w = W.enum_sites(n_sites=n, L=24.0, rc=8.0, lB=2.0, pH=5.0, pKa=5.0, pIS=2.0, n_pairs=4, seed=3,
                     n_base=n_base, schedule=schedule, trials_per_domain=64 if schedule == 1 else 2)
    if n_base:
        w.params["pH"] = 7.0
        w.pK[:] = np.where(w.type == W.BASE, 7.0, 7.0)
        w.params["pIS_minus"] = 2.5
    o = oracle.Oracle(w)
    P = enumeration_probs(w, n, o.chem())
    tps = o.trials_per_sweep
    o.sweep(tps * max(1, 20000 // tps), 1)
    B, per = 24, 16384
    H = []
    for b in range(B):
        h = o.sweep(tps * max(1, per // tps), 1000 + b, hist_n=n)["hist"]
        H.append(h / h.sum())
    H = np.array(H)
    mean = H.mean(0)
    se = H.std(0, ddof=1) / math.sqrt(B)
    big = P > 0.01
    z = np.abs(mean - P)[big] / np.maximum(se[big], 1e-4)
    assert z.max() < 5.0, (z.max(), mean[big], P[big])
    # total variation distance against its own sampling noise (batch means)
    tv = 0.5 * np.abs(mean - P).sum()
    tv_noise = 0.5 * float(np.sum(se)) * math.sqrt(2.0 / math.pi)
    assert tv < 3.0 * tv_noise + 0.005, (tv, tv_noise)


# ---------------------------------------------------------------- Delta E = E_new - E_old
def test_delta_E_equals_total_energy_difference():
    w = W.config1(seed=1, n_pairs=16)
    o = oracle.Oracle(w, schedule=1, trials_per_domain=1)
    n_acc = 0
    for t in range(400):
        e0 = o.energy()
        rec = o.sweep(1, 77 + t, log=True)["log"][0]
        e1 = o.energy()
        if rec["flags"] & oracle.F_ACC:
            n_acc += 1
            assert abs((e1 - e0) - rec["dE"]) < 1e-9 * max(1.0, rec["S"]), (t, rec, e1 - e0)
        else:
            assert e1 == e0
    assert n_acc > 20


def test_neutrality_ids_and_counts_invariants():
    w = W.config1(seed=2)
    o = oracle.Oracle(w)
    seen = set()
    for s in range(30):
        o.sweep(o.trials_per_sweep, 500 + s)  # raises if any trial leaves the system charged
        c = o.counts()
        assert c["net_charge"] == 0
        assert c["n_Xp"] - c["n_Xm"] == c["n_Am"] - c["n_Bp"]
        part = o.particles()
        assert len(np.unique(part["id"])) == len(part["id"])
        assert np.all((part["xyz"] >= 0) & (part["xyz"] < np.float32(w.params["box_L"])))
        seen.update(part["id"][part["id"] >= (1 << 32)].tolist())
    assert len(seen) > 0  # ions were inserted with phase-tagged ids


# ---------------------------------------------------------------- detailed balance
def test_site_transition_flux_symmetry():
    """For a reversible chain the flux s -> s' equals s' -> s for lumped states."""
    n = 5
    w = W.enum_sites(n_sites=n, L=24.0, rc=8.0, lB=2.0, n_pairs=6, seed=8, schedule=0, trials_per_domain=4)
    w.params["ion_coupling"] = 1  # interacting explicit ions
    o = oracle.Oracle(w)
    tps = o.trials_per_sweep
    o.sweep(tps * 200, 5)
    T = np.zeros(((1 << n), n), dtype=np.int64)
    for b in range(20):
        T += o.sweep(tps * 400, 900 + b, hist_n=n, trans=True)["trans"]
    chi, dof = 0.0, 0
    for s in range(1 << n):
        for i in range(n):
            if (s >> i) & 1:
                continue
            f_up, f_dn = T[s, i], T[s | (1 << i), i]
            if f_up + f_dn < 30:
                continue
            assert abs(f_up - f_dn) <= 5.0 * math.sqrt(f_up + f_dn) + 2, (s, i, f_up, f_dn)
            chi += (f_up - f_dn) ** 2 / (f_up + f_dn)
            dof += 1
    assert dof >= 10
    assert chi / dof < 3.0


def test_schedules_agree_on_interacting_system():
    """Domain-local coloured moves sample the same distribution as the paper's global moves."""
    res = []
    for sched, m in ((1, 64), (0, 2)):
        w = W.config1(seed=3, n_pairs=24, schedule=sched, trials_per_domain=m)
        w.params["lB"] = 2.0
        o = oracle.Oracle(w)
        res.append(run_alpha(o, 50, 30, 4096, seed=40 + sched, burn=40000))
    (m1, s1), (m2, s2) = res
    assert abs(m1 - m2) <= 4.0 * math.hypot(s1, s2) + 0.005, res


# ---------------------------------------------------------------- sensitivity: planted mistakes
@pytest.mark.parametrize("kind", ["drop_ion_count", "wrong_volume"])
def test_planted_mistake_fails_closed_form(kind):
    oracle.plant(kind)
    n, L = 50, 40.0
    w = W.ideal(n_sites=n, L=L, pH=5.0, pKa=5.0, n_pairs=20, seed=11, schedule=1, trials_per_domain=256)
    o = oracle.Oracle(w)
    ch = o.chem()
    ln10 = math.log(10.0)
    lnV = math.log(0.602214076 * (L * 0.355) ** 3)
    a_ex = exact_alpha(n, 0.0, lnV - ln10 * ch["pIX_plus"], lnV - ln10 * ch["pIX_minus"])
    try:
        mean, se = run_alpha(o, n, 20, 4096, seed=105)
    except RuntimeError:
        return  # the chain ran away (ion count without bound): caught
    assert abs(mean - a_ex) > 0.02


@pytest.mark.parametrize("kind", ["drop_self", "drop_pair_cc", "dE_sign"])
def test_planted_mistake_fails_energy_pin(kind):
    oracle.plant(kind)
    w = W.config1(seed=1, n_pairs=16)
    o = oracle.Oracle(w, schedule=1, trials_per_domain=1)
    bad = 0
    for t in range(300):
        e0 = o.energy()
        rec = o.sweep(1, 77 + t, log=True)["log"][0]
        e1 = o.energy()
        if rec["flags"] & oracle.F_ACC and abs((e1 - e0) - rec["dE"]) > 1e-6:
            bad += 1
    assert bad > 0


# ---------------------------------------------------------------- grand-reaction invocations
# Types of the four monovalent species when they are kept apart (App. B: the
# scheme invoked repeatedly with different types of ions; Sec. II.B: applied
# separately to dissociated and salt ions = the grand-reaction ensemble).
H_, OH_, SP_, SM_ = W.XP, W.XM, W.SP, W.SM


def grand_reaction_cycle(o, pH, pOH, pIS_p, pIS_m, T, seed):
    """One cycle of the grand-reaction ensemble as four invocations: the acid
    and salt reactions with (H+, OH-) and with (S+, S-), the mixed salt
    reactions (H+, S-) and (S+, OH-); every reaction attempted T/2 times."""
    tps = o.trials_per_sweep
    for k, (c, a, pc, pa, r, n) in enumerate(((H_, OH_, pH, pOH, 5, T), (SP_, SM_, pIS_p, pIS_m, 5, T),
                                              (H_, SM_, pH, pIS_m, 4, T // 2), (SP_, OH_, pIS_p, pOH, 4, T // 2))):
        o.set_invocation(c, a, pc, pa, r)
        o.sweep(max(tps, (n // tps) * tps), seed * 8 + k)


def _grand_reaction_run(w, pH, pIS, n_sites, cycles, per_batch, seed):
    o = oracle.Oracle(w)
    pOH = 14.0 - pH
    for c in range(20):
        grand_reaction_cycle(o, pH, pOH, pIS, pIS, 256, seed + c)
    al, fH, fOH = [], [], []
    for b in range(cycles):
        a = h = np_ = oh = nm = 0.0
        for r in range(per_batch):
            grand_reaction_cycle(o, pH, pOH, pIS, pIS, 256, seed + 1000 + b * per_batch + r)
            k = o.counts()
            assert k["net_charge"] == 0
            a += k["n_Am"] / n_sites
            h += k["n_Xp"]
            np_ += k["n_Xp"] + k["n_Sp"]
            oh += k["n_Xm"]
            nm += k["n_Xm"] + k["n_Sm"]
        al.append(a / per_batch)
        fH.append(h / max(np_, 1.0))
        fOH.append(oh / max(nm, 1.0))
    return [(float(np.mean(v)), float(np.std(v, ddof=1) / math.sqrt(len(v)))) for v in (al, fH, fOH)]


def test_grand_reaction_samples_the_grouped_distribution():
    """Ideal acids under the four grand-reaction invocations: the degree of
    dissociation is the grouped closed form (the H+/S+ ideal terms summed,
    Eqs. (mux1)-(mux2)), and the fraction of H+ among the cations is
    10^-pH / (10^-pH + 10^-pI_S+) (the ungrouping probability of Sec. III.A;
    multinomial at fixed totals in the ideal limit)."""
    n, L, pH, pIS, pKa, sig = 50, 40.0, 2.3, 2.0, 2.5, 0.355
    w = W.ideal(n_sites=n, L=L, pH=pH, pKa=pKa, pIS=pIS, n_pairs=20, seed=11, schedule=1, trials_per_domain=256)
    ln10 = math.log(10.0)
    lnV = math.log(0.602214076 * (L * sig) ** 3)
    pOH = 14.0 - pH
    pIXp = -math.log10(10 ** -pH + 10 ** -pIS)
    pIXm = -math.log10(10 ** -pOH + 10 ** -pIS)
    a_ex = exact_alpha(n, ln10 * (pH - pKa), lnV - ln10 * pIXp, lnV - ln10 * pIXm)
    pH_frac = 10 ** -pH / (10 ** -pH + 10 ** -pIS)
    (a, sa), (fh, sh), (foh, soh) = _grand_reaction_run(w, pH, pIS, n, 30, 8, seed=3)
    assert abs(a - a_ex) <= max(4.0 * sa, 0.004), (a, sa, a_ex)
    assert abs(fh - pH_frac) <= max(4.0 * sh, 0.01), (fh, sh, pH_frac)
    assert foh < 1e-3  # OH- at pOH 11.7 is absent from the box


def test_rxmc_invocation_matches_its_closed_form():
    """The RxMC special case (pI_X+ = pH, pI_X- = pOH; App. B) samples Eq.
    (QQ) with the dissociated ions alone: the closed form with z+ = V 10^-pH
    and z- = V 10^-pOH."""
    n, L, pH, pKa, sig = 50, 40.0, 3.5, 3.0, 0.355
    w = W.ideal(n_sites=n, L=L, pH=pH, pKa=pKa, pIS=2.0, n_pairs=20, seed=12, schedule=1, trials_per_domain=256)
    o = oracle.Oracle(w)
    o.set_invocation(H_, OH_, pH, 14.0 - pH, 7)
    ln10 = math.log(10.0)
    lnV = math.log(0.602214076 * (L * sig) ** 3)
    a_ex = exact_alpha(n, ln10 * (pH - pKa), lnV - ln10 * pH, lnV - ln10 * (14.0 - pH))
    mean, se = run_alpha(o, n, 40, 4096, seed=21, burn=40000)
    assert abs(mean - a_ex) <= max(4.0 * se, 0.003), (mean, se, a_ex)


def test_invocation_arguments_are_checked():
    w = W.ideal(n_sites=5, seed=2, schedule=1, trials_per_domain=16)
    o = oracle.Oracle(w)
    for args in ((W.ACID, OH_, 2.0, 2.0, 7), (H_, SP_, 2.0, 2.0, 7), (H_, OH_, float("nan"), 2.0, 7),
                 (H_, OH_, 2.0, 2.0, 0), (H_, OH_, 2.0, 2.0, 2)):  # 2: bases only, and there are none
        with pytest.raises(ValueError):
            o.set_invocation(*args)


def test_planted_species_count_fails_the_grand_reaction_pin():
    """Counting every like-charged ion (instead of the invocation's species)
    in the acceptance rules shifts the H+ fraction off its closed form."""
    oracle.plant("species_count")
    n, L, pH, pIS, pKa = 50, 40.0, 2.3, 2.0, 2.5
    w = W.ideal(n_sites=n, L=L, pH=pH, pKa=pKa, pIS=pIS, n_pairs=20, seed=11, schedule=1, trials_per_domain=256)
    (a, sa), (fh, sh), _ = _grand_reaction_run(w, pH, pIS, n, 10, 8, seed=5)
    pH_frac = 10 ** -pH / (10 ** -pH + 10 ** -pIS)
    assert abs(fh - pH_frac) > 0.05, (fh, pH_frac)
