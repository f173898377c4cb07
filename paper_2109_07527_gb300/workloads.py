"""Seeded synthetic inputs for the CR-MC path (shared by the CUDA path's tests,
the oracle's tests and the benchmark).

This module only places particles and fills parameter records; it holds none
of the method's arithmetic.  The workloads follow the systems of the paper's
numerical sections with synthetic coordinates (the paper's own systems are
synthetic too, Sec. II.D and App. C: random non-overlapping placement with
r_ij > 2^(1/6) sigma and no salt overlap):

* ``ideal``      -- non-interacting acids + ghost ions (closed-form titration)
* ``enum_sites`` -- <= 10 fixed interacting sites + ghost ions (exact enumeration)
* ``config1``    -- one FENE chain of 50 acid beads, L = 40, r_c = 10, 64 ion pairs
* ``config2``    -- 16 chains x 200 acid beads, L = 120, r_c = 12, ~4000 ion pairs
                    (``scale`` shrinks the box at fixed densities for parity runs)
* ``config3``    -- two nanoparticles with 1000 Fibonacci-lattice sites each
* ``config4``    -- 64 replicas, chain lengths log-uniform in [50, 1000]
* ``config5``    -- 100 chains x 200 beads, L = 250, ~25 000 ion pairs

Particle type codes (input encoding): 0 bead, 1 acid, 2 base, 3 X+, 4 X-, 5 core,
6 S+, 7 S- (salt ions kept apart from X+- by grand-reaction invocations).
Short-range classes: 0..2 use the WCA table; 3 has no short-range interaction.
"""
from __future__ import annotations

import dataclasses
import math
import numpy as np

BEAD, ACID, BASE, XP, XM, CORE, SP, SM = 0, 1, 2, 3, 4, 5, 6, 7
CLS_NONE = 3
WCA_CUT = 2.0 ** (1.0 / 6.0)


@dataclasses.dataclass
class Workload:
    name: str
    xyz: np.ndarray          # (n, 3) float32, in [0, L)
    type: np.ndarray         # (n,) int32
    cls: np.ndarray          # (n,) int32
    state: np.ndarray        # (n,) int8, 1 = ionised site
    pK: np.ndarray           # (n,) float64, pKa / pKb of sites (ignored elsewhere)
    bonds: np.ndarray        # (nb, 2) int32, FENE bonds by particle index
    vel: np.ndarray | None   # (n, 3) float32
    params: dict
    capacity: int
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_sites(self) -> int:
        return int(np.sum((self.type == ACID) | (self.type == BASE)))


def default_params(**kw) -> dict:
    eps = [1.0] * 16
    sig = [1.0] * 16
    dele = [0.0] * 16
    on = [1 if (i < 3 and j < 3) else 0 for i in range(4) for j in range(4)]
    p = dict(box_L=40.0, sigma_nm=0.355, lB=2.0, rc=10.0, alpha=0.2, dsf_self=1, ion_coupling=1, ion_cls=0,
             pH=5.0, pKw=14.0, pIS_plus=2.0, pIS_minus=2.0, pIX_explicit=0, pIX_plus=0.0, pIX_minus=0.0,
             nc=0, cells_per_rc=2, domain_cells=2, trials_per_domain=10, schedule=0,
             wca_eps=eps, wca_sig=sig, wca_del=dele, wca_on=on, fene_K=30.0, fene_R0=1.5, ewald_kmax=0)
    p.update(kw)
    return p


class _Grid:
    """Spatial hash for overlap-free placement (minimum image)."""

    def __init__(self, L: float, h: float):
        self.L = L
        self.n = max(1, int(L // h))
        self.h = L / self.n
        self.cells: dict = {}

    def _key(self, p):
        return tuple(int(c // self.h) % self.n for c in p)

    def add(self, p, tag):
        self.cells.setdefault(self._key(p), []).append((p[0], p[1], p[2], tag))

    def too_close(self, p, dmin, ignore=()):
        k = self._key(p)
        L = self.L
        d2 = dmin * dmin
        rng = range(-1, 2) if self.n >= 3 else range(self.n)
        for dx in rng:
            for dy in rng:
                for dz in rng:
                    if self.n >= 3:
                        key = ((k[0] + dx) % self.n, (k[1] + dy) % self.n, (k[2] + dz) % self.n)
                    else:
                        key = (dx, dy, dz)
                    for (x, y, z, tag) in self.cells.get(key, ()):
                        if tag in ignore:
                            continue
                        ex = x - p[0]; ex -= L * round(ex / L)
                        ey = y - p[1]; ey -= L * round(ey / L)
                        ez = z - p[2]; ez -= L * round(ez / L)
                        if ex * ex + ey * ey + ez * ez < d2:
                            return True
        return False


def _wrap(p, L):
    q = np.mod(np.asarray(p, dtype=np.float64), L)
    q = q.astype(np.float32)
    q[q >= np.float32(L)] = 0.0
    return q


def _place(rng, grid, L, dmin, tag, tries=10000):
    for _ in range(tries):
        p = _wrap(rng.random(3) * L, L)
        if not grid.too_close(p, dmin):
            grid.add(p, tag)
            return p
    raise RuntimeError("could not place a particle without overlap")


def _chain(rng, grid, L, N, tag0, bond=0.97, dmin=1.0):
    """Self-avoiding random walk: consecutive beads 0.97 sigma apart, every
    non-bonded pair (within the chain and with everything placed before) at
    least dmin apart."""
    for _attempt in range(200):
        pts = []
        start = _place_probe(rng, grid, L, WCA_CUT)
        if start is None:
            continue
        own = _Grid(L, 1.2)
        pts.append(start)
        own.add(start, 0)
        ok = True
        for i in range(1, N):
            placed = False
            for _ in range(200):
                v = rng.normal(size=3)
                v /= np.linalg.norm(v)
                p = _wrap(pts[-1].astype(np.float64) + bond * v, L)
                if grid.too_close(p, dmin) or own.too_close(p, dmin, ignore=(i - 1,)):
                    continue
                pts.append(p)
                own.add(p, i)
                placed = True
                break
            if not placed:
                ok = False
                break
        if ok:
            for i, p in enumerate(pts):
                grid.add(p, tag0 + i)
            return np.array(pts, dtype=np.float32)
    raise RuntimeError("could not grow a self-avoiding chain")


def _place_probe(rng, grid, L, dmin):
    for _ in range(10000):
        p = _wrap(rng.random(3) * L, L)
        if not grid.too_close(p, dmin):
            return p
    return None


def _assemble(name, parts, params, extra_capacity, rng, meta=None, bonds=None, with_vel=True):
    xyz = np.concatenate([p[0] for p in parts]).astype(np.float32)
    typ = np.concatenate([p[1] for p in parts]).astype(np.int32)
    cls = np.concatenate([p[2] for p in parts]).astype(np.int32)
    st = np.concatenate([p[3] for p in parts]).astype(np.int8)
    pK = np.concatenate([p[4] for p in parts]).astype(np.float64)
    n = xyz.shape[0]
    b = np.zeros((0, 2), np.int32) if bonds is None else np.asarray(bonds, np.int32).reshape(-1, 2)
    vel = rng.normal(size=(n, 3)).astype(np.float32) if with_vel else None
    return Workload(name=name, xyz=xyz, type=typ, cls=cls, state=st, pK=pK, bonds=b, vel=vel,
                    params=params, capacity=int(n + extra_capacity), meta=meta or {})


def _ions(rng, grid, L, n_pairs, tag0, dmin=WCA_CUT):
    xyz = np.zeros((2 * n_pairs, 3), np.float32)
    t = np.zeros(2 * n_pairs, np.int32)
    for i in range(n_pairs):
        xyz[2 * i] = _place(rng, grid, L, dmin, tag0 + 2 * i)
        t[2 * i] = XP
        xyz[2 * i + 1] = _place(rng, grid, L, dmin, tag0 + 2 * i + 1)
        t[2 * i + 1] = XM
    return (xyz, t, np.zeros(2 * n_pairs, np.int32), np.zeros(2 * n_pairs, np.int8), np.zeros(2 * n_pairs))


def ideal(n_sites=50, L=40.0, pH=5.0, pKa=5.0, pIS=2.0, n_pairs=20, seed=1, rc=10.0, schedule=0,
          trials_per_domain=10, sigma_nm=0.355, ghost=True, base=False):
    """Non-interacting weak acids (or bases) with ghost ions: l_B = 0 and the
    ions carry no charge and no short-range interaction, so the charge-state
    distribution has the closed form of Eq. (QQ) with E = 0."""
    rng = np.random.default_rng(seed)
    grid = _Grid(L, 1.2)
    sx = np.array([_place(rng, grid, L, WCA_CUT, i) for i in range(n_sites)], np.float32).reshape(-1, 3)
    st = (rng.random(n_sites) < 0.0).astype(np.int8)
    sites = (sx, np.full(n_sites, BASE if base else ACID, np.int32), np.zeros(n_sites, np.int32), st,
             np.full(n_sites, pKa))
    ions = _ions(rng, grid, L, n_pairs, n_sites)
    params = default_params(box_L=L, rc=rc, lB=0.0, ion_coupling=0 if ghost else 1, pH=pH, pIS_plus=pIS,
                            pIS_minus=pIS, schedule=schedule, trials_per_domain=trials_per_domain,
                            sigma_nm=sigma_nm)
    return _assemble("ideal", [sites, ions], params, 4 * n_sites + 4096, rng, with_vel=False)


def weak_acid_electrolyte(n_acid=500, L=100.0, pH=7.0, pKa=6.5, pIS=2.0, rc=20.0, seed=1, trials_per_domain=500,
                          sigma_nm=0.355, alpha=0.15):
    """The weak-acid electrolyte of the method comparison (Sec. III.A, Fig. 2):
    n_acid individual acid groups (pKa 6.5) placed at random with every pair
    farther apart than 2^(1/6) sigma, no free ions at the start, in a cubic
    box of L = 50 l_B (l_B = 2 sigma = 0.71 nm), pH 7 and pI_S+- = 2 (about
    0.01 M salt); electrostatics by DSF with r_c = 10 l_B (the paper's real-
    space cutoff; its PPPM long-range part is replaced by the damped shifted
    force), one domain (the global schedule: every trial sees the whole box)."""
    rng = np.random.default_rng(seed)
    grid = _Grid(L, 1.2)
    sx = np.array([_place(rng, grid, L, WCA_CUT, i) for i in range(n_acid)], np.float32).reshape(-1, 3)
    sites = (sx, np.full(n_acid, ACID, np.int32), np.zeros(n_acid, np.int32), np.zeros(n_acid, np.int8),
             np.full(n_acid, pKa))
    params = default_params(box_L=L, rc=rc, lB=2.0, alpha=alpha, ion_coupling=1, pH=pH, pIS_plus=pIS,
                            pIS_minus=pIS, schedule=1, trials_per_domain=trials_per_domain, sigma_nm=sigma_nm)
    return _assemble("weak_acid_electrolyte", [sites], params, 4096, rng, with_vel=False)


def enum_sites(n_sites=8, L=24.0, rc=8.0, lB=2.0, pH=5.0, pKa=5.0, pIS=2.0, n_pairs=4, seed=3, n_base=0,
               schedule=1, trials_per_domain=64, spread=3.0, sigma_nm=0.355):
    """n <= 10 fixed, mutually interacting sites (DSF among sites) with ghost
    ions, for exact enumeration of the 2^n charge states."""
    rng = np.random.default_rng(seed)
    grid = _Grid(L, 1.2)
    c = np.array([L / 2, L / 2, L / 2])
    pts = []
    for i in range(n_sites):
        for _ in range(10000):
            p = _wrap(c + (rng.random(3) - 0.5) * 2 * spread, L)
            if not grid.too_close(p, 1.5):
                grid.add(p, i)
                pts.append(p)
                break
    sx = np.array(pts, np.float32)
    types = np.array([BASE if i < n_base else ACID for i in range(n_sites)], np.int32)
    sites = (sx, types, np.zeros(n_sites, np.int32), np.zeros(n_sites, np.int8), np.full(n_sites, pKa))
    ions = _ions(rng, grid, L, n_pairs, n_sites)
    params = default_params(box_L=L, rc=rc, lB=lB, ion_coupling=0, pH=pH, pIS_plus=pIS, pIS_minus=pIS,
                            schedule=schedule, trials_per_domain=trials_per_domain, sigma_nm=sigma_nm)
    return _assemble("enum_sites", [sites, ions], params, 4 * n_sites + 4096, rng, with_vel=False)


def _chains(rng, grid, L, n_chains, N, pKa, tag0=0):
    xyz, bonds = [], []
    for c in range(n_chains):
        pts = _chain(rng, grid, L, N, tag0 + c * N)
        xyz.append(pts)
        base = tag0 + c * N
        bonds += [(base + i, base + i + 1) for i in range(N - 1)]
    xyz = np.concatenate(xyz) if xyz else np.zeros((0, 3), np.float32)
    n = n_chains * N
    return (xyz, np.full(n, ACID, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int8), np.full(n, pKa)), bonds


def config1(seed=1, lB=2.0, ghost=False, n_pairs=64, schedule=0, trials_per_domain=10):
    """Single weak polyacid: N = 50 FENE chain, every bead an acid (pKa 5),
    pH 5, l_B = 2 sigma, L = 40 sigma, DSF alpha = 0.2, r_c = 10 sigma,
    10 mM reservoir salt (pI_S = 2) and 64 initial ion pairs."""
    rng = np.random.default_rng(seed)
    L = 40.0
    grid = _Grid(L, 1.2)
    chain, bonds = _chains(rng, grid, L, 1, 50, 5.0)
    ions = _ions(rng, grid, L, n_pairs, 50)
    params = default_params(box_L=L, rc=10.0, lB=lB, ion_coupling=0 if ghost else 1, pH=5.0, pIS_plus=2.0,
                            pIS_minus=2.0, schedule=schedule, trials_per_domain=trials_per_domain)
    return _assemble("config1", [chain, ions], params, 4096, rng, bonds=bonds,
                     meta=dict(precision="fp64", trials=10_000))


def config2(seed=1, pH=4.5, scale=1.0, trials_per_domain=10, n_chains=None, N=200):
    """Polyelectrolyte solution: 16 chains x 200 acid beads (pKa 4.5),
    L = 120 sigma, r_c = 12 sigma, l_B = 2 sigma, salt pI_S = 1.066 (ideal
    reservoir count ~4000 pairs), explicit counter- and salt ions.
    ``scale`` < 1 shrinks the box at fixed monomer and salt density."""
    rng = np.random.default_rng(seed)
    L = 120.0 * scale
    if n_chains is None:
        n_chains = max(1, int(round(16 * scale ** 3)))
    n_pairs = int(round(4000 * scale ** 3))
    grid = _Grid(L, 1.2)
    chains, bonds = _chains(rng, grid, L, n_chains, N, 4.5)
    ions = _ions(rng, grid, L, n_pairs, n_chains * N)
    params = default_params(box_L=L, rc=12.0, lB=2.0, pH=pH, pIS_plus=1.066, pIS_minus=1.066,
                            trials_per_domain=trials_per_domain)
    n = n_chains * N + 2 * n_pairs
    return _assemble("config2", [chains, ions], params, n + 4096, rng, bonds=bonds,
                     meta=dict(trials=1_000_000, md_steps=100, dt=0.005, gamma=1.0, L=L))


def fibonacci_sphere(n, radius):
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = np.pi * (3.0 - np.sqrt(5.0)) * np.arange(n)
    r = np.sqrt(1.0 - z * z)
    return radius * np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def config3(separation=12.0, seed=1, L=100.0, n_sites=1000, R=5.0, pIS=None):
    """Two nanoparticles of radius 5 sigma, each with 1000 surface sites on a
    Fibonacci lattice at radius R - 0.5 sigma (NP1 acids pKa 4, NP2 bases
    pKb 4), pH 7, 20 mM salt, l_B = 0.7 sigma, r_c = 12 sigma.  Cores interact
    with ions by expanded WCA with Delta = R - r (Eq. LJe, Table II).  Fixed
    unless declared rigid bodies: ``meta["bodies"]`` gives each
    nanoparticle's first id and member count (core and sites)."""
    rng = np.random.default_rng(seed)
    grid = _Grid(L, 1.2)
    c1 = np.array([L / 2 - separation / 2, L / 2, L / 2])
    c2 = np.array([L / 2 + separation / 2, L / 2, L / 2])
    parts = []
    for ci, (cen, t) in enumerate([(c1, ACID), (c2, BASE)]):
        core = _wrap(cen, L)
        parts.append((core[None, :], np.array([CORE], np.int32), np.array([1], np.int32), np.zeros(1, np.int8),
                      np.zeros(1)))
        s = np.array([_wrap(cen + p, L) for p in fibonacci_sphere(n_sites, R - 0.5)], np.float32)
        parts.append((s, np.full(n_sites, t, np.int32), np.full(n_sites, CLS_NONE, np.int32),
                      np.zeros(n_sites, np.int8), np.full(n_sites, 4.0)))
    # exclusion zones for ion placement: the cores
    if pIS is None:
        pIS = -math.log10(0.02)
    sigma_nm = 0.355
    v_nm3 = (L * sigma_nm) ** 3
    n_pairs = int(round(0.602214076 * v_nm3 * 10 ** (-pIS)))
    for cen in (c1, c2):
        grid.add(_wrap(cen, L), -1)
    xyz = np.zeros((2 * n_pairs, 3), np.float32)
    t = np.zeros(2 * n_pairs, np.int32)
    for i in range(2 * n_pairs):
        for _ in range(10000):
            p = _wrap(rng.random(3) * L, L)
            e1 = p - c1; e1 -= L * np.round(e1 / L)
            e2 = p - c2; e2 -= L * np.round(e2 / L)
            if min(np.linalg.norm(e1), np.linalg.norm(e2)) < R + 0.7:
                continue
            if grid.too_close(p, WCA_CUT):
                continue
            grid.add(p, i)
            xyz[i] = p
            t[i] = XP if i % 2 == 0 else XM
            break
    ions = (xyz, t, np.zeros(2 * n_pairs, np.int32), np.zeros(2 * n_pairs, np.int8), np.zeros(2 * n_pairs))
    parts.append(ions)
    r_ion = 0.5
    dele = [0.0] * 16
    dele[0 * 4 + 1] = dele[1 * 4 + 0] = R - r_ion
    dele[1 * 4 + 1] = 2 * R - 2 * r_ion
    params = default_params(box_L=L, rc=12.0, lB=0.7, pH=7.0, pIS_plus=pIS, pIS_minus=pIS, wca_del=dele)
    # each nanoparticle (its core and its sites, ids in that order) as one
    # rigid body: first ids and member counts
    bodies = ([0, 1 + n_sites], [1 + n_sites, 1 + n_sites])
    return _assemble("config3", parts, params, 2 * n_sites * 2 + 8192, rng,
                     meta=dict(separation=separation, bodies=bodies), with_vel=False)


def config4(seed=1, n_rep=64, density=1e-3, lo=50, hi=1000):
    """Batched titration: 64 replicas, chain length log-uniform in [50, 1000],
    pH uniform in [2, 10], pKa 5, box sized to 1e-3 monomers per sigma^3,
    10 mM salt, per-replica seeds."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_rep):
        N = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        pH = float(rng.uniform(2.0, 10.0))
        L = (N / density) ** (1.0 / 3.0)
        sub = np.random.default_rng(seed * 1000 + r)
        grid = _Grid(L, 1.2)
        chains, bonds = _chains(sub, grid, L, 1, N, 5.0)
        v_nm3 = (L * 0.355) ** 3
        n_pairs = max(1, int(round(0.602214076 * v_nm3 * 0.01)))
        ions = _ions(sub, grid, L, n_pairs, N)
        params = default_params(box_L=L, rc=12.0, lB=2.0, pH=pH, pIS_plus=2.0, pIS_minus=2.0)
        out.append(_assemble(f"config4[{r}]", [chains, ions], params, N + 2 * n_pairs + 4 * N + 1024, sub,
                             bonds=bonds, meta=dict(N=N, pH=pH, L=L, seed=seed * 1000 + r)))
    return out


def config5(seed=1, scale=1.0):
    """Large system for the learned delayed-acceptance stage: 100 chains x 200
    acid beads (pKa 4.5, pH 4.5), L = 250 sigma, ~25 000 ion pairs
    (pI_S = 1.226), r_c = 12 sigma, l_B = 2 sigma."""
    rng = np.random.default_rng(seed)
    L = 250.0 * scale
    n_chains = max(1, int(round(100 * scale ** 3)))
    n_pairs = int(round(25000 * scale ** 3))
    grid = _Grid(L, 1.2)
    chains, bonds = _chains(rng, grid, L, n_chains, 200, 4.5)
    ions = _ions(rng, grid, L, n_pairs, n_chains * 200)
    params = default_params(box_L=L, rc=12.0, lB=2.0, pH=4.5, pIS_plus=1.226, pIS_minus=1.226)
    n = n_chains * 200 + 2 * n_pairs
    return _assemble("config5", [chains, ions], params, n + 8192, rng, bonds=bonds)


# ---------------------------------------------------------------- surrogate weights
def to_bf16_bits(x):
    """BF16 bit patterns of float32 values (round to nearest, ties to even)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def bf16_to_f32(bits):
    """float32 values of BF16 bit patterns (exact)."""
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def random_mlp(seed=1, gain=1.0, out_gain=1.0, n_in=48, n_hid=128):
    """Seeded random surrogate weights in the layout the ABI takes: W1 [128, 48],
    W2 and W3 [128, 128], w4 [128] as BF16 bit patterns, biases float32.
    He-style scales times `gain`; `out_gain` scales the output layer."""
    rng = np.random.default_rng(seed)
    def layer(o, i, g):
        return to_bf16_bits(rng.normal(0.0, g * math.sqrt(2.0 / i), (o, i)).astype(np.float32))
    return dict(W1=layer(n_hid, n_in, gain * 0.25), b1=(0.05 * rng.normal(size=n_hid)).astype(np.float32),
                W2=layer(n_hid, n_hid, gain), b2=(0.05 * rng.normal(size=n_hid)).astype(np.float32),
                W3=layer(n_hid, n_hid, gain), b3=(0.05 * rng.normal(size=n_hid)).astype(np.float32),
                w4=to_bf16_bits((out_gain * rng.normal(0.0, math.sqrt(1.0 / n_hid), n_hid)).astype(np.float32)),
                b4=float(0.1 * rng.normal()))
