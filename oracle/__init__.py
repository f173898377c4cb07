"""Plain FP64 CPU oracle for the CR-MC stage (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``crmc_oracle.c`` (plain C,
compiled with gcc here or on the GPU host by :func:`build`) and
``mlp_oracle.py`` (numpy float64, the surrogate's training step).  Nothing in it is shared with the CUDA path.

Paper sections it follows: Sec. II.B (grouped reactions), Sec. II.C (moves and
acceptance rules, Eq. QQ), App. A (ion grouping, Eq. mux), App. C (Eq. pIXgen).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "crmc_oracle.c")
_LIB = os.path.join(_HERE, "libcrmc_oracle.so")

# trial-record flags
F_ACC, F_NOELIG, F_EDGE, F_OVERLAP = 1, 2, 4, 8
PLANT = {"none": 0, "drop_ion_count": 1, "dE_sign": 2, "drop_self": 3, "drop_pair_cc": 4,
         "wrong_volume": 5, "da_one_sided": 6, "da_stage2_full": 7, "species_count": 8,
         "ewald_half_recip": 9, "rigid_torque_sign": 10, "rigid_no_rot_noise": 11,
         "ewald_force_sign": 12}
N_FEAT, N_HID = 48, 128


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("n", C.c_int32), ("capacity", C.c_int32),
                ("box_L", C.c_double), ("sigma_nm", C.c_double),
                ("lB", C.c_double), ("rc", C.c_double), ("alpha", C.c_double),
                ("dsf_self", C.c_int32), ("ion_coupling", C.c_int32), ("ion_cls", C.c_int32),
                ("pH", C.c_double), ("pKw", C.c_double), ("pIS_plus", C.c_double), ("pIS_minus", C.c_double),
                ("pIX_explicit", C.c_int32),
                ("pIX_plus", C.c_double), ("pIX_minus", C.c_double),
                ("nc", C.c_int32), ("domain_cells", C.c_int32), ("trials_per_domain", C.c_int32),
                ("schedule", C.c_int32), ("cells_per_rc", C.c_int32),
                ("wca_eps", C.c_double * 16), ("wca_sig", C.c_double * 16), ("wca_del", C.c_double * 16),
                ("wca_on", C.c_int32 * 16),
                ("fene_K", C.c_double), ("fene_R0", C.c_double),
                ("n_bonds", C.c_int32), ("ewald_kmax", C.c_int32)]


TRIAL_DTYPE = np.dtype([("move", "<i4"), ("flags", "<i4"), ("id_a", "<u8"), ("id_b", "<u8"),
                        ("dE", "<f8"), ("S", "<f8"), ("lnA", "<f8"), ("lnu", "<f8")])
# delayed-acceptance record: surrogate dE~, stage (0 none, 1 stage-1 reject,
# 2 passed stage 1), stage-2 log ratio dE~ - dE_pair, log of the stage-2 uniform
DA_DTYPE = np.dtype([("dE_sur", "<f4"), ("stage", "<i4"), ("lnA2", "<f8"), ("lnu2", "<f8")])

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.or_create.restype = P
        lib.or_create.argtypes = [C.POINTER(_Params), P, P, P, P, P, P, P, C.POINTER(C.c_int32)]
        lib.or_destroy.argtypes = [P]
        lib.or_sweep.restype = C.c_int32
        lib.or_sweep.argtypes = [P, C.c_int64, C.c_uint64, P, P, P, C.c_int32, P, P, P, P]
        lib.or_set_surrogate.restype = C.c_int32
        lib.or_set_surrogate.argtypes = [P, P, P, P, P, P, P, P, C.c_float]
        lib.or_set_da.restype = C.c_int32
        lib.or_set_da.argtypes = [P, C.c_int32]
        lib.or_mlp.restype = C.c_float
        lib.or_mlp.argtypes = [P, P]
        lib.or_surrogate.restype = C.c_float
        lib.or_surrogate.argtypes = [P, P]
        lib.or_trials_per_sweep.restype = C.c_int64
        lib.or_trials_per_sweep.argtypes = [P]
        lib.or_counts.argtypes = [P, P]
        lib.or_stats.argtypes = [P, P]
        lib.or_n.restype = C.c_int32
        lib.or_n.argtypes = [P]
        lib.or_geometry.argtypes = [P, P]
        lib.or_chem.argtypes = [P, P]
        lib.or_set_pH.argtypes = [P, C.c_double]
        lib.or_ungroup.argtypes = [P, P]
        lib.or_set_invocation.argtypes = [P, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_int32]
        lib.or_set_invocation.restype = C.c_int32
        lib.or_particles.argtypes = [P, P, P, P, P, P]
        lib.or_site_states.argtypes = [P, P]
        lib.or_energy.restype = C.c_double
        lib.or_energy.argtypes = [P]
        lib.or_ewald_parts.argtypes = [P, P]
        lib.or_ewald_nk.restype = C.c_int32
        lib.or_ewald_nk.argtypes = [P]
        lib.or_bond_energy.restype = C.c_double
        lib.or_bond_energy.argtypes = [P]
        lib.or_forces.restype = C.c_int32
        lib.or_forces.argtypes = [P, P, P]
        lib.or_md_step.restype = C.c_int32
        lib.or_md_step.argtypes = [P, C.c_int32, C.c_double, C.c_double, C.c_uint64]
        for f in ("or_md_begin", "or_md_end"):
            getattr(lib, f).restype = C.c_int32
            getattr(lib, f).argtypes = [P, C.c_double, C.c_double, C.c_uint64]
        lib.or_set_positions.restype = C.c_int32
        lib.or_set_positions.argtypes = [P, P, P, P, C.c_int32]
        lib.or_set_bodies.restype = C.c_int32
        lib.or_set_bodies.argtypes = [P, C.c_int32, P, P]
        lib.or_body_state.restype = C.c_int32
        lib.or_body_state.argtypes = [P, P]
        lib.or_set_body_state.restype = C.c_int32
        lib.or_set_body_state.argtypes = [P, P, C.c_int32]
        lib.or_philox.argtypes = [P, P, P]
        lib.or_plant.argtypes = [C.c_int]
        for f in ("or_dsf_phi", "or_dsf_force"):
            getattr(lib, f).restype = C.c_double
            getattr(lib, f).argtypes = [C.c_double, C.c_double, C.c_double]
        lib.or_wca_u.restype = C.c_double
        lib.or_wca_u.argtypes = [C.c_double] * 4
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox(ctr, key):
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox(_ptr(c), _ptr(k), _ptr(out))
    return out


def dsf_phi(alpha, rc, r):
    return _load().or_dsf_phi(alpha, rc, r)


def dsf_force(alpha, rc, r):
    return _load().or_dsf_force(alpha, rc, r)


def wca_u(eps, sig, delta, r):
    return _load().or_wca_u(eps, sig, delta, r)


def plant(kind: str):
    """Plant a deliberate mistake in the oracle (sensitivity tests only)."""
    _load().or_plant(PLANT[kind])


class Oracle:
    """One CR-MC system in the oracle.  Built from a workload spec (see
    ``paper_2109_07527_gb300.workloads.Workload``)."""

    def __init__(self, w, schedule=None, trials_per_domain=None, domain_cells=None):
        lib = _load()
        p = _Params()
        q = w.params
        p.n = w.n
        p.capacity = w.capacity
        p.box_L = q["box_L"]
        p.sigma_nm = q["sigma_nm"]
        p.lB, p.rc, p.alpha = q["lB"], q["rc"], q["alpha"]
        p.dsf_self, p.ion_coupling, p.ion_cls = int(q["dsf_self"]), int(q["ion_coupling"]), int(q["ion_cls"])
        p.pH, p.pKw, p.pIS_plus, p.pIS_minus = q["pH"], q["pKw"], q["pIS_plus"], q["pIS_minus"]
        p.pIX_explicit = int(q.get("pIX_explicit", 0))
        p.pIX_plus, p.pIX_minus = q.get("pIX_plus", 0.0), q.get("pIX_minus", 0.0)
        p.nc = int(q.get("nc", 0))
        p.domain_cells = int(domain_cells if domain_cells is not None else q.get("domain_cells", 0))
        p.trials_per_domain = int(trials_per_domain if trials_per_domain is not None else q["trials_per_domain"])
        p.schedule = int(schedule if schedule is not None else q["schedule"])
        p.cells_per_rc = int(q.get("cells_per_rc", 2))
        for i in range(16):
            p.wca_eps[i] = q["wca_eps"][i]
            p.wca_sig[i] = q["wca_sig"][i]
            p.wca_del[i] = q["wca_del"][i]
            p.wca_on[i] = int(q["wca_on"][i])
        p.fene_K, p.fene_R0 = q["fene_K"], q["fene_R0"]
        p.n_bonds = int(w.bonds.shape[0])
        p.ewald_kmax = int(q.get("ewald_kmax", 0))
        self._keep = [np.ascontiguousarray(w.xyz, dtype=np.float32), np.ascontiguousarray(w.type, dtype=np.int32),
                      np.ascontiguousarray(w.cls, dtype=np.int32), np.ascontiguousarray(w.state, dtype=np.int8),
                      np.ascontiguousarray(w.pK, dtype=np.float64), np.ascontiguousarray(w.bonds, dtype=np.int32),
                      None if w.vel is None else np.ascontiguousarray(w.vel, dtype=np.float32)]
        err = C.c_int32(0)
        h = lib.or_create(C.byref(p), *[_ptr(a) for a in self._keep], C.byref(err))
        if not h:
            raise ValueError(f"oracle rejected the system (code {err.value})")
        self._h = C.c_void_p(h)
        self._lib = lib
        self.capacity = w.capacity

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_destroy(h)
            self._h = None

    @property
    def trials_per_sweep(self) -> int:
        return int(self._lib.or_trials_per_sweep(self._h))

    def geometry(self):
        g = np.zeros(6, dtype=np.int32)
        self._lib.or_geometry(self._h, _ptr(g))
        return dict(nc=int(g[0]), k=int(g[1]), nd=int(g[2]), ncol=int(g[3]), m=int(g[4]), global_=bool(g[5]))

    def chem(self):
        c = np.zeros(7)
        self._lib.or_chem(self._h, _ptr(c))
        return dict(pIX_plus=c[0], pIX_minus=c[1], ln_z1=c[2], ln_salt=c[3], a=c[4], self_coef=c[5], pOH=c[6])

    def set_pH(self, pH):
        """A new reservoir pH from the next trial on (chemistry recomputed)."""
        self._lib.or_set_pH(self._h, float(pH))

    def set_invocation(self, cation, anion, pI_cation, pI_anion, reactions=7):
        """Reactions of the following sweeps exchange ions of types `cation`
        (3 X+ or 6 S+) and `anion` (4 X- or 7 S-) at the given pI; reactions:
        bit mask acid 1, base 2, salt 4."""
        rc = self._lib.or_set_invocation(self._h, int(cation), int(anion), float(pI_cation), float(pI_anion),
                                         int(reactions))
        if rc != 0:
            raise ValueError(f"or_set_invocation rejected the arguments ({rc})")

    def ungroup(self):
        """Subspecies fractions of the grouped ions: p_S+, p_H+ (in X+),
        p_S-, p_OH- (in X-)."""
        c = np.zeros(4)
        self._lib.or_ungroup(self._h, _ptr(c))
        return dict(p_Sp=c[0], p_H=c[1], p_Sm=c[2], p_OH=c[3])

    def set_surrogate(self, mlp):
        """Surrogate weights: dict with W1 [128,48], W2, W3 [128,128], w4 [128]
        as uint16 BF16 bit patterns and b1, b2, b3 [128] float32, b4 float."""
        self._mlp = {k: np.ascontiguousarray(mlp[k], dtype=np.uint16) for k in ("W1", "W2", "W3", "w4")}
        self._mlp.update({k: np.ascontiguousarray(mlp[k], dtype=np.float32) for k in ("b1", "b2", "b3")})
        m = self._mlp
        self._lib.or_set_surrogate(self._h, _ptr(m["W1"]), _ptr(m["b1"]), _ptr(m["W2"]), _ptr(m["b2"]),
                                   _ptr(m["W3"]), _ptr(m["b3"]), _ptr(m["w4"]), float(mlp["b4"]))

    def set_da(self, on=True):
        if self._lib.or_set_da(self._h, 1 if on else 0) != 0:
            raise ValueError("delayed acceptance needs a surrogate (set_surrogate)")

    def mlp(self, F):
        F = np.ascontiguousarray(F, dtype=np.float32)
        return float(self._lib.or_mlp(self._h, _ptr(F)))

    def surrogate(self, F):
        F = np.ascontiguousarray(F, dtype=np.float32)
        return float(self._lib.or_surrogate(self._h, _ptr(F)))

    def sweep(self, n_trials, seed, log=False, forced=None, hist_n=0, trans=False, da_log=False, features=False):
        n_trials = int(n_trials)
        rec = np.zeros(n_trials, dtype=TRIAL_DTYPE) if log else None
        f = None if forced is None else np.ascontiguousarray(forced, dtype=np.int8)
        hist = np.zeros(1 << hist_n, dtype=np.int64) if hist_n else None
        tr = np.zeros((1 << hist_n) * hist_n, dtype=np.int64) if (trans and hist_n) else None
        dl = np.zeros(n_trials, dtype=DA_DTYPE) if da_log else None
        feat = np.zeros((n_trials, N_FEAT), dtype=np.float32) if features else None
        dep = np.zeros(n_trials, dtype=np.float64) if features else None
        rc = self._lib.or_sweep(self._h, n_trials, C.c_uint64(seed), _ptr(rec), _ptr(f), _ptr(hist), hist_n,
                                _ptr(tr), _ptr(dl), _ptr(feat), _ptr(dep))
        if rc != 0:
            raise RuntimeError(f"or_sweep failed with code {rc}")
        out = {}
        if log:
            out["log"] = rec
        if da_log:
            out["da"] = dl
        if features:
            out["features"] = feat
            out["dE_pair"] = dep
        if hist_n:
            out["hist"] = hist
        if tr is not None:
            out["trans"] = tr.reshape(1 << hist_n, hist_n)
        return out

    def counts(self):
        c = np.zeros(10, dtype=np.int64)
        self._lib.or_counts(self._h, _ptr(c))
        return dict(n_A=int(c[0]), n_Am=int(c[1]), n_B=int(c[2]), n_Bp=int(c[3]), n_Xp=int(c[4]), n_Xm=int(c[5]),
                    n=int(c[6]), net_charge=int(c[7]), n_Sp=int(c[8]), n_Sm=int(c[9]))

    def stats(self):
        s = np.zeros(16, dtype=np.int64)
        self._lib.or_stats(self._h, _ptr(s))
        return dict(attempts=s[:6].copy(), accepts=s[6:12].copy())

    def particles(self):
        """Particles sorted by id: dict of id, xyz, type, state, vel."""
        n = int(self._lib.or_n(self._h))
        xyz = np.zeros((n, 3), dtype=np.float32)
        ids = np.zeros(n, dtype=np.uint64)
        t = np.zeros(n, dtype=np.int32)
        st = np.zeros(n, dtype=np.int8)
        v = np.zeros((n, 3), dtype=np.float64)
        self._lib.or_particles(self._h, _ptr(xyz), _ptr(ids), _ptr(t), _ptr(st), _ptr(v))
        o = np.argsort(ids, kind="stable")
        return dict(id=ids[o], xyz=xyz[o], type=t[o], state=st[o], vel=v[o], order=o)

    def site_states(self, n_sites):
        s = np.zeros(n_sites, dtype=np.int8)
        self._lib.or_site_states(self._h, _ptr(s))
        return s

    def energy(self) -> float:
        return float(self._lib.or_energy(self._h))

    def ewald_parts(self):
        """Ewald parts of the Coulomb energy: (real space within rc, reciprocal, self)."""
        out = np.zeros(3)
        self._lib.or_ewald_parts(self._h, _ptr(out))
        return tuple(float(v) for v in out)

    @property
    def ewald_nk(self) -> int:
        return int(self._lib.or_ewald_nk(self._h))

    def bond_energy(self) -> float:
        return float(self._lib.or_bond_energy(self._h))

    def forces(self):
        """Conservative forces, sorted by id, and the per-component sums of |pair force|."""
        n = int(self._lib.or_n(self._h))
        F = np.zeros((n, 3))
        S = np.zeros((n, 3))
        rc = self._lib.or_forces(self._h, _ptr(F), _ptr(S))
        if rc != 0:
            raise RuntimeError(f"or_forces failed with code {rc}")
        ids = np.zeros(n, dtype=np.uint64)
        self._lib.or_particles(self._h, None, _ptr(ids), None, None, None)
        o = np.argsort(ids, kind="stable")
        return ids[o], F[o], S[o]

    def md_step(self, n_steps, dt, gamma, seed):
        rc = self._lib.or_md_step(self._h, int(n_steps), float(dt), float(gamma), C.c_uint64(seed))
        if rc != 0:
            raise RuntimeError(f"or_md_step failed with code {rc}")

    def md_begin(self, dt, gamma, seed):
        """First half of an MD step (forces if stale, half kick, drift)."""
        rc = self._lib.or_md_begin(self._h, float(dt), float(gamma), C.c_uint64(seed))
        if rc != 0:
            raise RuntimeError(f"or_md_begin failed with code {rc}")

    def md_end(self, dt, gamma, seed):
        """Second half of an MD step (forces with the current charges, half kick)."""
        rc = self._lib.or_md_end(self._h, float(dt), float(gamma), C.c_uint64(seed))
        if rc != 0:
            raise RuntimeError(f"or_md_end failed with code {rc}")

    def set_bodies(self, first, count):
        """Declare rigid bodies: body b is the permanent ids [first[b], first[b] + count[b])."""
        f = np.ascontiguousarray(first, dtype=np.int32)
        c = np.ascontiguousarray(count, dtype=np.int32)
        if f.shape != c.shape:
            raise ValueError("first and count differ in length")
        rc = self._lib.or_set_bodies(self._h, len(f), _ptr(f), _ptr(c))
        if rc != 0:
            raise ValueError(f"or_set_bodies refused the bodies (code {rc})")
        self._n_bodies = len(f)
        self.bodies = (f.copy(), c.copy())

    def body_state(self):
        """Per body: X[3], V[3], R[9] (row-major, lab = R body), pi[3] (body frame), I[3], M."""
        out = np.zeros((getattr(self, "_n_bodies", 0), 22))
        self._lib.or_body_state(self._h, _ptr(out))
        return out

    def set_body_state(self, rec):
        rec = np.ascontiguousarray(rec, dtype=np.float64)
        if self._lib.or_set_body_state(self._h, _ptr(rec), len(rec)) != 0:
            raise ValueError("body count mismatch")

    def set_positions(self, ids, xyz, vel=None):
        ids = np.ascontiguousarray(ids, dtype=np.uint64)
        o = np.argsort(ids, kind="stable")
        ids = ids[o]
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32)[o])
        v = None if vel is None else np.ascontiguousarray(np.asarray(vel, dtype=np.float32)[o])
        rc = self._lib.or_set_positions(self._h, _ptr(ids), _ptr(xyz), _ptr(v), len(ids))
        if rc != 0:
            raise RuntimeError("or_set_positions: particle set mismatch")
