"""Python binding of libcrmc.so (the C ABI in include/crmc.h).

Argument marshalling only: every step of the CR-MC path runs in the library's
CUDA kernels.  Importing this module loads the library and raises if it has
not been built (``__graft_entry__.build()`` or ``python -m
paper_2109_07527_gb300.build``); there is no CPU fallback.  PyTorch, when
present, supplies the CUDA stream the library queues its work on.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrmc.so")

CR_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NOT_NEUTRAL", -3: "CELL_OVERFLOW", -4: "CAPACITY", -5: "TIMEOUT",
          -6: "BOND_BROKEN", -7: "CUDA", -8: "NOMEM", -9: "NO_DEVICE"}
SCHED_COLOURED, SCHED_GLOBAL = 0, 1
TRIAL_ACCEPTED, TRIAL_NO_ELIGIBLE, TRIAL_EDGE, TRIAL_OVERLAP = 1, 2, 4, 8


class CrError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what} failed: {ERRORS.get(code, code)} ({_lib().cr_strerror(code).decode()})")
        self.code = code


class cr_system(C.Structure):
    _fields_ = [("n", C.c_int32), ("capacity", C.c_int32), ("box_L", C.c_double), ("sigma_nm", C.c_double),
                ("xyz", C.c_void_p), ("type", C.c_void_p), ("cls", C.c_void_p), ("state", C.c_void_p),
                ("vel", C.c_void_p), ("n_bonds", C.c_int32), ("bonds", C.c_void_p),
                ("fene_K", C.c_double), ("fene_R0", C.c_double),
                ("wca_eps", C.c_double * 16), ("wca_sig", C.c_double * 16), ("wca_del", C.c_double * 16),
                ("wca_on", C.c_int32 * 16),
                ("dsf_alpha", C.c_double), ("dsf_self", C.c_int32), ("ion_coupling", C.c_int32),
                ("ion_cls", C.c_int32), ("cells_per_rc", C.c_int32), ("domain_cells", C.c_int32),
                ("trials_per_domain", C.c_int32), ("schedule", C.c_int32), ("nc", C.c_int32),
                ("cell_capacity", C.c_int32), ("list_capacity", C.c_int32), ("halo_capacity", C.c_int32),
                ("ewald_kmax", C.c_int32)]


class cr_mu_ions(C.Structure):
    _fields_ = [("pI_S_plus", C.c_double), ("pI_S_minus", C.c_double), ("pKw", C.c_double),
                ("pIX_explicit", C.c_int32), ("pIX_plus", C.c_double), ("pIX_minus", C.c_double)]


class cr_sweep_stats(C.Structure):
    _fields_ = [("trials", C.c_int64), ("attempts", C.c_int64 * 6), ("accepts", C.c_int64 * 6),
                ("no_eligible", C.c_int64), ("edge", C.c_int64), ("overlap", C.c_int64)]


class cr_state_view(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_A", C.c_int64), ("n_Am", C.c_int64), ("n_B", C.c_int64),
                ("n_Bp", C.c_int64), ("n_Xp", C.c_int64), ("n_Xm", C.c_int64), ("net_charge", C.c_int64),
                ("alpha", C.c_double), ("n_Sp", C.c_int64), ("n_Sm", C.c_int64), ("xyz", C.c_void_p),
                ("vel", C.c_void_p), ("force", C.c_void_p), ("id", C.c_void_p), ("type", C.c_void_p),
                ("state", C.c_void_p), ("site_state", C.c_void_p), ("cls", C.c_void_p)]


class cr_load_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("xyz", C.c_void_p), ("vel", C.c_void_p), ("type", C.c_void_p),
                ("cls", C.c_void_p), ("state", C.c_void_p)]


class cr_batch_packed(C.Structure):
    _fields_ = [("stride", C.c_int64), ("xyz", C.c_void_p), ("vel", C.c_void_p), ("id", C.c_void_p),
                ("type", C.c_void_p), ("cls", C.c_void_p), ("state", C.c_void_p), ("n", C.c_void_p)]


class cr_info(C.Structure):
    _fields_ = [("nc", C.c_int32), ("k", C.c_int32), ("h", C.c_int32), ("nd", C.c_int32), ("ncol", C.c_int32),
                ("m", C.c_int32), ("cap", C.c_int32), ("global_", C.c_int32), ("trials_per_sweep", C.c_int64),
                ("n_sites", C.c_int32), ("n_perm", C.c_int32), ("cell_side", C.c_double),
                ("domain_side", C.c_double)]


TRIAL_DTYPE = np.dtype([("move", "<i4"), ("flags", "<i4"), ("id_a", "<u8"), ("id_b", "<u8"),
                        ("dE", "<f8"), ("S", "<f8"), ("lnA", "<f8"), ("lnu", "<f8")])
DA_DTYPE = np.dtype([("dE_sur", "<f4"), ("stage", "<i4"), ("lnA2", "<f8"), ("lnu2", "<f8")])
N_FEAT = 48


class cr_device_buffers(C.Structure):
    _fields_ = [("cnt", C.c_void_p), ("pos", C.c_void_p), ("vel", C.c_void_p), ("id", C.c_void_p),
                ("info", C.c_void_p), ("n_cells", C.c_int64), ("n_slots", C.c_int64)]


class cr_mlp(C.Structure):
    _fields_ = [("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p), ("b2", C.c_void_p),
                ("W3", C.c_void_p), ("b3", C.c_void_p), ("w4", C.c_void_p), ("b4", C.c_float)]

# every entry point of include/crmc.h
EXPORTS = ("cr_init", "cr_sweep", "cr_sweep_log", "cr_md_forces", "cr_md_step", "cr_state", "cr_get_info",
           "cr_set_stream", "cr_check", "cr_destroy", "cr_strerror", "cr_philox", "cr_load", "cr_set_timing",
           "cr_get_timing", "cr_set_launch_shape", "cr_get_launch_shape", "cr_batch_create", "cr_batch_sweep",
           "cr_batch_md_step", "cr_batch_get_launch_shape", "cr_batch_destroy", "cr_md_forces_noalloc",
           "cr_set_surrogate", "cr_sweep_da", "cr_sweep_da_log", "cr_batch_sweep_da", "cr_train_create",
           "cr_train_set_stream", "cr_train_step", "cr_train_gradients", "cr_train_get", "cr_train_stats",
           "cr_train_destroy", "cr_mma_bf16", "cr_md_begin", "cr_md_end", "cr_batch_md_begin",
           "cr_batch_md_end", "cr_batch_set_launch_shape", "cr_batch_state", "cr_batch_load",
           "cr_batch_state_packed", "cr_batch_load_packed", "cr_train_apply", "cr_train_moments",
           "cr_checkpoint", "cr_restore", "cr_selftest_mma_timeout", "cr_set_pH", "cr_ungroup",
           "cr_batch_set_persistent", "cr_batch_selftest_wait_timeout", "cr_batch_cycle", "cr_set_invocation",
           "cr_bind_device_buffers", "cr_set_rigid_bodies", "cr_rigid_body_state")
N_PARAMS = 39425  # CR_TRAIN_N_PARAMS


class cr_counters(C.Structure):
    _fields_ = [("sweep", C.c_uint64), ("md_eval", C.c_uint32), ("forces_valid", C.c_int32)]


class cr_ungrouped(C.Structure):
    _fields_ = [(f, C.c_double) for f in ("p_S_plus", "p_H", "p_S_minus", "p_OH", "n_S_plus", "n_H", "n_S_minus",
                                          "n_OH")]


class cr_train_cfg(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double), ("target_clip", C.c_double), ("unfused", C.c_int32)]

_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcrmc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        lib = C.CDLL(LIB_PATH)
        P = C.c_void_p
        lib.cr_init.restype = C.c_int
        lib.cr_init.argtypes = [C.POINTER(P), C.POINTER(cr_system), C.c_double, P, cr_mu_ions, C.c_double, C.c_double]
        lib.cr_sweep.restype = C.c_int
        lib.cr_sweep.argtypes = [P, C.c_uint64, C.c_uint64, C.POINTER(cr_sweep_stats)]
        lib.cr_sweep_log.restype = C.c_int
        lib.cr_sweep_log.argtypes = [P, C.c_uint64, C.c_uint64, C.POINTER(cr_sweep_stats), P]
        lib.cr_md_forces.restype = C.c_int
        lib.cr_md_forces.argtypes = [P]
        lib.cr_md_step.restype = C.c_int
        for f in ("cr_md_begin", "cr_md_end", "cr_batch_md_begin", "cr_batch_md_end"):
            getattr(lib, f).restype = C.c_int
            getattr(lib, f).argtypes = [P, C.c_double, C.c_double, C.c_uint64]
        lib.cr_train_create.restype = C.c_int
        lib.cr_train_create.argtypes = [C.POINTER(P), C.POINTER(cr_mlp), C.POINTER(cr_train_cfg)]
        lib.cr_train_set_stream.restype = C.c_int
        lib.cr_train_set_stream.argtypes = [P, P]
        lib.cr_train_step.restype = C.c_int
        lib.cr_train_step.argtypes = [P, P, P, C.c_int32, P]
        lib.cr_train_gradients.restype = C.c_int
        lib.cr_train_gradients.argtypes = [P, P, P, C.c_int32, P, P]
        lib.cr_train_get.restype = C.c_int
        lib.cr_train_get.argtypes = [P] + [P] * 9
        lib.cr_train_apply.restype = C.c_int
        lib.cr_train_apply.argtypes = [P, P]
        lib.cr_train_moments.restype = C.c_int
        lib.cr_train_moments.argtypes = [P, P, P]
        lib.cr_train_stats.restype = C.c_int
        lib.cr_train_stats.argtypes = [P, P, P]
        lib.cr_train_destroy.restype = None
        lib.cr_train_destroy.argtypes = [P]
        lib.cr_selftest_mma_timeout.restype = C.c_int
        lib.cr_selftest_mma_timeout.argtypes = [P, P, P, C.c_uint32, P]
        lib.cr_mma_bf16.restype = C.c_int
        lib.cr_mma_bf16.argtypes = [P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P]
        lib.cr_set_surrogate.restype = C.c_int
        lib.cr_set_surrogate.argtypes = [P, C.POINTER(cr_mlp)]
        lib.cr_sweep_da.restype = C.c_int
        lib.cr_sweep_da.argtypes = [P, C.c_uint64, C.c_uint64, C.POINTER(cr_sweep_stats)]
        lib.cr_sweep_da_log.restype = C.c_int
        lib.cr_sweep_da_log.argtypes = [P, C.c_uint64, C.c_uint64, C.POINTER(cr_sweep_stats), P, P, P]
        lib.cr_batch_sweep_da.restype = C.c_int
        lib.cr_batch_sweep_da.argtypes = [P, C.c_uint64, C.c_uint64]
        lib.cr_md_forces_noalloc.restype = C.c_int
        lib.cr_md_forces_noalloc.argtypes = [P, P, P, C.c_int64]
        lib.cr_bind_device_buffers.restype = C.c_int
        lib.cr_bind_device_buffers.argtypes = [P, C.POINTER(cr_device_buffers)]
        lib.cr_set_rigid_bodies.restype = C.c_int
        lib.cr_set_rigid_bodies.argtypes = [P, C.c_int32, P, P]
        lib.cr_rigid_body_state.restype = C.c_int
        lib.cr_rigid_body_state.argtypes = [P, C.c_int32, P]
        lib.cr_md_step.argtypes = [P, C.c_int32, C.c_double, C.c_double, C.c_uint64]
        lib.cr_state.restype = C.c_int
        lib.cr_state.argtypes = [P, C.POINTER(cr_state_view)]
        lib.cr_batch_state.restype = C.c_int
        lib.cr_batch_state.argtypes = [P, C.POINTER(cr_state_view)]
        lib.cr_batch_load.restype = C.c_int
        lib.cr_batch_load.argtypes = [P, C.POINTER(cr_load_args)]
        for f in ("cr_batch_state_packed", "cr_batch_load_packed"):
            getattr(lib, f).restype = C.c_int
            getattr(lib, f).argtypes = [P, C.POINTER(cr_batch_packed)]
        lib.cr_get_info.restype = C.c_int
        lib.cr_get_info.argtypes = [P, C.POINTER(cr_info)]
        lib.cr_set_stream.restype = C.c_int
        lib.cr_set_stream.argtypes = [P, P]
        lib.cr_check.restype = C.c_int
        lib.cr_check.argtypes = [P]
        lib.cr_destroy.restype = None
        lib.cr_destroy.argtypes = [P]
        lib.cr_strerror.restype = C.c_char_p
        lib.cr_strerror.argtypes = [C.c_int]
        lib.cr_set_pH.restype = C.c_int
        lib.cr_set_pH.argtypes = [P, C.c_double]
        lib.cr_set_invocation.restype = C.c_int
        lib.cr_set_invocation.argtypes = [P, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_uint32]
        lib.cr_ungroup.restype = C.c_int
        lib.cr_ungroup.argtypes = [P, C.POINTER(cr_ungrouped)]
        lib.cr_checkpoint.restype = C.c_int
        lib.cr_checkpoint.argtypes = [P, C.POINTER(cr_state_view), C.POINTER(cr_counters)]
        lib.cr_restore.restype = C.c_int
        lib.cr_restore.argtypes = [P, C.c_int32, P, P, P, P, P, P, P, C.POINTER(cr_counters)]
        lib.cr_load.restype = C.c_int
        lib.cr_load.argtypes = [P, C.c_int32, P, P, P, P, P]
        lib.cr_set_timing.restype = C.c_int
        lib.cr_set_timing.argtypes = [P, C.c_int32]
        lib.cr_get_timing.restype = C.c_int
        lib.cr_get_timing.argtypes = [P, P, P, P, C.c_int32]
        lib.cr_set_launch_shape.restype = C.c_int
        lib.cr_set_launch_shape.argtypes = [P, C.c_int32, C.c_int32]
        lib.cr_get_launch_shape.restype = C.c_int
        lib.cr_get_launch_shape.argtypes = [P, P, P]
        lib.cr_batch_create.restype = C.c_int
        lib.cr_batch_create.argtypes = [C.POINTER(P), P, C.c_int32]
        lib.cr_batch_sweep.restype = C.c_int
        lib.cr_batch_sweep.argtypes = [P, C.c_uint64, C.c_uint64]
        lib.cr_batch_md_step.restype = C.c_int
        lib.cr_batch_md_step.argtypes = [P, C.c_int32, C.c_double, C.c_double, C.c_uint64]
        lib.cr_batch_cycle.restype = C.c_int
        lib.cr_batch_cycle.argtypes = [P, C.c_int32, C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_int32]
        lib.cr_batch_set_persistent.restype = C.c_int
        lib.cr_batch_set_persistent.argtypes = [P, C.c_int32, C.c_int32]
        lib.cr_batch_selftest_wait_timeout.restype = C.c_int
        lib.cr_batch_selftest_wait_timeout.argtypes = [P, C.c_int32, C.c_double]
        lib.cr_batch_set_launch_shape.restype = C.c_int
        lib.cr_batch_set_launch_shape.argtypes = [P, C.c_int32, C.c_int32]
        lib.cr_batch_get_launch_shape.restype = C.c_int
        lib.cr_batch_get_launch_shape.argtypes = [P, P, P]
        lib.cr_batch_destroy.restype = None
        lib.cr_batch_destroy.argtypes = [P]
        lib.cr_philox.restype = C.c_int
        lib.cr_philox.argtypes = [C.c_uint32] * 6 + [C.c_int32, P]
        _L = lib
    return _L


def _chk(code, what):
    if code != CR_OK:
        raise CrError(code, what)


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox(c0, c1, c2, c3, k0, k1, n):
    """Philox4x32-10 blocks for counters (c0 + i, c1, c2, c3), i < n, on the GPU."""
    out = np.zeros((n, 4), dtype=np.uint32)
    _chk(_lib().cr_philox(c0, c1, c2, c3, k0, k1, n, _p(out)), "cr_philox")
    return out


def _view(**arrays):
    """A cr_state_view over caller arrays (numpy arrays or raw pointers; None = not wanted)."""
    v = cr_state_view()
    for k, a in arrays.items():
        setattr(v, k, None if a is None else (C.c_void_p(a) if isinstance(a, int) else _p(a)))
    return v


def _view_counts(v):
    return dict(n=v.n, n_A=v.n_A, n_Am=v.n_Am, n_B=v.n_B, n_Bp=v.n_Bp, n_Xp=v.n_Xp, n_Xm=v.n_Xm,
                net_charge=v.net_charge, alpha=v.alpha, n_Sp=v.n_Sp, n_Sm=v.n_Sm)


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


class Context:
    """A CR-MC system on the GPU (owns one cr_ctx)."""

    def __init__(self, w, schedule=None, trials_per_domain=None, domain_cells=None, cell_capacity=0, stream=None,
                 list_capacity=0, halo_capacity=0):
        lib = _lib()
        self._nbatch = 0  # live batches that hold this context (it must outlive them)
        q = w.params
        s = cr_system()
        self._keep = dict(xyz=np.ascontiguousarray(w.xyz, np.float32), type=np.ascontiguousarray(w.type, np.int32),
                          cls=np.ascontiguousarray(w.cls, np.int32), state=np.ascontiguousarray(w.state, np.int8),
                          vel=None if w.vel is None else np.ascontiguousarray(w.vel, np.float32),
                          bonds=np.ascontiguousarray(w.bonds, np.int32), pK=np.ascontiguousarray(w.pK, np.float64))
        k = self._keep
        s.n, s.capacity, s.box_L, s.sigma_nm = w.n, w.capacity, q["box_L"], q["sigma_nm"]
        s.xyz, s.type, s.cls, s.state, s.vel = _p(k["xyz"]), _p(k["type"]), _p(k["cls"]), _p(k["state"]), _p(k["vel"])
        s.n_bonds, s.bonds = int(w.bonds.shape[0]), _p(k["bonds"])
        s.fene_K, s.fene_R0 = q["fene_K"], q["fene_R0"]
        for i in range(16):
            s.wca_eps[i], s.wca_sig[i], s.wca_del[i] = q["wca_eps"][i], q["wca_sig"][i], q["wca_del"][i]
            s.wca_on[i] = int(q["wca_on"][i])
        s.dsf_alpha, s.dsf_self = q["alpha"], int(q["dsf_self"])
        s.ion_coupling, s.ion_cls = int(q["ion_coupling"]), int(q["ion_cls"])
        s.cells_per_rc = int(q.get("cells_per_rc", 2))
        s.domain_cells = int(domain_cells if domain_cells is not None else q.get("domain_cells", 0))
        s.trials_per_domain = int(trials_per_domain if trials_per_domain is not None else q["trials_per_domain"])
        s.schedule = int(schedule if schedule is not None else q["schedule"])
        s.nc = int(q.get("nc", 0))
        s.cell_capacity = int(cell_capacity)
        s.list_capacity = int(list_capacity)
        s.halo_capacity = int(halo_capacity)
        s.ewald_kmax = int(q.get("ewald_kmax", 0))
        mu = cr_mu_ions(q["pIS_plus"], q["pIS_minus"], q["pKw"], int(q.get("pIX_explicit", 0)),
                        q.get("pIX_plus", 0.0), q.get("pIX_minus", 0.0))
        h = C.c_void_p()
        _chk(lib.cr_init(C.byref(h), C.byref(s), q["pH"], _p(k["pK"]), mu, q["lB"], q["rc"]), "cr_init")
        self._h = h
        self._lib = lib
        st = stream if stream is not None else _torch_stream()
        if st is not None:
            _chk(lib.cr_set_stream(h, st), "cr_set_stream")
        self.n_sites = w.n_sites
        self.capacity = w.capacity

    def close(self):
        if getattr(self, "_nbatch", 0):
            raise RuntimeError("the context is part of a live Batch: close the batch first")
        if getattr(self, "_h", None):
            self._lib.cr_destroy(self._h)
            self._h = None

    def __del__(self):
        if not getattr(self, "_nbatch", 0):
            self.close()

    @property
    def info(self):
        i = cr_info()
        _chk(self._lib.cr_get_info(self._h, C.byref(i)), "cr_get_info")
        return {f: getattr(i, f) for f, _ in cr_info._fields_}

    @property
    def trials_per_sweep(self):
        return int(self.info["trials_per_sweep"])

    def sweep(self, n_trials, seed, stats=False, log=False):
        st = cr_sweep_stats() if stats else None
        if log:
            rec = np.zeros(int(n_trials), dtype=TRIAL_DTYPE)
            _chk(self._lib.cr_sweep_log(self._h, int(n_trials), int(seed), C.byref(st) if st else None, _p(rec)),
                 "cr_sweep_log")
        else:
            rec = None
            _chk(self._lib.cr_sweep(self._h, int(n_trials), int(seed), C.byref(st) if st else None), "cr_sweep")
        out = {}
        if st is not None:
            out["stats"] = dict(trials=st.trials, attempts=np.array(st.attempts[:]), accepts=np.array(st.accepts[:]),
                                no_eligible=st.no_eligible, edge=st.edge, overlap=st.overlap)
        if rec is not None:
            out["log"] = rec
        return out

    def set_surrogate(self, mlp):
        """Surrogate weights: dict with W1 [128,48], W2, W3 [128,128], w4 [128]
        (uint16 BF16 bit patterns), b1, b2, b3 [128] float32 and b4."""
        k = {n: np.ascontiguousarray(mlp[n], dtype=np.uint16) for n in ("W1", "W2", "W3", "w4")}
        k.update({n: np.ascontiguousarray(mlp[n], dtype=np.float32) for n in ("b1", "b2", "b3")})
        m = cr_mlp(_p(k["W1"]), _p(k["b1"]), _p(k["W2"]), _p(k["b2"]), _p(k["W3"]), _p(k["b3"]), _p(k["w4"]),
                   float(mlp["b4"]))
        _chk(self._lib.cr_set_surrogate(self._h, C.byref(m)), "cr_set_surrogate")

    def sweep_da(self, n_trials, seed, stats=False, log=False, features=False):
        """Delayed-acceptance sweeps; log=True also returns the DA records
        ("da") and, with features=True, the 48 surrogate inputs per trial."""
        st = cr_sweep_stats() if stats else None
        out = {}
        if log:
            n = int(n_trials)
            rec = np.zeros(n, dtype=TRIAL_DTYPE)
            drec = np.zeros(n, dtype=DA_DTYPE)
            feat = np.zeros((n, N_FEAT), dtype=np.float32) if features else None
            _chk(self._lib.cr_sweep_da_log(self._h, n, int(seed), C.byref(st) if st else None, _p(rec), _p(drec),
                                           _p(feat)), "cr_sweep_da_log")
            out.update(log=rec, da=drec)
            if features:
                out["features"] = feat
        else:
            _chk(self._lib.cr_sweep_da(self._h, int(n_trials), int(seed), C.byref(st) if st else None), "cr_sweep_da")
        if st is not None:
            out["stats"] = dict(trials=st.trials, attempts=np.array(st.attempts[:]), accepts=np.array(st.accepts[:]),
                                no_eligible=st.no_eligible, edge=st.edge, overlap=st.overlap)
        return out

    def md_forces(self):
        _chk(self._lib.cr_md_forces(self._h), "cr_md_forces")

    def md_forces_noalloc(self, force_ptr, id_ptr, n_slots):
        """cr_md_forces_noalloc into caller-owned device memory given as raw
        pointers: force [4 * n_slots] float32, id [n_slots] uint64."""
        _chk(self._lib.cr_md_forces_noalloc(self._h, C.c_void_p(int(force_ptr)), C.c_void_p(int(id_ptr)),
                                            int(n_slots)), "cr_md_forces_noalloc")

    def bind_device_buffers(self, cnt_ptr, pos_ptr, vel_ptr, id_ptr, info_ptr, n_cells, n_slots):
        """cr_bind_device_buffers: the configuration's slot arrays in caller-owned
        device memory given as raw pointers (cnt [n_cells] int32, pos and vel
        [4 n_slots] float32, id [n_slots] uint64, info [n_slots] int32)."""
        b = cr_device_buffers(C.c_void_p(int(cnt_ptr)), C.c_void_p(int(pos_ptr)), C.c_void_p(int(vel_ptr)),
                              C.c_void_p(int(id_ptr)), C.c_void_p(int(info_ptr)), int(n_cells), int(n_slots))
        _chk(self._lib.cr_bind_device_buffers(self._h, C.byref(b)), "cr_bind_device_buffers")

    def set_rigid_bodies(self, first, count):
        """cr_set_rigid_bodies: body b is the permanent ids [first[b], first[b] + count[b])."""
        f = np.ascontiguousarray(first, dtype=np.int32)
        c = np.ascontiguousarray(count, dtype=np.int32)
        if f.shape != c.shape or f.ndim != 1:
            raise ValueError("first and count must be 1-d arrays of one length")
        _chk(self._lib.cr_set_rigid_bodies(self._h, len(f), f.ctypes.data_as(C.c_void_p),
                                           c.ctypes.data_as(C.c_void_p)), "cr_set_rigid_bodies")
        self.n_bodies = len(f)

    def rigid_body_state(self):
        """cr_rigid_body_state: per body X[3], V[3], R[9] (row-major), pi[3], I[3], M."""
        n = getattr(self, "n_bodies", 0)
        out = np.zeros((n, 22))
        _chk(self._lib.cr_rigid_body_state(self._h, n, out.ctypes.data_as(C.c_void_p)), "cr_rigid_body_state")
        return out

    def md_begin(self, dt, gamma, seed):
        _chk(self._lib.cr_md_begin(self._h, float(dt), float(gamma), int(seed)), "cr_md_begin")

    def md_end(self, dt, gamma, seed):
        _chk(self._lib.cr_md_end(self._h, float(dt), float(gamma), int(seed)), "cr_md_end")

    def md_step(self, n_steps, dt, gamma, seed):
        _chk(self._lib.cr_md_step(self._h, int(n_steps), float(dt), float(gamma), int(seed)), "cr_md_step")

    def load(self, n, xyz_ptr, vel_ptr, type_ptr, cls_ptr, state_ptr):
        """Upload a configuration from host buffers given as raw pointers (ints) or numpy arrays."""
        conv = lambda a: None if a is None else (C.c_void_p(a) if isinstance(a, int) else _p(a))
        _chk(self._lib.cr_load(self._h, int(n), conv(xyz_ptr), conv(vel_ptr), conv(type_ptr), conv(cls_ptr),
                               conv(state_ptr)), "cr_load")

    def set_launch_shape(self, threads, regs):
        _chk(self._lib.cr_set_launch_shape(self._h, int(threads), int(regs)), "cr_set_launch_shape")

    def launch_shape(self):
        t = C.c_int32()
        r = C.c_int32()
        _chk(self._lib.cr_get_launch_shape(self._h, C.byref(t), C.byref(r)), "cr_get_launch_shape")
        return t.value, r.value

    def set_timing(self, on=True):
        _chk(self._lib.cr_set_timing(self._h, 1 if on else 0), "cr_set_timing")

    def timing(self, reset=True):
        ms = np.zeros(2)
        la = np.zeros(2, np.int64)
        tot = np.zeros(1, np.int64)
        _chk(self._lib.cr_get_timing(self._h, _p(ms), _p(la), _p(tot), 1 if reset else 0), "cr_get_timing")
        return dict(phase_ms=float(ms[0]), phase_launches=int(la[0]), md_ms=float(ms[1]), md_launches=int(la[1]),
                    launches=int(tot[0]))

    def check(self):
        _chk(self._lib.cr_check(self._h), "cr_check")

    def counts(self):
        v = cr_state_view()
        _chk(self._lib.cr_state(self._h, C.byref(v)), "cr_state")
        return _view_counts(v)

    def state_into(self, xyz=None, vel=None, id=None, type=None, state=None, site_state=None, force=None, cls=None):
        """cr_state into caller-owned host arrays (numpy arrays or raw pointers,
        e.g. pinned buffers reused every step, each sized for the capacity);
        returns the counts."""
        v = _view(xyz=xyz, vel=vel, id=id, type=type, state=state, site_state=site_state, force=force, cls=cls)
        _chk(self._lib.cr_state(self._h, C.byref(v)), "cr_state")
        return _view_counts(v)

    def state(self):
        """Counts and all particles sorted by id."""
        c = self.counts()
        n = int(c["n"])
        arr = dict(xyz=np.zeros((n, 3), np.float32), vel=np.zeros((n, 3), np.float32),
                   force=np.zeros((n, 3), np.float32), id=np.zeros(n, np.uint64), type=np.zeros(n, np.int32),
                   state=np.zeros(n, np.int8), site_state=np.zeros(max(self.n_sites, 1), np.int8),
                   cls=np.zeros(n, np.int32))
        v = cr_state_view()
        v.xyz, v.vel, v.force = _p(arr["xyz"]), _p(arr["vel"]), _p(arr["force"])
        v.id, v.type, v.state, v.site_state = _p(arr["id"]), _p(arr["type"]), _p(arr["state"]), _p(arr["site_state"])
        v.cls = _p(arr["cls"])
        _chk(self._lib.cr_state(self._h, C.byref(v)), "cr_state")
        arr["site_state"] = arr["site_state"][: self.n_sites]
        c.update(arr)
        return c


    def set_pH(self, pH):
        """cr_set_pH: a new reservoir pH from the next trial on."""
        _chk(self._lib.cr_set_pH(self._h, float(pH)), "cr_set_pH")

    def set_invocation(self, cation, anion, pI_cation, pI_anion, reactions=7):
        """cr_set_invocation: the following sweeps' reactions exchange ions of
        types `cation` (CR_XP 3 / CR_SP 6) and `anion` (CR_XM 4 / CR_SM 7) at the
        given pI; reactions: bit mask acid 1, base 2, salt 4."""
        _chk(self._lib.cr_set_invocation(self._h, int(cation), int(anion), float(pI_cation), float(pI_anion),
                                         int(reactions)), "cr_set_invocation")

    def ungroup(self):
        """cr_ungroup: subspecies fractions of X+ / X- and their expected numbers."""
        u = cr_ungrouped()
        _chk(self._lib.cr_ungroup(self._h, C.byref(u)), "cr_ungroup")
        return {f: getattr(u, f) for f, _ in cr_ungrouped._fields_}

    def checkpoint(self):
        """cr_checkpoint: the state arrays (ordered by id; force = the
        integrator's forces when valid) and the counters, as one dict."""
        c = self.counts()
        n = int(c["n"])
        arr = dict(xyz=np.zeros((n, 3), np.float32), vel=np.zeros((n, 3), np.float32),
                   force=np.zeros((n, 3), np.float32), id=np.zeros(n, np.uint64), type=np.zeros(n, np.int32),
                   state=np.zeros(n, np.int8), cls=np.zeros(n, np.int32))
        v = _view(**arr)
        k = cr_counters()
        _chk(self._lib.cr_checkpoint(self._h, C.byref(v), C.byref(k)), "cr_checkpoint")
        arr.update(n=n, sweep=int(k.sweep), md_eval=int(k.md_eval), forces_valid=int(k.forces_valid))
        return arr

    def restore(self, ck):
        """cr_restore from a dict as checkpoint() returns it."""
        k = cr_counters(int(ck["sweep"]), int(ck["md_eval"]), int(ck["forces_valid"]))
        a = {x: np.ascontiguousarray(ck[x]) for x in ("xyz", "vel", "force", "id", "type", "cls", "state")}
        _chk(self._lib.cr_restore(self._h, int(ck["n"]), _p(a["xyz"]), _p(a["vel"]), _p(a["force"]), _p(a["id"]),
                                  _p(a["type"]), _p(a["cls"]), _p(a["state"]), C.byref(k)), "cr_restore")


class Batch:
    """Independent replicas advanced together (one phase launch per colour)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = C.c_void_p()
        _chk(_lib().cr_batch_create(C.byref(h), arr, len(self.contexts)), "cr_batch_create")
        self._h = h
        self._lib = _lib()
        for c in self.contexts:
            c._nbatch += 1

    def sweep(self, n_sweeps, seed):
        _chk(self._lib.cr_batch_sweep(self._h, int(n_sweeps), int(seed)), "cr_batch_sweep")

    def sweep_da(self, n_sweeps, seed):
        _chk(self._lib.cr_batch_sweep_da(self._h, int(n_sweeps), int(seed)), "cr_batch_sweep_da")

    def md_step(self, n_steps, dt, gamma, seed):
        _chk(self._lib.cr_batch_md_step(self._h, int(n_steps), float(dt), float(gamma), int(seed)), "cr_batch_md_step")

    def md_begin(self, dt, gamma, seed):
        _chk(self._lib.cr_batch_md_begin(self._h, float(dt), float(gamma), int(seed)), "cr_batch_md_begin")

    def load(self, loads):
        """cr_batch_load: one dict per replica with n and the arrays xyz, vel,
        type, cls, state (numpy arrays or raw pointers), as Context.load."""
        args = (cr_load_args * len(self.contexts))()
        conv = lambda a: None if a is None else (C.c_void_p(a) if isinstance(a, int) else _p(a))
        for r, a in enumerate(loads):
            args[r].n = int(a["n"])
            for k in ("xyz", "vel", "type", "cls", "state"):
                setattr(args[r], k, conv(a.get(k)))
        _chk(self._lib.cr_batch_load(self._h, args), "cr_batch_load")

    @staticmethod
    def _packed(stride, arrays, n):
        conv = lambda a: None if a is None else (C.c_void_p(a) if isinstance(a, int) else _p(a))
        pk = cr_batch_packed()
        pk.stride = int(stride)
        for k in ("xyz", "vel", "id", "type", "cls", "state"):
            setattr(pk, k, conv(arrays.get(k)))
        pk.n = conv(n)
        return pk

    def state_packed(self, stride, arrays, n):
        """cr_batch_state_packed: arrays (numpy arrays or raw pointers) hold all
        replicas, replica r from r * stride; n (int64 [replicas], numpy array
        or pointer) receives the particle counts."""
        pk = self._packed(stride, arrays, n)
        _chk(self._lib.cr_batch_state_packed(self._h, C.byref(pk)), "cr_batch_state_packed")

    def load_packed(self, stride, arrays, n):
        """cr_batch_load_packed: every replica from packed arrays (xyz, vel, type,
        cls, state), n (int64 [replicas]) particles each."""
        pk = self._packed(stride, arrays, n)
        _chk(self._lib.cr_batch_load_packed(self._h, C.byref(pk)), "cr_batch_load_packed")

    def state_into(self, arrays):
        """cr_batch_state: one dict of caller arrays (as Context.state_into
        takes them) per replica; returns the counts of every replica."""
        views = (cr_state_view * len(self.contexts))()
        for r, a in enumerate(arrays):
            views[r] = _view(**a)
        _chk(self._lib.cr_batch_state(self._h, views), "cr_batch_state")
        return [_view_counts(views[r]) for r in range(len(self.contexts))]

    def md_end(self, dt, gamma, seed):
        _chk(self._lib.cr_batch_md_end(self._h, float(dt), float(gamma), int(seed)), "cr_batch_md_end")

    def cycle(self, n_steps, dt, gamma, sweep_seed0, md_seed0, da=False):
        """cr_batch_cycle: n_steps MD/CR-MC cycles (one CUDA graph launch per
        step once tuned); step s uses seeds sweep_seed0 + s and md_seed0 + s."""
        _chk(self._lib.cr_batch_cycle(self._h, int(n_steps), float(dt), float(gamma), int(sweep_seed0),
                                      int(md_seed0), 1 if da else 0), "cr_batch_cycle")

    def set_launch_shape(self, threads, regs):
        _chk(self._lib.cr_batch_set_launch_shape(self._h, int(threads), int(regs)), "cr_batch_set_launch_shape")

    def set_persistent(self, mode=1, ctas_per_sm=0):
        """cr_batch_set_persistent: mode 1 per-domain dependencies (default), 2
        per-colour ones, 0 (or False) one launch per colour."""
        _chk(self._lib.cr_batch_set_persistent(self._h, int(mode), int(ctas_per_sm)), "cr_batch_set_persistent")

    def selftest_wait_timeout(self, replica, timeout_ms):
        """cr_batch_selftest_wait_timeout: the status code (CR_ERR_TIMEOUT = -5
        when the bounded-wait path worked)."""
        return int(self._lib.cr_batch_selftest_wait_timeout(self._h, int(replica), float(timeout_ms)))

    def launch_shape(self):
        t = C.c_int32()
        r = C.c_int32()
        _chk(self._lib.cr_batch_get_launch_shape(self._h, C.byref(t), C.byref(r)), "cr_batch_get_launch_shape")
        return t.value, r.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cr_batch_destroy(self._h)
            self._h = None
            for c in self.contexts:
                c._nbatch -= 1

    def __del__(self):
        self.close()


def _mlp_struct(mlp):
    k = {n: np.ascontiguousarray(mlp[n], dtype=np.uint16) for n in ("W1", "W2", "W3", "w4")}
    k.update({n: np.ascontiguousarray(mlp[n], dtype=np.float32) for n in ("b1", "b2", "b3")})
    m = cr_mlp(_p(k["W1"]), _p(k["b1"]), _p(k["W2"]), _p(k["b2"]), _p(k["W3"]), _p(k["b3"]), _p(k["w4"]),
               float(mlp["b4"]))
    return m, k


class Trainer:
    """Surrogate training on the tensor cores (owns one cr_trainer).  Batches
    are device pointers (raw ints, e.g. torch tensors' data_ptr())."""

    def __init__(self, mlp, max_batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, target_clip=20.0, stream=None,
                 unfused=False):
        self._lib = _lib()
        m, keep = _mlp_struct(mlp)
        cfg = cr_train_cfg(int(max_batch), lr, beta1, beta2, eps, target_clip, 1 if unfused else 0)
        h = C.c_void_p()
        _chk(self._lib.cr_train_create(C.byref(h), C.byref(m), C.byref(cfg)), "cr_train_create")
        self._h = h
        st = stream if stream is not None else _torch_stream()
        if st is not None:
            _chk(self._lib.cr_train_set_stream(h, st), "cr_train_set_stream")

    def step(self, X_ptr, t_ptr, batch, want_loss=False):
        loss = C.c_float()
        _chk(self._lib.cr_train_step(self._h, C.c_void_p(int(X_ptr)), C.c_void_p(int(t_ptr)), int(batch),
                                     C.byref(loss) if want_loss else None), "cr_train_step")
        return loss.value if want_loss else None

    def gradients(self, X_ptr, t_ptr, batch):
        g = np.zeros(N_PARAMS, np.float32)
        loss = C.c_float()
        _chk(self._lib.cr_train_gradients(self._h, C.c_void_p(int(X_ptr)), C.c_void_p(int(t_ptr)), int(batch),
                                          _p(g), C.byref(loss)), "cr_train_gradients")
        return loss.value, g

    def apply(self, grads):
        """cr_train_apply: one Adam step with the given gradient vector."""
        g = np.ascontiguousarray(grads, dtype=np.float32)
        if g.shape != (N_PARAMS,):
            raise ValueError("gradient vector of CR_TRAIN_N_PARAMS floats expected")
        _chk(self._lib.cr_train_apply(self._h, _p(g)), "cr_train_apply")

    def moments(self):
        """(first, second) Adam moments, FP32 vectors in the parameter order."""
        m = np.zeros(N_PARAMS, np.float32)
        v = np.zeros(N_PARAMS, np.float32)
        _chk(self._lib.cr_train_moments(self._h, _p(m), _p(v)), "cr_train_moments")
        return m, v

    def get(self):
        """(FP32 master vector, surrogate dict in the cr_mlp layout)."""
        P = np.zeros(N_PARAMS, np.float32)
        out = dict(W1=np.zeros((128, 48), np.uint16), W2=np.zeros((128, 128), np.uint16),
                   W3=np.zeros((128, 128), np.uint16), w4=np.zeros(128, np.uint16), b1=np.zeros(128, np.float32),
                   b2=np.zeros(128, np.float32), b3=np.zeros(128, np.float32))
        b4 = C.c_float()
        _chk(self._lib.cr_train_get(self._h, _p(P), _p(out["W1"]), _p(out["b1"]), _p(out["W2"]), _p(out["b2"]),
                                    _p(out["W3"]), _p(out["b3"]), _p(out["w4"]), C.byref(b4)), "cr_train_get")
        out["b4"] = b4.value
        return P, out

    def stats(self):
        a, b = C.c_int64(), C.c_int64()
        _chk(self._lib.cr_train_stats(self._h, C.byref(a), C.byref(b)), "cr_train_stats")
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.cr_train_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


def selftest_mma_timeout(A_ptr, B_ptr, D_ptr, polls, stream=None):
    """cr_selftest_mma_timeout: the status code (CR_ERR_TIMEOUT = -5 when the
    bounded-wait expiry path worked)."""
    st = stream if stream is not None else _torch_stream()
    return int(_lib().cr_selftest_mma_timeout(C.c_void_p(int(A_ptr)), C.c_void_p(int(B_ptr)),
                                              C.c_void_p(int(D_ptr)), int(polls), st))


def mma_bf16(A_ptr, B_ptr, D_ptr, M, N, K, accumulate=False, stream=None):
    """D [M][N] = A [M][K] B [N][K]^T on the tensor cores (device pointers)."""
    st = stream if stream is not None else _torch_stream()
    _chk(_lib().cr_mma_bf16(C.c_void_p(int(A_ptr)), C.c_void_p(int(B_ptr)), C.c_void_p(int(D_ptr)), int(M), int(N),
                            int(K), 1 if accumulate else 0, st), "cr_mma_bf16")
