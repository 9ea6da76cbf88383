"""ctypes binding of libmm (include/mm.h): argument marshalling only.

Every function of the C ABI is exposed under its own name (mm_create, ...)
on the object returned by `lib()`; `Context` wraps them for numpy arrays
(host buffers, double) and torch CUDA tensors (device buffers in the
context precision).  All arithmetic runs in libmm's CUDA kernels: there is
no CPU path, and a missing libmm.so raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmm.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA, MM_ENAN, MM_ESTEP, MM_ETIMEOUT, MM_EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
MM_F64, MM_F32, MM_F64_NATIVE = 0, 1, 2
PRECISIONS = {"f64": MM_F64, "f32": MM_F32, "f64_native": MM_F64_NATIVE}
MM_HOST, MM_DEVICE = 0, 1
MM_ATTEMPT_AUTO, MM_ATTEMPT_PASSES = 0, 1
ENERGY_TERMS = ("exchange", "dmi", "uniaxial", "cubic", "zeeman", "demag", "total")


class mm_mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double)]


class mm_material(C.Structure):
    _fields_ = [("Ms", C.c_double), ("A", C.c_double), ("D", C.c_double), ("dmi_kind", C.c_int),
                ("Ku", C.c_double), ("u", C.c_double * 3), ("Kc", C.c_double), ("H", C.c_double * 3),
                ("alpha", C.c_double), ("gamma", C.c_double), ("precession", C.c_int), ("demag", C.c_int)]


class mm_checkpoint(C.Structure):
    _fields_ = [("t", C.c_double), ("h", C.c_double), ("t_end", C.c_double), ("rtol", C.c_double),
                ("max_dmdt", C.c_double), ("n_accepted", C.c_longlong), ("n_rejected", C.c_longlong),
                ("status", C.c_int), ("pad", C.c_int)]


class mm_status(C.Structure):
    _fields_ = [("t", C.c_double), ("h", C.c_double), ("err", C.c_double), ("max_dmdt", C.c_double),
                ("n_accepted", C.c_longlong), ("n_rejected", C.c_longlong), ("status", C.c_int),
                ("pad", C.c_int)]


class mm_tuning(C.Structure):
    _fields_ = [("Ty", C.c_int), ("Rx", C.c_int), ("x_threads", C.c_int), ("col_threads", C.c_int),
                ("col_group", C.c_int), ("col_occ", C.c_int), ("x_stage", C.c_int)]


TUNING_FIELDS = ("Ty", "Rx", "x_threads", "col_threads", "col_group", "col_occ", "x_stage")

_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "mm_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, _P]),
    "mm_destroy": (C.c_int, [_P]),
    "mm_last_error": (C.c_char_p, [_P]),
    "mm_add_sim": (C.c_int, [_P, C.POINTER(mm_mesh), C.POINTER(mm_material), _D, C.POINTER(C.c_int)]),
    "mm_batch_layout": (C.c_int, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "mm_num_sims": (C.c_int, [_P]),
    "mm_set_field": (C.c_int, [_P, C.c_int, _D]),
    "mm_precompute_demag": (C.c_int, [_P]),
    "mm_newell_tensor": (C.c_int, [_P, C.c_int, _D]),
    "mm_set_m": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "mm_get_m": (C.c_int, [_P, C.c_int, _P, C.c_int]),
    "mm_rhs_eval": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mm_rhs_eval_host": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "mm_rk45_setup": (C.c_int, [_P, C.c_double, C.c_double, C.c_double]),
    "mm_rk45_attempts": (C.c_int, [_P, C.c_int]),
    "mm_rk45_step": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mm_relax": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_longlong, C.c_int,
                           C.POINTER(C.c_longlong)]),
    "mm_get_status": (C.c_int, [_P, C.c_int, C.POINTER(mm_status)]),
    "mm_reset_time": (C.c_int, [_P]),
    "mm_energy": (C.c_int, [_P, C.c_int, _D]),
    "mm_neb_setup": (C.c_int, [_P, C.c_int, C.c_int, C.c_double]),
    "mm_neb_relax": (C.c_int, [_P, C.c_double, C.c_longlong, _D]),
    "mm_minimize": (C.c_int, [_P, C.c_double, C.c_longlong, C.c_int, C.POINTER(C.c_longlong),
                              C.POINTER(C.c_int)]),
    "mm_minimize_info": (C.c_int, [_P, C.c_int, C.POINTER(C.c_longlong), _D, _D, C.POINTER(C.c_int)]),
    "mm_rk4": (C.c_int, [_P, C.c_double, C.c_longlong, C.c_int]),
    "mm_set_cell_params": (C.c_int, [_P, C.c_int, _D, _D]),
    "mm_get_checkpoint": (C.c_int, [_P, C.c_int, C.POINTER(mm_checkpoint)]),
    "mm_set_checkpoint": (C.c_int, [_P, C.c_int, C.POINTER(mm_checkpoint)]),
    "mm_set_spin_torque": (C.c_int, [_P, C.c_int, _D, C.c_double, C.c_double, C.c_double, _D]),
    "mm_profile_attempts": (C.c_int, [_P, C.c_int, _D, C.POINTER(C.c_longlong)]),
    "mm_debug_bounded_wait": (C.c_int, [_P, C.c_longlong]),
    "mm_kernel_launches": (C.c_longlong, [_P]),
    "mm_rhs_eval_static": (C.c_int, [C.POINTER(mm_mesh), C.POINTER(mm_material), C.c_int, _P, _P, _P, _P]),
    "mm_set_tuning": (C.c_int, [_P, C.c_int, C.POINTER(mm_tuning)]),
    "mm_get_tuning": (C.c_int, [_P, C.c_int, C.POINTER(mm_tuning)]),
    "mm_autotune": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(mm_tuning), _D, _D]),
    "mm_set_attempt_kernel": (C.c_int, [_P, C.c_int]),
    "mm_demag_potential": (C.c_int, [_P, C.c_int, _P, _P]),
    "mm_get_attempt_kernel": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
}

_lib = None


def lib():
    """Load libmm.so (built by paper_2406_16064_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmm.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                               "-- there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class MMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libmm error {code}: {msg}")
        self.code = code


def _dptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Context:
    """One libmm context: a batch of simulations on one GPU."""

    def __init__(self, precision="f64", device=0, stream=None):
        self.L = lib()
        self.precision = precision
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        # f64: FP64 state, double-float transforms; f64_native: FP64 arithmetic throughout
        self.dtype = np.float32 if precision == "f32" else np.float64
        h = _P()
        rc = self.L.mm_create(C.byref(h), device, PRECISIONS[precision],
                              _P(stream) if stream else None)
        if rc != MM_OK:
            raise MMError(rc, self.L.mm_last_error(None).decode())
        self.h = h
        self.sims = []

    def _check(self, rc):
        if rc != MM_OK:
            raise MMError(rc, self.L.mm_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.mm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- setup
    def add_sim(self, mesh, mat, Ms_cells=None):
        m = mm_mesh(mesh.nx, mesh.ny, mesh.nz, mesh.dx, mesh.dy, mesh.dz)
        t = mm_material()
        t.Ms, t.A, t.D, t.dmi_kind = mat.Ms, mat.A, mat.D, int(mat.dmi)
        t.Ku, t.Kc = mat.Ku, mat.Kc
        for i in range(3):
            t.u[i] = float(mat.u[i])
            t.H[i] = float(mat.H[i])
        t.alpha, t.gamma = mat.alpha, mat.gamma
        t.precession, t.demag = int(mat.precession), int(mat.demag)
        ms = None if Ms_cells is None else np.ascontiguousarray(Ms_cells, dtype=np.float64).ravel()
        sid = C.c_int()
        self._check(self.L.mm_add_sim(self.h, C.byref(m), C.byref(t), _dptr(ms), C.byref(sid)))
        self.sims.append((mesh.nx * mesh.ny * mesh.nz))
        Ac, Dc = getattr(mat, "A_cells", None), getattr(mat, "D_cells", None)
        if Ac is not None or Dc is not None:
            self.set_cell_params(sid.value, Ac, Dc)
        u = tuple(getattr(mat, "u_stt", (0.0, 0.0, 0.0)))
        aJ, bJ = getattr(mat, "aJ", 0.0), getattr(mat, "bJ", 0.0)
        if any(v != 0.0 for v in u) or aJ != 0.0 or bJ != 0.0:
            self.set_spin_torque(sid.value, u, getattr(mat, "beta", 0.0), aJ, bJ, getattr(mat, "p", (0.0, 0.0, 1.0)))
        return sid.value

    def set_cell_params(self, sim, A_cells=None, D_cells=None):
        """Per-cell exchange / DMI constants (arrays of nz*ny*nx values, None = uniform)."""
        a = None if A_cells is None else np.ascontiguousarray(A_cells, dtype=np.float64).ravel()
        d = None if D_cells is None else np.ascontiguousarray(D_cells, dtype=np.float64).ravel()
        n = self.sims[sim]
        assert (a is None or a.size == n) and (d is None or d.size == n)
        self._check(self.L.mm_set_cell_params(self.h, sim, _dptr(a), _dptr(d)))

    def set_spin_torque(self, sim, u=(0.0, 0.0, 0.0), beta=0.0, aJ=0.0, bJ=0.0, p=(0.0, 0.0, 1.0)):
        """Zhang-Li (u in m/s, beta) and Slonczewski / spin-orbit (a_J, b_J in 1/s, p) torques."""
        uu = np.ascontiguousarray(u, dtype=np.float64)
        pp = np.ascontiguousarray(p, dtype=np.float64)
        self._check(self.L.mm_set_spin_torque(self.h, sim, _dptr(uu), float(beta), float(aJ), float(bJ), _dptr(pp)))

    def precompute(self):
        self._check(self.L.mm_precompute_demag(self.h))

    # ---- tile shapes and schedules (mm_tuning; 0 = the library's rule)
    def set_tuning(self, sim, tuning):
        t = mm_tuning(*(int(tuning.get(k, 0)) for k in TUNING_FIELDS))
        self._check(self.L.mm_set_tuning(self.h, sim, C.byref(t)))

    def get_tuning(self, sim):
        t = mm_tuning()
        self._check(self.L.mm_get_tuning(self.h, sim, C.byref(t)))
        return {k: getattr(t, k) for k in TUNING_FIELDS}

    def autotune(self, sim, reps=8):
        """Time candidate tunings of sim's mesh (mm_autotune) and set the fastest on every
        simulation with that mesh; returns (tuning, ms per attempt, rule ms per attempt)."""
        t = mm_tuning()
        best, rule = C.c_double(), C.c_double()
        self._check(self.L.mm_autotune(self.h, sim, reps, C.byref(t), C.byref(best), C.byref(rule)))
        return {k: getattr(t, k) for k in TUNING_FIELDS}, best.value, rule.value

    def layout(self):
        n = len(self.sims)
        offs = (C.c_longlong * max(n, 1))()
        tot = C.c_longlong()
        self._check(self.L.mm_batch_layout(self.h, offs, C.byref(tot)))
        return [offs[i] for i in range(n)], tot.value

    def set_field(self, sim, H):
        h = np.ascontiguousarray(H, dtype=np.float64)
        self._check(self.L.mm_set_field(self.h, sim, _dptr(h)))

    def newell_tensor(self, sim, mesh):
        out = np.empty((6, 2 * mesh.nz - 1, 2 * mesh.ny - 1, 2 * mesh.nx - 1))
        self._check(self.L.mm_newell_tensor(self.h, sim, _dptr(out)))
        return out

    def _count(self, sim):
        return self.layout()[1] if sim < 0 else 3 * self.sims[sim]

    # ---- state
    def set_m(self, m, sim=-1):
        if _is_torch(m):
            self._check(self.L.mm_set_m(self.h, sim, _P(m.data_ptr()), MM_DEVICE))
        else:
            a = np.ascontiguousarray(m, dtype=np.float64).ravel()
            assert a.size == self._count(sim)
            self._check(self.L.mm_set_m(self.h, sim, a.ctypes.data_as(_P), MM_HOST))

    def get_m(self, sim=-1, out=None):
        """The state as host doubles: into `out` (a contiguous float64 array of the right
        size, for example a page-locked one) or a new array."""
        if out is None:
            out = np.empty(self._count(sim))
        assert out.dtype == np.float64 and out.flags["C_CONTIGUOUS"] and out.size == self._count(sim)
        self._check(self.L.mm_get_m(self.h, sim, out.ctypes.data_as(_P), MM_HOST))
        return out

    # ---- right-hand side
    def rhs_host(self, m, sim=-1, want_heff=True):
        a = np.ascontiguousarray(m, dtype=np.float64).ravel()
        assert a.size == self._count(sim)
        dmdt = np.empty_like(a)
        heff = np.empty_like(a) if want_heff else None
        self._check(self.L.mm_rhs_eval_host(self.h, sim, _dptr(a), _dptr(dmdt), _dptr(heff)))
        return dmdt, heff

    def rhs_device(self, m, dmdt, heff=None, sim=-1):
        self._check(self.L.mm_rhs_eval(self.h, sim, _P(m.data_ptr()), _P(dmdt.data_ptr()),
                                       _P(heff.data_ptr()) if heff is not None else None))

    def demag_potential(self, m, hd, sim):
        """Scalar-potential demag field of simulation sim: torch CUDA tensors m (in) and hd
        (out), [3][N] in the context precision."""
        self._check(self.L.mm_demag_potential(self.h, sim, _P(m.data_ptr()), _P(hd.data_ptr())))

    # ---- integration
    def set_attempt_kernel(self, passes=False, cluster=0):
        """passes=True: every RK45 attempt runs the pass kernels; False: the library's rule
        (one launch per call for small single-plane meshes), on `cluster` CTAs per
        simulation (2, 4, 8 or 16; 0 = the largest the device co-schedules)."""
        kind = MM_ATTEMPT_PASSES if passes else (cluster if cluster else MM_ATTEMPT_AUTO)
        self._check(self.L.mm_set_attempt_kernel(self.h, kind))

    def attempt_kernel(self):
        """(single_launch, cluster CTAs per simulation) of the next attempt."""
        one, nc = C.c_int(), C.c_int()
        self._check(self.L.mm_get_attempt_kernel(self.h, C.byref(one), C.byref(nc)))
        return bool(one.value), nc.value

    def rk45_setup(self, rtol, t_end=0.0, max_dmdt=0.0):
        self._check(self.L.mm_rk45_setup(self.h, rtol, t_end, max_dmdt))

    def rk45_attempts(self, n):
        self._check(self.L.mm_rk45_attempts(self.h, n))

    def rk45_step(self):
        a, r = C.c_int(), C.c_int()
        self._check(self.L.mm_rk45_step(self.h, C.byref(a), C.byref(r)))
        return a.value, r.value

    def relax(self, rtol, t_end=0.0, max_dmdt=0.0, max_steps=10 ** 9, sync_every=16):
        done = C.c_longlong()
        self._check(self.L.mm_relax(self.h, rtol, t_end, max_dmdt, max_steps, sync_every, C.byref(done)))
        return done.value

    def reset_time(self):
        self._check(self.L.mm_reset_time(self.h))

    def status(self, sim):
        s = mm_status()
        self._check(self.L.mm_get_status(self.h, sim, C.byref(s)))
        return {k: getattr(s, k) for k, _ in mm_status._fields_ if k != "pad"}

    def checkpoint(self, sim):
        """Integrator state of one simulation (t, h, t_end, rtol, max_dmdt, counters, status)."""
        c = mm_checkpoint()
        self._check(self.L.mm_get_checkpoint(self.h, sim, C.byref(c)))
        return {k: getattr(c, k) for k, _ in mm_checkpoint._fields_ if k != "pad"}

    def restore(self, sim, ckpt):
        """Set the integrator state of one simulation from checkpoint()'s dict."""
        c = mm_checkpoint(**{k: ckpt[k] for k, _ in mm_checkpoint._fields_ if k != "pad"})
        self._check(self.L.mm_set_checkpoint(self.h, sim, C.byref(c)))

    def energy(self, sim):
        E = np.zeros(7)
        self._check(self.L.mm_energy(self.h, sim, _dptr(E)))
        return dict(zip(ENERGY_TERMS, E))

    # ---- steepest descent
    def minimize(self, max_dmdt, max_steps=10 ** 6, sync_every=32):
        """Steepest descent with Barzilai-Borwein steps; returns (steps, converged)."""
        done = C.c_longlong()
        conv = C.c_int()
        self._check(self.L.mm_minimize(self.h, max_dmdt, max_steps, sync_every, C.byref(done), C.byref(conv)))
        return done.value, bool(conv.value)

    def minimize_info(self, sim):
        k, st = C.c_longlong(), C.c_int()
        tau, mx = C.c_double(), C.c_double()
        self._check(self.L.mm_minimize_info(self.h, sim, C.byref(k), C.byref(tau), C.byref(mx), C.byref(st)))
        return {"steps": k.value, "tau": tau.value, "max_dmdt": mx.value, "status": st.value}

    def rk4(self, h, n_steps, cayley=True):
        """n_steps fixed classical RK4 steps of size h on the Cayley variable
        (cayley=True) or on dm/dt with projection onto |m| = 1."""
        self._check(self.L.mm_rk4(self.h, float(h), int(n_steps), 1 if cayley else 0))

    # ---- NEB
    def neb_setup(self, first, n, k_spring):
        self._check(self.L.mm_neb_setup(self.h, first, n, k_spring))

    def neb_relax(self, rtol, n_steps):
        E = np.zeros(len(self.sims))
        self._check(self.L.mm_neb_relax(self.h, rtol, n_steps, _dptr(E)))
        return E

    # ---- misc
    KINDS = ("x_forward", "y_forward", "z_fused", "y_inverse", "y_fused", "x_inverse_epilogue",
             "control", "project", "neb", "yz_cluster")

    def profile_attempts(self, reps):
        ms = np.zeros(10)
        cnt = (C.c_longlong * 10)()
        self._check(self.L.mm_profile_attempts(self.h, reps, _dptr(ms), cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KINDS)}

    def bounded_wait(self, spins):
        return self.L.mm_debug_bounded_wait(self.h, spins)

    def launches(self):
        return int(self.L.mm_kernel_launches(self.h))
