"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Functions keep the C names (``lbm_create``, ``lbm_step`` ...) and only marshal
arguments; every step of the method runs in the library's CUDA kernels.  The
:class:`Lattice` class wraps one context for convenience.  Importing this
module raises if ``liblbm.so`` has not been built (``build.py``); there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads as W

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "liblbm.so")

LBM_OK = 0
STATUS = {0: "LBM_OK", -1: "LBM_ERR_ARG", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA",
          -4: "LBM_ERR_UNSUPPORTED", -5: "LBM_ERR_STATE", -6: "LBM_ERR_TIMEOUT",
          -7: "LBM_ERR_DIVERGED", -8: "LBM_ERR_CAPACITY"}
D2Q9, D3Q19 = 0, 1
BGK, MRT = 0, 1
FP64, FP32, FP32_BF16STORE, FP32_FP16STORE = 0, 1, 2, 3
FORCE_FLUID_ONLY, FORCE_ALL = 0, 1
SPHERE, CYLINDER_Z = 0, 1
(SCHEME_NONE, BOUNCE_BACK, BOUZIDI_LIN, BOUZIDI_QUAD, YU_LIN, YU_QUAD,
 IBM_DIRECT, ZHAO_YONG) = range(8)
TK_BULK, TK_LIST, TK_IBM, TK_GEOM = range(4)
DELTA_PESKIN4, DELTA_ROMA3, DELTA_LINEAR2, DELTA_COSINE4 = range(4)
FACE_PERIODIC, FACE_VELOCITY, FACE_FREE_SLIP, FACE_CONVECTIVE = range(4)
INERTIA_FENG, INERTIA_KEMPE, INERTIA_UHLMANN = range(3)
# lbm_set_timing masks: every kind, or bit (kind + 1) per kind
TIME_ALL = 1
TIME_BULK, TIME_LIST, TIME_IBM, TIME_GEOM = (2 << k for k in range(4))


class lbm_lattice_desc(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("collision", C.c_int),
                ("mrt_rates", C.c_double * 19), ("precision", C.c_int),
                ("body_force", C.c_double * 3), ("force_region", C.c_int)]


class lbm_solid_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("centre", C.c_double * 3), ("radius", C.c_double),
                ("velocity", C.c_double * 3), ("omega", C.c_double * 3),
                ("fluid_inside", C.c_int)]


class lbm_scheme_desc(C.Structure):
    _fields_ = [("scheme", C.c_int), ("ibm_iters", C.c_int),
                ("ibm_retraction", C.c_double), ("ibm_marker_density", C.c_double),
                ("ibm_kernel", C.c_int), ("ibm_inertia", C.c_int)]


class lbm_request(C.Structure):
    _fields_ = [("lattice", lbm_lattice_desc), ("nsolids", C.c_int),
                ("solids", lbm_solid_desc * 8), ("scheme", lbm_scheme_desc),
                ("rho0", C.c_double), ("u0", C.c_double * 3), ("keep_velocity", C.c_int),
                ("deadline_s", C.c_double)]


class lbm_result(C.Structure):
    _fields_ = [("status", C.c_int), ("error", C.c_int), ("steps", C.c_int64),
                ("residual", C.c_double), ("force", C.c_double * 3), ("torque", C.c_double * 3),
                ("submit_s", C.c_double), ("start_s", C.c_double), ("finish_s", C.c_double),
                ("device_bytes", C.c_int64)]


REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED, REQ_UNCONVERGED = range(6)


class lbm_domain_desc(C.Structure):
    _fields_ = [("type", C.c_int * 6), ("u", (C.c_double * 3) * 6)]


class lbm_info(C.Structure):
    _fields_ = [("nodes", C.c_int64), ("fluid_nodes", C.c_int64),
                ("list_nodes", C.c_int64), ("cut_links", C.c_int64),
                ("markers", C.c_int64), ("steps", C.c_int64),
                ("kernel_launches", C.c_int64), ("device_bytes", C.c_int64),
                ("num_solids", C.c_int32), ("precision", C.c_int32),
                ("bulk_kernel", C.c_int32)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -m paper_1906_05445_gb300.build` (nvcc, sm_103a)")
    L = C.CDLL(_LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    dp = C.POINTER(C.c_double)
    st = C.c_int
    sigs = {
        "lbm_create": (st, [C.POINTER(vp), C.POINTER(lbm_lattice_desc), vp]),
        "lbm_destroy": (None, [vp]),
        "lbm_add_solid": (st, [vp, C.POINTER(lbm_solid_desc), C.POINTER(i)]),
        "lbm_set_solid_motion": (st, [vp, i, dp, dp, dp]),
        "lbm_set_scheme": (st, [vp, C.POINTER(lbm_scheme_desc)]),
        "lbm_init_equilibrium": (st, [vp, d, dp]),
        "lbm_set_distributions": (st, [vp, dp, sz]),
        "lbm_set_distributions_async": (st, [vp, dp, sz]),
        "lbm_get_distributions": (st, [vp, dp, sz]),
        "lbm_step": (st, [vp, i]),
        "lbm_run_to_steady": (st, [vp, d, i, i, C.POINTER(i), dp]),
        "lbm_get_density": (st, [vp, dp, sz]),
        "lbm_get_velocity": (st, [vp, dp, sz]),
        "lbm_get_velocity_async": (st, [vp, dp, sz]),
        "lbm_get_strain_rate": (st, [vp, dp, sz]),
        "lbm_get_stress": (st, [vp, dp, sz]),
        "lbm_get_dissipation": (st, [vp, dp, sz]),
        "lbm_get_solid_mask": (st, [vp, C.POINTER(C.c_ubyte), sz]),
        "lbm_get_force_torque": (st, [vp, i, dp, dp]),
        "lbm_get_force_history": (st, [vp, i, dp, sz, C.POINTER(sz)]),
        "lbm_copy_force_torque_async": (st, [vp, i, dp]),
        "lbm_set_solid_dynamics": (st, [vp, i, d, dp]),
        "lbm_set_domain": (st, [vp, C.POINTER(lbm_domain_desc)]),
        "lbm_step_multi": (st, [C.POINTER(vp), i, i]),
        "lbm_server_create": (st, [C.POINTER(vp), sz, d, i, i]),
        "lbm_server_submit": (st, [vp, C.POINTER(lbm_request), C.POINTER(C.c_int64)]),
        "lbm_server_poll": (st, [vp, C.c_int64, C.POINTER(lbm_result)]),
        "lbm_server_wait": (st, [vp, C.c_int64, C.POINTER(lbm_result), d]),
        "lbm_server_velocity": (st, [vp, C.c_int64, dp, sz]),
        "lbm_server_destroy": (None, [vp]),
        "lbm_server_cancel": (st, [vp, C.c_int64]),
        "lbm_debug_fail_allocations_after": (None, [C.c_longlong]),
        "lbm_get_solid_velocity": (st, [vp, i, dp, dp]),
        "lbm_get_residual": (st, [vp, dp]),
        "lbm_get_solid_centre": (st, [vp, i, dp]),
        "lbm_get_info": (st, [vp, C.POINTER(lbm_info)]),
        "lbm_device_field": (st, [vp, i, C.POINTER(vp), C.POINTER(sz), C.POINTER(sz)]),
        "lbm_save": (st, [vp, vp, C.POINTER(sz)]),
        "lbm_load": (st, [vp, vp, sz]),
        "lbm_set_timing": (st, [vp, i, i]),
        "lbm_get_kernel_time": (st, [vp, i, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "lbm_get_velocity_noalloc": (st, [vp, dp, sz]),
        "lbm_batch_create": (st, [C.POINTER(vp), C.POINTER(vp), i, vp, i]),
        "lbm_batch_destroy": (None, [vp]),
        "lbm_batch_step": (st, [vp, i]),
        "lbm_batch_run_to_steady": (st, [vp, d, i, i, C.POINTER(C.c_int64), dp]),
        "lbm_batch_info": (st, [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(C.c_int64)]),
        "lbm_batch_last_error": (C.c_char_p, [vp]),
        "lbm_sync": (st, [vp]),
        "lbm_last_error": (C.c_char_p, [vp]),
        "lbm_version": (C.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


lib = _load()
globals().update({name: getattr(lib, name) for name in (
    "lbm_create", "lbm_destroy", "lbm_add_solid", "lbm_set_solid_motion",
    "lbm_set_scheme", "lbm_init_equilibrium", "lbm_set_distributions",
    "lbm_set_distributions_async",
    "lbm_get_distributions", "lbm_step", "lbm_run_to_steady", "lbm_get_density",
    "lbm_get_velocity", "lbm_get_velocity_async", "lbm_get_strain_rate", "lbm_get_stress",
    "lbm_get_dissipation", "lbm_get_solid_mask", "lbm_get_force_torque", "lbm_get_force_history",
    "lbm_copy_force_torque_async", "lbm_set_solid_dynamics", "lbm_get_solid_velocity",
    "lbm_set_domain", "lbm_step_multi", "lbm_server_create", "lbm_server_submit",
    "lbm_server_poll", "lbm_server_wait", "lbm_server_velocity", "lbm_server_destroy",
    "lbm_server_cancel", "lbm_debug_fail_allocations_after",
    "lbm_get_residual", "lbm_get_solid_centre", "lbm_get_info",
    "lbm_device_field", "lbm_save", "lbm_load", "lbm_set_timing",
    "lbm_get_kernel_time", "lbm_get_velocity_noalloc", "lbm_sync", "lbm_last_error",
    "lbm_version", "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_step",
    "lbm_batch_run_to_steady", "lbm_batch_info", "lbm_batch_last_error")})


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _v3(v) -> np.ndarray:
    a = np.zeros(3)
    if v is not None:
        v = np.asarray(v, dtype=np.float64).ravel()
        a[:len(v)] = v
    return a


class Lattice:
    """One lattice context of the CUDA library."""

    def __init__(self, lattice: int, nx: int, ny: int, nz: int, tau: float,
                 collision: int = BGK, precision: int = FP32, g=None,
                 force_all: bool = False, rates: Optional[Sequence[float]] = None,
                 stream: Optional[int] = None):
        d = lbm_lattice_desc()
        d.lattice, d.nx, d.ny, d.nz = lattice, nx, ny, nz
        d.tau, d.collision, d.precision = tau, collision, precision
        if rates is not None:
            for k, r in enumerate(rates):
                d.mrt_rates[k] = r
        gv = _v3(g)
        for k in range(3):
            d.body_force[k] = gv[k]
        d.force_region = FORCE_ALL if force_all else FORCE_FLUID_ONLY
        self.h = C.c_void_p()
        self._check(lbm_create(C.byref(self.h), C.byref(d), C.c_void_p(stream or 0)))
        self.lattice = lattice
        self.Q = 9 if lattice == D2Q9 else 19
        self.d = 2 if lattice == D2Q9 else 3
        self.shape = (1 if lattice == D2Q9 else nz, ny, nx)
        self.N = int(np.prod(self.shape))

    @classmethod
    def from_problem(cls, p: W.Problem, stream: Optional[int] = None) -> "Lattice":
        lat = cls(p.lattice, p.nx, p.ny, p.nz, p.tau, p.collision, p.precision, p.g,
                  p.force_all, stream=stream)
        for s in p.solids:
            lat.add_solid(s.kind, s.centre, s.radius, s.velocity, s.omega, s.fluid_inside)
        lat.set_scheme(p.scheme, p.ibm_iters, p.retraction, p.marker_density, p.ibm_kernel,
                       p.ibm_inertia)
        if p.faces is not None:
            lat.set_domain(p.faces, p.u_face)
        return lat

    def _check(self, st: int):
        if st != LBM_OK:
            msg = lbm_last_error(self.h).decode() if getattr(self, "h", None) else ""
            raise LbmError(st, msg)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_solid(self, kind, centre, radius, velocity=None, omega=None,
                  fluid_inside=False) -> int:
        s = lbm_solid_desc()
        s.kind, s.radius, s.fluid_inside = kind, radius, int(fluid_inside)
        for k, (c, u, o) in enumerate(zip(_v3(centre), _v3(velocity), _v3(omega))):
            s.centre[k], s.velocity[k], s.omega[k] = c, u, o
        sid = C.c_int()
        self._check(lbm_add_solid(self.h, C.byref(s), C.byref(sid)))
        return sid.value

    def set_solid_motion(self, sid, centre=None, velocity=None, omega=None):
        args = [None if v is None else _v3(v) for v in (centre, velocity, omega)]
        self._check(lbm_set_solid_motion(self.h, sid, *[None if a is None else _dp(a) for a in args]))

    def set_scheme(self, scheme, ibm_iters=1, retraction=0.0, marker_density=1.0,
                   ibm_kernel=DELTA_PESKIN4, ibm_inertia=INERTIA_FENG):
        s = lbm_scheme_desc(scheme, ibm_iters, retraction, marker_density, ibm_kernel,
                            ibm_inertia)
        self._check(lbm_set_scheme(self.h, C.byref(s)))

    def init_equilibrium(self, rho=1.0, u=None):
        self._check(lbm_init_equilibrium(self.h, rho, _dp(_v3(u))))

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        self._check(lbm_set_distributions(self.h, _dp(f), f.size))

    def set_f_async(self, f):
        """Upload without waiting.  `f` (C-contiguous float64, best
        page-locked) must stay alive and unchanged until sync() or a query."""
        if f.dtype != np.float64 or not f.flags.c_contiguous:
            raise ValueError("f must be C-contiguous float64")
        self._check(lbm_set_distributions_async(self.h, _dp(f), f.size))

    def get_f(self):
        out = np.zeros((self.Q, self.N))
        self._check(lbm_get_distributions(self.h, _dp(out), out.size))
        return out.reshape((self.Q,) + self.shape)

    def step(self, n=1):
        self._check(lbm_step(self.h, int(n)))

    def run_to_steady(self, tol, check_every=100, max_steps=100000):
        done, r = C.c_int(), C.c_double()
        self._check(lbm_run_to_steady(self.h, tol, check_every, max_steps,
                                      C.byref(done), C.byref(r)))
        return done.value, r.value

    def _field(self, fn, comps, out=None):
        """The field into a new array, or into `out` (C-contiguous float64 of
        comps * nodes values, e.g. page-locked memory for a faster copy)."""
        if out is None:
            out = np.zeros((comps, self.N))
        elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size < comps * self.N:
            raise ValueError(f"out must be C-contiguous float64 with {comps * self.N} values")
        self._check(fn(self.h, _dp(out), out.size))
        return out.reshape((comps,) + self.shape)

    def density(self):
        return self._field(lbm_get_density, 1)[0]

    def velocity(self, out=None):
        return self._field(lbm_get_velocity, self.d, out)

    def velocity_async(self, out):
        """Enqueue the velocity query and its copy into `out` (C-contiguous
        float64, page-locked for an asynchronous copy) and return; `sync()`
        waits for it."""
        return self._field(lbm_get_velocity_async, self.d, out)

    def strain_rate(self):
        return self._field(lbm_get_strain_rate, 3 if self.d == 2 else 6)

    def stress(self):
        return self._field(lbm_get_stress, 3 if self.d == 2 else 6)

    def dissipation(self):
        return self._field(lbm_get_dissipation, 1)[0]

    def solid_mask(self):
        m = np.zeros(self.N, dtype=np.uint8)
        self._check(lbm_get_solid_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte)), m.size))
        return m.reshape(self.shape).astype(bool)

    def force_torque(self, sid=0):
        F, T = np.zeros(3), np.zeros(3)
        self._check(lbm_get_force_torque(self.h, sid, _dp(F), _dp(T)))
        return F, T

    def copy_force_torque_async(self, out, sid=0):
        """Enqueue the copy of the current (Fx Fy Fz Tx Ty Tz) into `out`, a
        float64 array of 6 (page-locked for the copy to be asynchronous);
        valid after sync()."""
        assert out.dtype == np.float64 and out.size >= 6 and out.flags.c_contiguous
        self._check(lbm_copy_force_torque_async(self.h, sid, _dp(out)))

    def force_history(self, sid=0, max_steps=4096):
        out = np.zeros((max_steps, 6))
        n = C.c_size_t()
        self._check(lbm_get_force_history(self.h, sid, _dp(out), max_steps, C.byref(n)))
        return out[:n.value]

    def solid_centre(self, sid=0):
        c = np.zeros(3)
        self._check(lbm_get_solid_centre(self.h, sid, _dp(c)))
        return c

    def set_domain(self, faces=None, u_face=None):
        """Face types x-, x+, y-, y+, z-, z+ (FACE_*) and the [6][3] wall
        velocities of the velocity faces; None restores the periodic box."""
        if faces is None:
            self._check(lbm_set_domain(self.h, None))
            return
        d = lbm_domain_desc()
        u = np.zeros((6, 3)) if u_face is None else np.asarray(u_face, dtype=np.float64)
        for k in range(6):
            d.type[k] = int(faces[k])
            for c in range(3):
                d.u[k][c] = float(u[k][c])
        self._check(lbm_set_domain(self.h, C.byref(d)))

    def set_solid_dynamics(self, sid, density_ratio, gravity=None):
        self._check(lbm_set_solid_dynamics(self.h, sid, float(density_ratio),
                                           _dp(_v3(gravity))))

    def solid_velocity(self, sid=0):
        U, Om = np.zeros(3), np.zeros(3)
        self._check(lbm_get_solid_velocity(self.h, sid, _dp(U), _dp(Om)))
        return U, Om

    def info(self) -> lbm_info:
        i = lbm_info()
        self._check(lbm_get_info(self.h, C.byref(i)))
        return i

    def save(self) -> bytes:
        n = C.c_size_t()
        self._check(lbm_save(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(lbm_save(self.h, C.cast(buf, C.c_void_p), C.byref(n)))
        return buf.raw[:n.value]

    def load(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        self._check(lbm_load(self.h, C.cast(buf, C.c_void_p), len(data)))

    def set_timing(self, on=True, every=1):
        """on: False, True (every kind) or a TIME_* mask; every: time only
        the launches of every n-th step."""
        self._check(lbm_set_timing(self.h, int(on), int(every)))

    def kernel_time(self, kernel=TK_BULK):
        ms, nl, nn = C.c_double(), C.c_int64(), C.c_int64()
        self._check(lbm_get_kernel_time(self.h, kernel, C.byref(ms), C.byref(nl), C.byref(nn)))
        return ms.value, nl.value, nn.value

    def sync(self):
        self._check(lbm_sync(self.h))


def step_multi(lattices: Sequence["Lattice"], nsteps: int = 1):
    """Advance distinct lattices together; their bulk sweeps run as grouped
    launches (lbm_step_multi)."""
    arr = (C.c_void_p * len(lattices))(*[lt.h.value for lt in lattices])
    st = lbm_step_multi(arr, len(lattices), int(nsteps))
    if st != LBM_OK:
        msg = "; ".join(m for m in (lbm_last_error(lt.h).decode() for lt in lattices) if m)
        raise LbmError(st, msg)


class Batch:
    """Several lattices advanced together (one CUDA graph launch per step
    pair, per-lattice residual checks); see lbm_batch_create."""

    def __init__(self, lattices: Sequence[Lattice], stream: Optional[int] = None,
                 autotune: bool = True):
        self.lattices = list(lattices)
        arr = (C.c_void_p * len(self.lattices))(*[lt.h.value for lt in self.lattices])
        self.h = C.c_void_p()
        st = lbm_batch_create(C.byref(self.h), arr, len(self.lattices),
                              C.c_void_p(stream or 0), int(autotune))
        if st != LBM_OK:
            raise LbmError(st, "lbm_batch_create failed")

    def _check(self, st: int):
        if st != LBM_OK:
            raise LbmError(st, lbm_batch_last_error(self.h).decode())

    def step(self, n=1):
        self._check(lbm_batch_step(self.h, int(n)))

    def run_to_steady(self, tol, check_every=100, max_steps=100000):
        n = len(self.lattices)
        steps = (C.c_int64 * n)()
        res = np.zeros(n)
        self._check(lbm_batch_run_to_steady(self.h, tol, check_every, max_steps, steps,
                                            _dp(res)))
        return np.array(list(steps), dtype=np.int64), res

    def info(self, i=0):
        bb, lb, gl = C.c_int(), C.c_int(), C.c_int64()
        self._check(lbm_batch_info(self.h, i, C.byref(bb), C.byref(lb), C.byref(gl)))
        return bb.value, lb.value, gl.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_of(p: W.Problem, u0=None, keep_velocity: bool = False,
               deadline: float = 0.0) -> lbm_request:
    """The lbm_request of a workload problem (periodic domain, started at the
    equilibrium at rest or at u0)."""
    r = lbm_request()
    d = r.lattice
    d.lattice, d.nx, d.ny, d.nz = p.lattice, p.nx, p.ny, p.nz
    d.tau, d.collision, d.precision = p.tau, p.collision, p.precision
    for k, v in enumerate(_v3(p.g)):
        d.body_force[k] = v
    d.force_region = 1 if p.force_all else 0
    if len(p.solids) > 8:
        raise ValueError("at most 8 solids")
    r.nsolids = len(p.solids)
    for k, b in enumerate(p.solids):
        sd = r.solids[k]
        sd.kind, sd.radius, sd.fluid_inside = b.kind, b.radius, int(b.fluid_inside)
        for a, (c, u, o) in enumerate(zip(_v3(b.centre), _v3(b.velocity), _v3(b.omega))):
            sd.centre[a], sd.velocity[a], sd.omega[a] = c, u, o
    r.scheme = lbm_scheme_desc(p.scheme, p.ibm_iters, p.retraction, p.marker_density,
                               p.ibm_kernel, p.ibm_inertia)
    r.rho0 = 1.0
    for k, v in enumerate(_v3(u0)):
        r.u0[k] = v
    r.keep_velocity = int(keep_velocity)
    r.deadline_s = float(deadline)
    return r


class Server:
    """The library's serving engine (lbm_server_*): solves are admitted by
    device-memory footprint and stepped together under continuous batching by
    a worker thread of the library."""

    def __init__(self, hbm_budget: int, tol: float, check_every: int = 200,
                 max_steps: int = 200000):
        self.h = C.c_void_p()
        st = lbm_server_create(C.byref(self.h), int(hbm_budget), float(tol), int(check_every),
                               int(max_steps))
        if st != LBM_OK:
            raise LbmError(st, "lbm_server_create failed")

    def submit(self, p: W.Problem, u0=None, keep_velocity: bool = False,
               deadline: float = 0.0) -> int:
        i = C.c_int64()
        st = lbm_server_submit(self.h, C.byref(request_of(p, u0, keep_velocity, deadline)),
                               C.byref(i))
        if st != LBM_OK:
            raise LbmError(st, f"lbm_server_submit refused {p.name}")
        return i.value

    @staticmethod
    def _dict(r: lbm_result) -> dict:
        return {"status": r.status, "error": r.error, "steps": r.steps, "residual": r.residual,
                "force": np.array(r.force[:]), "torque": np.array(r.torque[:]),
                "submit_s": r.submit_s, "start_s": r.start_s, "finish_s": r.finish_s,
                "device_bytes": r.device_bytes}

    def poll(self, rid: int) -> dict:
        r = lbm_result()
        st = lbm_server_poll(self.h, rid, C.byref(r))
        if st != LBM_OK:
            raise LbmError(st, f"unknown request {rid}")
        return self._dict(r)

    def wait(self, rid: int, timeout: float = -1.0) -> dict:
        r = lbm_result()
        st = lbm_server_wait(self.h, rid, C.byref(r), float(timeout))
        if st != LBM_OK:
            raise LbmError(st, f"request {rid}")
        return self._dict(r)

    def velocity(self, rid: int, p: W.Problem) -> np.ndarray:
        d = 2 if p.lattice == D2Q9 else 3
        shape = (p.nz if p.lattice == D3Q19 else 1, p.ny, p.nx)
        out = np.zeros((d,) + shape)
        st = lbm_server_velocity(self.h, rid, _dp(out), out.size)
        if st != LBM_OK:
            raise LbmError(st, f"no velocity kept for request {rid}")
        return out

    def cancel(self, rid: int):
        st = lbm_server_cancel(self.h, rid)
        if st != LBM_OK:
            raise LbmError(st, f"request {rid} cannot be cancelled")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_fail_allocations_after(n: int):
    """Fault injection: the next n device allocations succeed, later ones fail
    with LBM_ERR_OOM; n < 0 turns the hook off."""
    lbm_debug_fail_allocations_after(int(n))
