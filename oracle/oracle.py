"""ctypes binding of the FP64 C oracle (test infrastructure only).

The C source is ``lbm_oracle.c`` in this directory; ``build()`` compiles it
with gcc into ``oracle/_build/liblbm_oracle.so``.  Arrays cross the boundary as
contiguous float64 numpy arrays in the interface layout [component][z][y][x].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liblbm_oracle.so")

D2Q9, D3Q19 = 0, 1
BGK, MRT = 0, 1
SPHERE, CYLINDER_Z = 0, 1
NONE, BB, BOUZIDI_LIN, BOUZIDI_QUAD, YU_LIN, YU_QUAD, IBM = range(7)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, single thread) if it is stale."""
    src = os.path.join(HERE, "lbm_oracle.c")
    hdr = os.path.join(HERE, "lbm_oracle.h")
    os.makedirs(BUILD_DIR, exist_ok=True)
    stale = force or not os.path.exists(LIB_PATH) or max(
        os.path.getmtime(src), os.path.getmtime(hdr)) > os.path.getmtime(LIB_PATH)
    if stale:
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, vp = C.c_double, C.c_int, C.c_void_p
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            sig = {
                "ora_q": (i, [i]),
                "ora_lattice": (None, [i, ip, dp]),
                "ora_mrt_matrix": (None, [i, dp]),
                "ora_mrt_default_rates": (None, [i, d, dp]),
                "ora_equilibrium": (None, [i, d, dp, dp]),
                "ora_collide": (None, [i, i, d, dp, dp, dp, dp]),
                "ora_ibb_coeffs": (i, [i, d, i, i, dp]),
                "ora_phi": (d, [d]),
                "ora_phi_kernel": (d, [i, d]),
                "ora_set_ibm_kernel": (None, [vp, i]),
                "ora_set_ibm_inertia": (None, [vp, i]),
                "ora_cell_fraction": (d, [vp, i, C.c_long, C.c_long, C.c_long]),
                "ora_internal_fluid": (None, [vp, i, dp]),
                "ora_set_solid_dynamics": (None, [vp, i, d, dp]),
                "ora_solid_velocity": (None, [vp, i, dp, dp]),
                "ora_set_domain": (i, [vp, C.POINTER(C.c_int), dp]),
                "ora_dissipation": (None, [vp, dp]),
                "ora_stress": (None, [vp, dp]),
                "ora_create": (vp, [i, i, i, i, d, i, dp, dp, i]),
                "ora_destroy": (None, [vp]),
                "ora_add_solid": (i, [vp, i, dp, d, dp, dp, i]),
                "ora_set_scheme": (None, [vp, i, i, d, d]),
                "ora_init_equilibrium": (None, [vp, d, dp]),
                "ora_set_f": (None, [vp, dp]),
                "ora_get_f": (None, [vp, dp]),
                "ora_step": (None, [vp, i]),
                "ora_density": (None, [vp, dp]),
                "ora_velocity": (None, [vp, dp]),
                "ora_strain_rate": (None, [vp, dp]),
                "ora_solid_mask": (None, [vp, C.POINTER(C.c_ubyte)]),
                "ora_force_torque": (None, [vp, i, dp, dp]),
                "ora_num_markers": (i, [vp, i]),
                "ora_snapshot_velocity": (None, [vp]),
                "ora_residual": (d, [vp]),
                "ora_steps_done": (C.c_long, [vp]),
                "ora_solid_centre": (None, [vp, i, dp]),
                "ora_link_stats": (None, [vp, C.POINTER(C.c_long)]),
                "ora_ibm_interp": (None, [i, i, i, i, dp, i, dp, dp]),
                "ora_ibm_spread": (None, [i, i, i, i, dp, i, dp, dp, dp]),
                "ora_ibm_interp_k": (None, [i, i, i, i, i, dp, i, dp, dp]),
                "ora_ibm_spread_k": (None, [i, i, i, i, i, dp, i, dp, dp, dp]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec3(v):
    a = np.zeros(3)
    if v is not None:
        v = np.asarray(v, dtype=np.float64).ravel()
        a[:len(v)] = v
    return a


def q_of(lat: int) -> int:
    return lib().ora_q(lat)


def lattice(lat: int):
    Q = q_of(lat)
    e = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q)
    lib().ora_lattice(lat, e.ctypes.data_as(C.POINTER(C.c_int)), _p(w))
    return e, w


def mrt_matrix(lat: int) -> np.ndarray:
    Q = q_of(lat)
    M = np.zeros((Q, Q))
    lib().ora_mrt_matrix(lat, _p(M))
    return M


def mrt_default_rates(lat: int, tau: float) -> np.ndarray:
    s = np.zeros(q_of(lat))
    lib().ora_mrt_default_rates(lat, tau, _p(s))
    return s


def equilibrium(lat: int, rho: float, u) -> np.ndarray:
    feq = np.zeros(q_of(lat))
    lib().ora_equilibrium(lat, rho, _p(_vec3(u)), _p(feq))
    return feq


def collide(lat: int, coll: int, tau: float, f, F=None, rates=None) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    r = None if rates is None else np.ascontiguousarray(rates, dtype=np.float64)
    lib().ora_collide(lat, coll, tau, None if r is None else _p(r), _p(f),
                      _p(_vec3(F)), _p(out))
    return out


def ibb_coeffs(scheme: int, q: float, have_ff=True, have_fff=True):
    c = np.zeros(6)
    used = lib().ora_ibb_coeffs(scheme, q, int(have_ff), int(have_fff), _p(c))
    return c, used


# delta-function kernels (same selectors as the library's LBM_DELTA_*)
PESKIN4, ROMA3, LINEAR2, COSINE4 = range(4)


def phi(r: float, kernel: int = PESKIN4) -> float:
    if kernel == PESKIN4:
        return lib().ora_phi(float(r))
    return lib().ora_phi_kernel(int(kernel), float(r))


def ibm_interp(d, shape, u, X, kernel: int = PESKIN4):
    """u: [d][nz][ny][nx] (nz=1 for d=2); X: [3][n] -> U [d][n]."""
    nx, ny, nz = shape
    u = np.ascontiguousarray(u, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[1]
    U = np.zeros((d, n))
    if kernel == PESKIN4:
        lib().ora_ibm_interp(d, nx, ny, nz, _p(u), n, _p(X), _p(U))
    else:
        lib().ora_ibm_interp_k(int(kernel), d, nx, ny, nz, _p(u), n, _p(X), _p(U))
    return U


def ibm_spread(d, shape, F, X, dV, kernel: int = PESKIN4):
    nx, ny, nz = shape
    N = nx * ny * (nz if d == 3 else 1)
    f = np.zeros((d, N))
    F = np.ascontiguousarray(F, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    dV = np.ascontiguousarray(dV, dtype=np.float64)
    if kernel == PESKIN4:
        lib().ora_ibm_spread(d, nx, ny, nz, _p(f), X.shape[1], _p(X), _p(F), _p(dV))
    else:
        lib().ora_ibm_spread_k(int(kernel), d, nx, ny, nz, _p(f), X.shape[1], _p(X), _p(F),
                               _p(dV))
    return f


class OracleSim:
    """One lattice of the oracle.  Parameters mirror the library's lattice,
    solid and scheme descriptors, but are plain keyword arguments."""

    def __init__(self, lattice: int, nx: int, ny: int, nz: int, tau: float,
                 collision: int = BGK, rates=None, g=None, force_all=False):
        self.L = lib()
        self.lattice = lattice
        self.Q = q_of(lattice)
        self.d = 2 if lattice == D2Q9 else 3
        self.shape = (nz if self.d == 3 else 1, ny, nx)
        self.N = int(np.prod(self.shape))
        r = None
        if rates is not None:
            r = np.zeros(19)
            rr = np.asarray(rates, dtype=np.float64).ravel()
            r[:len(rr)] = rr
        self._rates = r
        self.h = self.L.ora_create(lattice, nx, ny, nz, tau, collision,
                                   None if r is None else _p(r), _p(_vec3(g)),
                                   int(force_all))
        if not self.h:
            raise MemoryError("ora_create failed")

    def close(self):
        if getattr(self, "h", None):
            self.L.ora_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def add_solid(self, kind, centre, radius, velocity=None, omega=None,
                  fluid_inside=False) -> int:
        sid = self.L.ora_add_solid(self.h, kind, _p(_vec3(centre)), float(radius),
                                   _p(_vec3(velocity)), _p(_vec3(omega)),
                                   int(fluid_inside))
        if sid < 0:
            raise ValueError("too many solids")
        return sid

    def set_scheme(self, scheme, ibm_iters=1, retraction=0.0, marker_density=1.0,
                   ibm_kernel=PESKIN4, ibm_inertia=0):
        self.L.ora_set_ibm_kernel(self.h, int(ibm_kernel))
        self.L.ora_set_ibm_inertia(self.h, int(ibm_inertia))
        self.L.ora_set_scheme(self.h, scheme, ibm_iters, retraction, marker_density)

    def init_equilibrium(self, rho=1.0, u=None):
        self.L.ora_init_equilibrium(self.h, rho, _p(_vec3(u)))

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.Q, self.N)
        self.L.ora_set_f(self.h, _p(f))

    def get_f(self):
        f = np.zeros((self.Q, self.N))
        self.L.ora_get_f(self.h, _p(f))
        return f.reshape((self.Q,) + self.shape)

    def step(self, n=1):
        self.L.ora_step(self.h, int(n))

    def density(self):
        r = np.zeros(self.N)
        self.L.ora_density(self.h, _p(r))
        return r.reshape(self.shape)

    def velocity(self):
        u = np.zeros((self.d, self.N))
        self.L.ora_velocity(self.h, _p(u))
        return u.reshape((self.d,) + self.shape)

    def strain_rate(self):
        nc = 3 if self.d == 2 else 6
        S = np.zeros((nc, self.N))
        self.L.ora_strain_rate(self.h, _p(S))
        return S.reshape((nc,) + self.shape)

    def stress(self):
        nc = 3 if self.d == 2 else 6
        S = np.zeros((nc, self.N))
        self.L.ora_stress(self.h, _p(S))
        return S.reshape((nc,) + self.shape)

    def solid_mask(self):
        m = np.zeros(self.N, dtype=np.uint8)
        self.L.ora_solid_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return m.reshape(self.shape).astype(bool)

    def force_torque(self, sid=0):
        F = np.zeros(3)
        T = np.zeros(3)
        self.L.ora_force_torque(self.h, sid, _p(F), _p(T))
        return F, T

    def num_markers(self, sid=0):
        return self.L.ora_num_markers(self.h, sid)

    def snapshot_velocity(self):
        self.L.ora_snapshot_velocity(self.h)

    def residual(self):
        return self.L.ora_residual(self.h)

    def steps_done(self):
        return self.L.ora_steps_done(self.h)

    def solid_centre(self, sid=0):
        c = np.zeros(3)
        self.L.ora_solid_centre(self.h, sid, _p(c))
        return c

    def dissipation(self):
        e = np.zeros(self.N)
        self.L.ora_dissipation(self.h, _p(e))
        return e.reshape(self.shape)

    def set_domain(self, faces, u_face=None):
        """Face types x-, x+, y-, y+, z-, z+ and the velocity of each face
        ([6][3]); raises ValueError where the oracle refuses them."""
        fc = (C.c_int * 6)(*[int(t) for t in faces])
        u = np.zeros((6, 3)) if u_face is None else np.ascontiguousarray(u_face, dtype=np.float64)
        if self.L.ora_set_domain(self.h, fc, _p(u)) != 0:
            raise ValueError(f"domain refused: {list(faces)}")

    def cell_fraction(self, sid, x, y, z=0):
        return self.L.ora_cell_fraction(self.h, sid, int(x), int(y), int(z))

    def internal_fluid(self, sid=0):
        I = np.zeros(6)
        self.L.ora_internal_fluid(self.h, sid, _p(I))
        return I[:3], I[3:]

    def set_solid_dynamics(self, sid, rho_ratio, gravity=None):
        self.L.ora_set_solid_dynamics(self.h, sid, float(rho_ratio), _p(_vec3(gravity)))

    def solid_velocity(self, sid=0):
        U, Om = np.zeros(3), np.zeros(3)
        self.L.ora_solid_velocity(self.h, sid, _p(U), _p(Om))
        return U, Om

    def link_stats(self):
        c = (C.c_long * 8)()
        self.L.ora_link_stats(self.h, c)
        return list(c)

    def run_to_steady(self, tol, max_steps, check_every=100):
        """Step until the velocity residual over `check_every` steps drops
        below tol; returns (steps done, last residual)."""
        done = 0
        r = float("inf")
        self.snapshot_velocity()
        while done < max_steps:
            k = min(check_every, max_steps - done)
            self.step(k)
            done += k
            r = self.residual()
            if r < tol:
                break
            self.snapshot_velocity()
        return done, r
