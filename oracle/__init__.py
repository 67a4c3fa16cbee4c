"""Plain FP64 CPU oracle of the LBM-PSM hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path: the C file ``psm_oracle.c`` is
written from the paper's equations (Sec. 2, Eqs. 1-27) and ``mlp.py`` holds the
FP64 reference of the eps surrogate network.

``build()`` compiles ``psm_oracle.c`` with plain gcc (``-ffp-contract=off``, so
every product and sum rounds the way the source reads) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so and return its path."""
    src = os.path.join(_HERE, "psm_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, src]
    try:  # OpenMP for the threaded loops; without it the oracle runs on one thread
        subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, _SO)
    return _SO


class _Config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("wall", C.c_int * 6), ("tau", C.c_double), ("relax", C.c_int),
                ("magic", C.c_double), ("fbody", C.c_double * 3),
                ("weighting", C.c_int), ("eps_mode", C.c_int), ("eps_n", C.c_int),
                ("gravity", C.c_double * 3), ("kn", C.c_double),
                ("restitution", C.c_double), ("subcycles", C.c_int), ("dem", C.c_int),
                ("bc_velocity", C.c_double * 3), ("bc_density", C.c_double),
                ("kt_ratio", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.or_create.restype = P
            L.or_create.argtypes = [C.POINTER(_Config)]
            L.or_destroy.argtypes = [P]
            L.or_set_particles.argtypes = [P, C.c_int, dp, dp, dp, dp, dp, C.c_void_p]
            L.or_set_mlp.argtypes = [P, dp, dp, dp, dp, dp, dp]
            L.or_set_pdfs.argtypes = [P, dp]
            L.or_get_pdfs.argtypes = [P, dp]
            L.or_map.argtypes = [P]
            L.or_get_slots.argtypes = [P, ip, dp, ip, dp]
            L.or_step.argtypes = [P, C.c_int]
            L.or_set_threads.argtypes = [P, C.c_int]
            L.or_dem_only.argtypes = [P, C.c_int]
            L.or_get_force_torque.argtypes = [P, dp, dp]
            L.or_set_hydro.argtypes = [P, dp, dp]
            L.or_get_contact.argtypes = [P, dp, dp]
            L.or_get_particles.argtypes = [P, dp, dp, dp]
            L.or_macroscopic.argtypes = [P, dp, dp]
            L.or_mass.argtypes = [P]
            L.or_mass.restype = C.c_double
            L.or_momentum.argtypes = [P, dp]
            L.or_last_fext.argtypes = [P, dp]
            L.or_last_fluid_volume.argtypes = [P]
            L.or_last_fluid_volume.restype = C.c_double
            L.or_Va.argtypes = [C.c_double]
            L.or_Va.restype = C.c_double
            L.or_eps_linear.argtypes = [C.c_double, C.c_double]
            L.or_eps_linear.restype = C.c_double
            L.or_eps_supersample_count.argtypes = [C.c_double] * 4 + [C.c_int]
            L.or_eps_supersample_count.restype = C.c_long
            L.or_nt_weight.argtypes = [C.c_double, C.c_double]
            L.or_nt_weight.restype = C.c_double
            L.or_supersample_batch.argtypes = [C.c_long, dp, dp, C.c_int,
                                               C.POINTER(C.c_long)]
            L.or_eps_linear_batch.argtypes = [C.c_long, dp, dp, dp]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


Q = 19


class Oracle:
    """One oracle simulation (wraps ``or_ctx``).

    Arguments mirror the engine's configuration: grid ``(nx, ny, nz)``, ``walls``
    as six face types for faces -x,+x,-y,+y,-z,+z (0 periodic, 1 wall, 2
    velocity inflow at ``bc_velocity``, 3 pressure outflow at ``bc_density``;
    2 and 3 on the z faces only), relaxation time ``tau``,
    ``relax`` ("srt"/"trt"), TRT ``magic``, fluid body force ``fbody``,
    ``weighting`` ("eps"/"nt"), ``eps_mode`` ("supersample"/"linear"/"mlp")
    with ``eps_n`` samples per axis, and the DEM parameters.
    """

    def __init__(self, nx, ny, nz, tau, relax="srt", magic=3.0 / 16.0,
                 walls=(0, 0, 0, 0, 0, 0), fbody=(0.0, 0.0, 0.0), weighting="eps",
                 eps_mode="supersample", eps_n=4, gravity=(0.0, 0.0, 0.0), kn=1e3,
                 restitution=0.9, subcycles=10, dem=False, bc_velocity=(0.0, 0.0, 0.0),
                 bc_density=1.0, kt_ratio=2.0 / 7.0):
        L = lib()
        cfg = _Config()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        for i, w in enumerate(walls):
            cfg.wall[i] = int(w)
        cfg.tau = tau
        cfg.relax = {"srt": 0, "trt": 1}[relax]
        cfg.magic = magic
        for i in range(3):
            cfg.fbody[i] = fbody[i]
            cfg.gravity[i] = gravity[i]
        cfg.weighting = {"eps": 0, "nt": 1}[weighting]
        cfg.eps_mode = {"supersample": 0, "linear": 1, "mlp": 2}[eps_mode]
        cfg.eps_n = eps_n
        cfg.kn = kn
        cfg.restitution = restitution
        cfg.subcycles = subcycles
        cfg.dem = int(bool(dem))
        for i in range(3):
            cfg.bc_velocity[i] = bc_velocity[i]
        cfg.bc_density = bc_density
        cfg.kt_ratio = kt_ratio
        self._L = L
        self.h = L.or_create(C.byref(cfg))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.np = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self._L.or_destroy(h)
            self.h = None

    def set_particles(self, x, r, u=None, omega=None, density=None, fixed=None):
        r = _f64(r)
        n = r.size
        x = _f64(x, 3 * n)
        u = _f64(np.zeros(3 * n) if u is None else u, 3 * n)
        omega = _f64(np.zeros(3 * n) if omega is None else omega, 3 * n)
        density = _f64(np.ones(n) if density is None else density, n)
        fx = None
        if fixed is not None:
            fx = np.ascontiguousarray(np.asarray(fixed, dtype=np.uint8))
        st = self._L.or_set_particles(
            self.h, n, _dp(x), _dp(r), _dp(u), _dp(omega), _dp(density),
            fx.ctypes.data_as(C.c_void_p) if fx is not None else None)
        if st != 0:
            raise ValueError("oracle rejected the particles")
        self.np = n
        self._keep = fx

    def set_mlp(self, W1, b1, W2, b2, W3, b3):
        a = [_f64(v) for v in (W1, b1, W2, b2, W3, b3)]
        self._L.or_set_mlp(self.h, *[_dp(v) for v in a])

    def set_pdfs(self, f):
        f = _f64(f, Q * self.N)
        self._L.or_set_pdfs(self.h, _dp(f))

    def pdfs(self):
        f = np.empty(Q * self.N)
        self._L.or_get_pdfs(self.h, _dp(f))
        return f.reshape((Q,) + self.shape)

    def map(self):
        return self._L.or_map(self.h)

    def slots(self):
        p0 = np.empty(self.N, np.int32)
        p1 = np.empty(self.N, np.int32)
        b0 = np.empty(self.N)
        b1 = np.empty(self.N)
        ip = C.POINTER(C.c_int)
        self._L.or_get_slots(self.h, p0.ctypes.data_as(ip), _dp(b0),
                             p1.ctypes.data_as(ip), _dp(b1))
        return (p0.reshape(self.shape), b0.reshape(self.shape),
                p1.reshape(self.shape), b1.reshape(self.shape))

    def set_threads(self, n):
        """Host threads of the step's loops; results do not depend on it."""
        self._L.or_set_threads(self.h, int(n))

    def step(self, n=1):
        st = self._L.or_step(self.h, n)
        if st != 0:
            raise RuntimeError(f"oracle step failed with status {st}")

    def dem_only(self, n=1):
        self._L.or_dem_only(self.h, n)

    def force_torque(self):
        F = np.empty(3 * max(self.np, 1))
        T = np.empty(3 * max(self.np, 1))
        self._L.or_get_force_torque(self.h, _dp(F), _dp(T))
        return F[: 3 * self.np].reshape(-1, 3), T[: 3 * self.np].reshape(-1, 3)

    def contact(self):
        """Contact force and torque of every particle at the last DEM sub-step."""
        n = max(self.np, 1)
        F, T = np.empty(3 * n), np.empty(3 * n)
        self._L.or_get_contact(self.h, _dp(F), _dp(T))
        return F[: 3 * self.np].reshape(-1, 3), T[: 3 * self.np].reshape(-1, 3)

    def set_hydro(self, F, T):
        F = _f64(F, 3 * self.np)
        T = _f64(T, 3 * self.np)
        self._L.or_set_hydro(self.h, _dp(F), _dp(T))

    def particles(self):
        n = max(self.np, 1)
        x, u, om = np.empty(3 * n), np.empty(3 * n), np.empty(3 * n)
        self._L.or_get_particles(self.h, _dp(x), _dp(u), _dp(om))
        k = 3 * self.np
        return x[:k].reshape(-1, 3), u[:k].reshape(-1, 3), om[:k].reshape(-1, 3)

    def macroscopic(self):
        rho = np.empty(self.N)
        u = np.empty(3 * self.N)
        self._L.or_macroscopic(self.h, _dp(rho), _dp(u))
        return rho.reshape(self.shape), u.reshape((3,) + self.shape)

    def mass(self):
        return self._L.or_mass(self.h)

    def momentum(self):
        P = np.empty(3)
        self._L.or_momentum(self.h, _dp(P))
        return P

    def last_fext(self):
        fe = np.empty(3)
        self._L.or_last_fext(self.h, _dp(fe))
        return fe

    def last_fluid_volume(self):
        return self._L.or_last_fluid_volume(self.h)


# --- stand-alone mapping pieces (Sec. 2.3.2) --------------------------------

def Va(r: float) -> float:
    """Eq. 27 closed form."""
    return lib().or_Va(float(r))


def eps_linear(dist: float, r: float) -> float:
    """Eqs. 25-26, clamped to [0, 1]."""
    return lib().or_eps_linear(float(dist), float(r))


def supersample_count(d, r: float, n: int) -> int:
    """Number of the n^3 sub-cell sample points of the cell at offset d inside."""
    return int(lib().or_eps_supersample_count(float(d[0]), float(d[1]), float(d[2]),
                                              float(r), int(n)))


def supersample_batch(d, r, n: int) -> np.ndarray:
    d = _f64(d)
    r = _f64(r)
    m = r.size
    assert d.size == 3 * m
    out = np.empty(m, dtype=np.int64)
    lib().or_supersample_batch(m, _dp(d), _dp(r), int(n),
                               out.ctypes.data_as(C.POINTER(C.c_long)))
    return out


def eps_linear_batch(dist, r) -> np.ndarray:
    dist = _f64(dist)
    r = _f64(r)
    out = np.empty(r.size)
    lib().or_eps_linear_batch(r.size, _dp(dist), _dp(r), _dp(out))
    return out


def nt_weight(eps: float, tau: float) -> float:
    return lib().or_nt_weight(float(eps), float(tau))
