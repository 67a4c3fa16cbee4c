"""Thin ctypes binding of the engine's C ABI (``include/psm.h``).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libpsm.so``.  PyTorch supplies the device allocator (its caching
allocator, through the ``alloc``/``free`` callbacks) and the CUDA stream.
There is no CPU fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpsm.so")

PSM_OK, PSM_ERR_ARG, PSM_ERR_CUDA, PSM_ERR_OOM = 0, 1, 2, 3
PSM_ERR_SLOT_OVERFLOW, PSM_ERR_NONFINITE, PSM_ERR_TIMEOUT, PSM_ERR_STATE = 4, 5, 6, 7
STATUS_NAMES = {0: "PSM_OK", 1: "PSM_ERR_ARG", 2: "PSM_ERR_CUDA", 3: "PSM_ERR_OOM",
                4: "PSM_ERR_SLOT_OVERFLOW", 5: "PSM_ERR_NONFINITE", 6: "PSM_ERR_TIMEOUT",
                7: "PSM_ERR_STATE"}
PSM_SRT, PSM_TRT = 0, 1
PSM_FP64, PSM_FP32_DEV, PSM_FP64_DF = 0, 1, 2
PSM_PULL, PSM_AA = 0, 1
PSM_EPS_SUPERSAMPLE, PSM_EPS_LINEAR, PSM_EPS_MLP = 0, 1, 2
PSM_W_EPS, PSM_W_NT = 0, 1
PSM_MLP_PARAMS = 1249
Q = 19

EXPORTS = [
    "psm_default_options", "psm_create", "psm_set_particles", "psm_update_particles",
    "psm_step", "psm_step_host_dem", "psm_dem_step_host",
    "psm_get_force_torque", "psm_get_macroscopic", "psm_get_particles", "psm_get_pdfs",
    "psm_get_pdfs_box", "psm_get_fluid_force",
    "psm_set_pdfs", "psm_get_slots", "psm_check", "psm_set_mlp", "psm_get_mlp",
    "psm_train_surrogate", "psm_mlp_samples", "psm_mlp_loss_grad", "psm_mlp_infer",
    "psm_set_timing", "psm_get_timings", "psm_last_launch_count", "psm_last_error",
    "psm_destroy", "psm_field_sums_noalloc", "psm_save", "psm_load", "psm_get_particle_count",
    "psm_selftest_waits", "psm_get_slot_forces",
]

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class PsmGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("wall", C.c_int * 6)]


class PsmOptions(C.Structure):
    _fields_ = [("magic", C.c_double), ("precision", C.c_int), ("streaming", C.c_int),
                ("eps_mode", C.c_int), ("eps_n", C.c_int), ("weighting", C.c_int),
                ("body_force", C.c_double * 3), ("gravity", C.c_double * 3),
                ("k_n", C.c_double), ("restitution", C.c_double),
                ("dem_subcycles", C.c_int), ("dem", C.c_int), ("deterministic", C.c_int),
                ("use_graphs", C.c_int), ("stream", C.c_void_p), ("alloc", ALLOC_FN),
                ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("bc_velocity", C.c_double * 3), ("bc_density", C.c_double),
                ("kt_ratio", C.c_double)]


_lib = None


def lib():
    """Load libpsm.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA engine library not built: {LIB_PATH} is missing "
                           "(run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    fp = C.POINTER(C.c_float)
    ip = C.POINTER(C.c_int)
    st = C.c_int
    L.psm_default_options.argtypes = [C.POINTER(PsmOptions)]
    L.psm_default_options.restype = None
    L.psm_create.argtypes = [C.POINTER(PsmGrid), C.c_double, C.c_int, C.POINTER(PsmOptions),
                             C.POINTER(P)]
    L.psm_create.restype = st
    L.psm_set_particles.argtypes = [P, C.c_int, dp, dp, dp, dp, dp, C.c_void_p]
    L.psm_set_particles.restype = st
    L.psm_update_particles.argtypes = [P, C.c_void_p, C.c_void_p, C.c_void_p]
    L.psm_update_particles.restype = st
    L.psm_step.argtypes = [P, C.c_int]
    L.psm_step.restype = st
    L.psm_step_host_dem.argtypes = [P, C.c_int, C.c_int, C.POINTER(C.c_double)]
    L.psm_step_host_dem.restype = st
    dpp = C.POINTER(C.c_double)
    ipp = C.POINTER(C.c_int)
    L.psm_dem_step_host.argtypes = [C.POINTER(PsmGrid), C.c_double, C.c_double, C.c_double,
                                    C.c_int, dpp, C.c_int, dpp, dpp, dpp, dpp, dpp, ipp, ipp,
                                    dpp, dpp, dpp, dpp, dpp, C.POINTER(C.c_ubyte), C.c_int]
    L.psm_dem_step_host.restype = st
    L.psm_get_pdfs_box.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, dp]
    L.psm_get_pdfs_box.restype = st
    L.psm_get_fluid_force.argtypes = [P, dp, C.POINTER(C.c_double)]
    L.psm_get_fluid_force.restype = st
    for name in ("psm_get_force_torque",):
        getattr(L, name).argtypes = [P, dp, dp]
        getattr(L, name).restype = st
    L.psm_get_macroscopic.argtypes = [P, dp, dp]
    L.psm_get_macroscopic.restype = st
    L.psm_get_particles.argtypes = [P, dp, dp, dp]
    L.psm_get_particles.restype = st
    L.psm_get_pdfs.argtypes = [P, dp]
    L.psm_get_pdfs.restype = st
    L.psm_set_pdfs.argtypes = [P, dp]
    L.psm_set_pdfs.restype = st
    L.psm_get_slots.argtypes = [P, ip, dp, ip, dp]
    L.psm_get_slots.restype = st
    L.psm_check.argtypes = [P, dp, dp]
    L.psm_check.restype = st
    L.psm_set_mlp.argtypes = [P, fp]
    L.psm_set_mlp.restype = st
    L.psm_get_mlp.argtypes = [P, fp]
    L.psm_get_mlp.restype = st
    L.psm_train_surrogate.argtypes = [P, C.c_long, C.c_ulonglong, C.c_int, C.c_int, C.c_float,
                                      fp]
    L.psm_train_surrogate.restype = st
    L.psm_mlp_samples.argtypes = [P, C.c_ulonglong, C.c_long, C.c_long, fp, fp]
    L.psm_mlp_samples.restype = st
    L.psm_mlp_loss_grad.argtypes = [P, fp, C.c_long, fp, fp, fp, fp]
    L.psm_mlp_loss_grad.restype = st
    L.psm_mlp_infer.argtypes = [P, fp, C.c_long, fp, fp]
    L.psm_mlp_infer.restype = st
    L.psm_set_timing.argtypes = [P, C.c_int]
    L.psm_set_timing.restype = st
    L.psm_get_timings.argtypes = [P, dp]
    L.psm_get_timings.restype = st
    L.psm_last_launch_count.argtypes = [P]
    L.psm_last_launch_count.restype = C.c_long
    L.psm_last_error.argtypes = [P]
    L.psm_last_error.restype = C.c_char_p
    L.psm_destroy.argtypes = [P]
    L.psm_destroy.restype = None
    L.psm_field_sums_noalloc.argtypes = [C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p]
    L.psm_field_sums_noalloc.restype = st
    L.psm_save.argtypes = [P, C.c_char_p]
    L.psm_save.restype = st
    L.psm_load.argtypes = [P, C.c_char_p]
    L.psm_load.restype = st
    L.psm_get_particle_count.argtypes = [P, ip]
    L.psm_get_particle_count.restype = st
    L.psm_get_slot_forces.argtypes = [P, ip, ip, dp, dp]
    L.psm_get_slot_forces.restype = st
    L.psm_selftest_waits.argtypes = [P, C.c_longlong]
    L.psm_selftest_waits.restype = st
    _lib = L
    return L


class PsmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fp(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _f32(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


class TorchAllocator:
    """Routes the engine's device allocations through PyTorch's caching
    allocator on the current device and stream."""

    def __init__(self, stream=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.live = {}

        def _alloc(nbytes, user):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), stream=self.stream)
            except RuntimeError:
                return None
            self.live[int(ptr)] = True
            return int(ptr)

        def _free(ptr, user):
            if ptr and self.live.pop(int(ptr), None):
                torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc_fn = ALLOC_FN(_alloc)
        self.free_fn = FREE_FN(_free)


class Engine:
    """One engine context.  Arguments mirror the oracle's configuration:
    grid (nx, ny, nz), ``walls`` six face types (-x,+x,-y,+y,-z,+z: 0 periodic,
    1 wall, 2 velocity inflow at ``bc_velocity`` and 3 pressure outflow at
    ``bc_density``, the last two on the z faces only), ``tau``,
    ``relax`` "srt"/"trt", ``magic``, ``fbody``, ``weighting`` "eps"/"nt",
    ``eps_mode`` "supersample"/"linear"/"mlp", ``eps_n``, DEM parameters,
    ``precision`` "fp64"/"fp32"/"df64" (FP64, FP32 deviations, double-float
    pairs), ``streaming`` "pull"/"aa"."""

    def __init__(self, nx, ny, nz, tau, relax="srt", magic=3.0 / 16.0,
                 walls=(0, 0, 0, 0, 0, 0), fbody=(0.0, 0.0, 0.0), weighting="eps",
                 eps_mode="supersample", eps_n=4, gravity=(0.0, 0.0, 0.0), kn=1e3,
                 restitution=0.9, subcycles=10, dem=False, precision="fp64",
                 streaming="pull", deterministic=True, use_graphs=True, torch_alloc=True,
                 stream=None, bc_velocity=(0.0, 0.0, 0.0), bc_density=1.0,
                 kt_ratio=2.0 / 7.0):
        L = lib()
        self._L = L
        opt = PsmOptions()
        L.psm_default_options(C.byref(opt))
        opt.magic = magic
        opt.precision = {"fp64": PSM_FP64, "fp32": PSM_FP32_DEV, "df64": PSM_FP64_DF}[precision]
        opt.streaming = {"pull": PSM_PULL, "aa": PSM_AA}[streaming]
        opt.eps_mode = {"supersample": 0, "linear": 1, "mlp": 2}[eps_mode]
        opt.eps_n = eps_n
        opt.weighting = {"eps": 0, "nt": 1}[weighting]
        for i in range(3):
            opt.body_force[i] = fbody[i]
            opt.gravity[i] = gravity[i]
        opt.k_n = kn
        opt.restitution = restitution
        opt.dem_subcycles = subcycles
        opt.dem = int(bool(dem))
        opt.deterministic = int(bool(deterministic))
        opt.use_graphs = int(bool(use_graphs))
        for i in range(3):
            opt.bc_velocity[i] = bc_velocity[i]
        opt.bc_density = bc_density
        opt.kt_ratio = kt_ratio
        self._alloc = None
        if torch_alloc:
            import torch
            s = stream if stream is not None else torch.cuda.current_stream()
            self._alloc = TorchAllocator(s)
            opt.stream = s.cuda_stream
            opt.alloc = self._alloc.alloc_fn
            opt.free = self._alloc.free_fn
        g = PsmGrid()
        g.nx, g.ny, g.nz = nx, ny, nz
        for i, w in enumerate(walls):
            g.wall[i] = int(w)
        h = C.c_void_p()
        rc = L.psm_create(C.byref(g), tau, {"srt": PSM_SRT, "trt": PSM_TRT}[relax],
                          C.byref(opt), C.byref(h))
        if rc != PSM_OK:
            raise PsmError(rc, "psm_create failed")
        self.h = h
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.np = 0

    def _check(self, rc):
        if rc != PSM_OK:
            raise PsmError(rc, self._L.psm_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self._L.psm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, x, r, u=None, omega=None, density=None, fixed=None):
        r = _f64(r)
        n = r.size
        x = _f64(x, 3 * n)
        u = _f64(np.zeros(3 * n) if u is None else u, 3 * n)
        omega = _f64(np.zeros(3 * n) if omega is None else omega, 3 * n)
        density = _f64(np.ones(n) if density is None else density, n)
        fx = None if fixed is None else np.ascontiguousarray(np.asarray(fixed, np.uint8))
        self._check(self._L.psm_set_particles(
            self.h, n, _dp(x), _dp(r), _dp(u), _dp(omega), _dp(density),
            fx.ctypes.data_as(C.c_void_p) if fx is not None else None))
        self.np = n

    def update_particles(self, x, u, omega):
        """x, u, omega: float64 numpy arrays (n x 3), or integer host addresses
        (e.g. the data_ptr() of pinned torch tensors)."""
        args = []
        for a in (x, u, omega):
            if isinstance(a, int):
                args.append(C.c_void_p(a))
            else:
                a = _f64(a, 3 * self.np)
                args.append(a.ctypes.data_as(C.c_void_p))
                self._keep_upd = getattr(self, "_keep_upd", []) + [a]
        self._check(self._L.psm_update_particles(self.h, *args))
        self._keep_upd = []

    def force_torque_into(self, F_addr, T_addr):
        """psm_get_force_torque into caller-owned host buffers (addresses)."""
        dp = C.POINTER(C.c_double)
        self._check(self._L.psm_get_force_torque(self.h, C.cast(F_addr, dp), C.cast(T_addr, dp)))

    def particles_into(self, x_addr, u_addr, om_addr):
        dp = C.POINTER(C.c_double)
        self._check(self._L.psm_get_particles(self.h, C.cast(x_addr, dp), C.cast(u_addr, dp),
                                              C.cast(om_addr, dp)))

    def step(self, n=1):
        return self._check(self._L.psm_step(self.h, int(n)))

    def step_status(self, n=1):
        """psm_step without raising: returns the status code."""
        return self._L.psm_step(self.h, int(n))

    def step_host_dem(self, n=1, threads=0):
        """n steps with the particle dynamics on the host cores; returns the
        milliseconds spent in the host phase (force copy, DEM, state copy)."""
        ms = C.c_double(0.0)
        self._check(self._L.psm_step_host_dem(self.h, int(n), int(threads), C.byref(ms)))
        return ms.value

    def force_torque(self):
        F = np.zeros(3 * max(self.np, 1))
        T = np.zeros(3 * max(self.np, 1))
        self._check(self._L.psm_get_force_torque(self.h, _dp(F), _dp(T)))
        k = 3 * self.np
        return F[:k].reshape(-1, 3), T[:k].reshape(-1, 3)

    def particles(self):
        n = max(self.np, 1)
        x, u, om = np.zeros(3 * n), np.zeros(3 * n), np.zeros(3 * n)
        self._check(self._L.psm_get_particles(self.h, _dp(x), _dp(u), _dp(om)))
        k = 3 * self.np
        return x[:k].reshape(-1, 3), u[:k].reshape(-1, 3), om[:k].reshape(-1, 3)

    def pdfs(self):
        f = np.empty(Q * self.N)
        self._check(self._L.psm_get_pdfs(self.h, _dp(f)))
        return f.reshape((Q,) + self.shape)

    def pdfs_box(self, x0, y0, z0, bx, by, bz):
        """Post-collision PDFs of a box of cells, shape (19, bz, by, bx)."""
        f = np.empty(Q * bx * by * bz)
        self._check(self._L.psm_get_pdfs_box(self.h, int(x0), int(y0), int(z0), int(bx),
                                             int(by), int(bz), _dp(f)))
        return f.reshape((Q, bz, by, bx))

    def fluid_force(self):
        """(fluid force density of the last step (3,), fluid volume)."""
        f = np.empty(3)
        v = C.c_double(0.0)
        self._check(self._L.psm_get_fluid_force(self.h, _dp(f), C.byref(v)))
        return f, v.value

    def set_pdfs(self, f):
        f = _f64(f, Q * self.N)
        self._check(self._L.psm_set_pdfs(self.h, _dp(f)))

    def macroscopic(self):
        rho = np.empty(self.N)
        u = np.empty(3 * self.N)
        self._check(self._L.psm_get_macroscopic(self.h, _dp(rho), _dp(u)))
        return rho.reshape(self.shape), u.reshape((3,) + self.shape)

    def slots(self):
        p0 = np.empty(self.N, np.int32)
        p1 = np.empty(self.N, np.int32)
        b0 = np.empty(self.N)
        b1 = np.empty(self.N)
        ip = C.POINTER(C.c_int)
        self._check(self._L.psm_get_slots(self.h, p0.ctypes.data_as(ip), _dp(b0),
                                          p1.ctypes.data_as(ip), _dp(b1)))
        return (p0.reshape(self.shape), b0.reshape(self.shape), p1.reshape(self.shape),
                b1.reshape(self.shape))

    def slot_forces(self):
        """Per-slot forces of the last step with the mapping they belong to
        (psm_get_slot_forces): pid0, pid1 (nz, ny, nx) and F0, F1
        (nz, ny, nx, 3)."""
        p0 = np.empty(self.N, np.int32)
        p1 = np.empty(self.N, np.int32)
        F0 = np.empty(3 * self.N)
        F1 = np.empty(3 * self.N)
        ipp = C.POINTER(C.c_int)
        self._check(self._L.psm_get_slot_forces(self.h, p0.ctypes.data_as(ipp),
                                                p1.ctypes.data_as(ipp), _dp(F0), _dp(F1)))
        return (p0.reshape(self.shape), p1.reshape(self.shape),
                F0.reshape(self.shape + (3,)), F1.reshape(self.shape + (3,)))

    def check(self):
        m = C.c_double()
        P = np.zeros(3)
        self._check(self._L.psm_check(self.h, C.byref(m), _dp(P)))
        return m.value, P

    def save(self, path):
        """Checkpoint of the stepper state (psm_save)."""
        self._check(self._L.psm_save(self.h, os.fsencode(path)))

    def load(self, path):
        """Restart from a checkpoint written by save() (psm_load)."""
        self._check(self._L.psm_load(self.h, os.fsencode(path)))
        n = C.c_int()
        self._check(self._L.psm_get_particle_count(self.h, C.byref(n)))
        self.np = n.value

    def selftest_waits(self, limit_ns):
        """Status of psm_selftest_waits (PSM_OK when every bounded wait gave up)."""
        return self._L.psm_selftest_waits(self.h, int(limit_ns))

    def set_mlp(self, params):
        p = _f32(params, PSM_MLP_PARAMS)
        self._check(self._L.psm_set_mlp(self.h, _fp(p)))

    def get_mlp(self):
        p = np.empty(PSM_MLP_PARAMS, np.float32)
        self._check(self._L.psm_get_mlp(self.h, _fp(p)))
        return p

    def train_surrogate(self, nsamples, seed, epochs, batch, lr):
        loss = C.c_float()
        self._check(self._L.psm_train_surrogate(self.h, int(nsamples), int(seed), int(epochs),
                                                int(batch), float(lr), C.byref(loss)))
        return loss.value

    def mlp_samples(self, seed, first, count):
        X = np.empty(4 * count, np.float32)
        e = np.empty(count, np.float32)
        self._check(self._L.psm_mlp_samples(self.h, int(seed), int(first), int(count), _fp(X),
                                            _fp(e)))
        return X.reshape(-1, 4), e

    def mlp_loss_grad(self, params, X, t):
        p = _f32(params, PSM_MLP_PARAMS)
        X = _f32(X)
        t = _f32(t)
        m = t.size
        loss = C.c_float()
        g = np.empty(PSM_MLP_PARAMS, np.float32)
        self._check(self._L.psm_mlp_loss_grad(self.h, _fp(p), m, _fp(X), _fp(t),
                                              C.byref(loss), _fp(g)))
        return loss.value, g

    def mlp_infer(self, params, X):
        p = _f32(params, PSM_MLP_PARAMS)
        X = _f32(X)
        m = X.size // 4
        e = np.empty(m, np.float32)
        self._check(self._L.psm_mlp_infer(self.h, _fp(p), m, _fp(X), _fp(e)))
        return e

    def set_timing(self, on):
        self._check(self._L.psm_set_timing(self.h, int(bool(on))))

    def timings(self):
        """[mapping, stream-collide, force reduction, DEM] ms summed, steps."""
        t = np.zeros(5)
        self._check(self._L.psm_get_timings(self.h, _dp(t)))
        return t

    def last_launch_count(self):
        return int(self._L.psm_last_launch_count(self.h))


def field_sums_noalloc(f_dev_ptr: int, ncells: int, sums_dev_ptr: int, stream_ptr: int) -> int:
    """psm_field_sums_noalloc on device addresses; returns the status code.
    The call allocates no device memory (for callers that cannot)."""
    return lib().psm_field_sums_noalloc(C.c_void_p(f_dev_ptr), int(ncells),
                                        C.c_void_p(sums_dev_ptr), C.c_void_p(stream_ptr))


DEM_HIST_CAP = 64  # partners per particle in the tangential contact history


def dem_history(n):
    """An empty tangential contact history for n particles: counts (n),
    partners (n x 64) and accumulated tangential displacements (n x 64 x 3)."""
    return (np.zeros(n, np.int32), np.zeros((n, DEM_HIST_CAP), np.int32),
            np.zeros((n, DEM_HIST_CAP, 3), np.float64))


def dem_step_host(shape, walls, x, u, omega, F_old, T_old, F_hyd, T_hyd, r, density,
                  fixed=None, kn=1e3, restitution=0.9, subcycles=10, gravity=(0.0, 0.0, 0.0),
                  threads=0, kt_ratio=2.0 / 7.0, history=None):
    """One LBM step of particle dynamics on the host cores (psm_dem_step_host):
    x, u, omega, F_old, T_old (float64, n x 3, C-contiguous) and the contact
    ``history`` (from dem_history; a fresh one when None) are advanced in
    place.  Raises PsmError on a non-OK status."""
    n = int(np.asarray(r).size)
    if history is None:
        history = dem_history(n)
    hc, hj, hd = history
    if (hc.dtype != np.int32 or hj.dtype != np.int32 or hd.dtype != np.float64 or
            hc.size != n or hj.size != n * DEM_HIST_CAP or hd.size != 3 * n * DEM_HIST_CAP or
            not (hc.flags.c_contiguous and hj.flags.c_contiguous and hd.flags.c_contiguous)):
        raise ValueError("history arrays must come from dem_history(n)")
    g = PsmGrid()
    g.nx, g.ny, g.nz = (int(v) for v in shape)
    for k in range(6):
        g.wall[k] = int(walls[k])
    arrs = [x, u, omega, F_old, T_old]
    for a in arrs:
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != 3 * n:
            raise ValueError("state arrays must be C-contiguous float64 of n x 3")
    Fh, Th = _f64(F_hyd, 3 * n), _f64(T_hyd, 3 * n)
    rr, dd = _f64(r, n), _f64(density, n)
    fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
    gv = _f64(gravity, 3)
    ip = C.POINTER(C.c_int)
    st = lib().psm_dem_step_host(
        C.byref(g), float(kn), float(restitution), float(kt_ratio), int(subcycles), _dp(gv), n,
        _dp(x), _dp(u), _dp(omega), _dp(F_old), _dp(T_old), hc.ctypes.data_as(ip),
        hj.ctypes.data_as(ip), _dp(hd), _dp(Fh), _dp(Th), _dp(rr), _dp(dd),
        None if fx is None else fx.ctypes.data_as(C.POINTER(C.c_ubyte)), int(threads))
    if st != 0:
        raise PsmError(st, "psm_dem_step_host failed")
    return x, u, omega, F_old, T_old


def pack_mlp(params) -> np.ndarray:
    """[W1 (32x4), b1, W2 (32x32), b2, W3 (1x32), b3] -> packed FP32 vector."""
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in params]).astype(np.float32)


def unpack_mlp(v):
    v = np.asarray(v, np.float64)
    W1 = v[0:128].reshape(32, 4)
    b1 = v[128:160]
    W2 = v[160:1184].reshape(32, 32)
    b2 = v[1184:1216]
    W3 = v[1216:1248].reshape(1, 32)
    b3 = v[1248:1249]
    return [W1, b1, W2, b2, W3, b3]
