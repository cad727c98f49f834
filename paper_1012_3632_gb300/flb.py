"""Thin ctypes binding of the C ABI in ``include/flb.h``.

Argument marshalling only: every step of the fluctuating lattice Boltzmann
update runs in the CUDA kernels of ``libflb.so``.  The Python names mirror the
C entry points (``flb_create`` -> ``Context(...)``, ``flb_step`` ->
``Context.step`` ...); the raw functions are reachable through ``lib()``.

If ``libflb.so`` is missing the binding raises ``FLBError`` -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflb.so")

FLB_OK, FLB_EINVAL, FLB_ENOMEM, FLB_ECUDA, FLB_EDIVERGED, FLB_ETIMEOUT, FLB_EIO, FLB_EBOUNDS = 0, -1, -2, -3, -4, -5, -6, -7
D2Q9, D3Q19 = 9, 19
FP64, FP32, BF16 = 0, 1, 2
RHO, U, MODES, MODE_VAR = 0, 1, 2, 3
NKERNEL_TIMERS = 3
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16": BF16}

# Symbols declared in include/flb.h (checked by the ABI test).
EXPORTS = [
    "flb_default_options", "flb_create", "flb_init", "flb_step", "flb_moments", "flb_structure_factor",
    "flb_snapshot_count", "flb_reset_accumulators", "flb_conservation", "flb_get_populations",
    "flb_set_populations", "flb_get_sites", "flb_check_guards", "flb_z_chunk", "flb_adjoint_segment", "flb_step_sums", "flb_step_sums_async", "flb_get_step", "flb_set_step", "flb_set_stream", "flb_synchronize",
    "flb_get_info", "flb_kernel_timing", "flb_kernel_times", "flb_save", "flb_load", "flb_error_string",
    "flb_last_error", "flb_destroy", "flb_structure_factor_noalloc",
    "flb_batch_create", "flb_batch_init", "flb_batch_step", "flb_batch_autotune", "flb_batch_mode_variance",
    "flb_batch_structure_factor", "flb_batch_get_populations", "flb_batch_info", "flb_batch_synchronize",
    "flb_batch_destroy", "flb_get_state_device", "flb_set_state_device", "flb_adjoint_step",
    "flb_interface_heights", "flb_height_spectrum",
]
BATCH_MAX = 96
NOALLOC_MAX_SITES = 1 << 20


class FLBError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class FreeEnergy(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("A", ctypes.c_double), ("B", ctypes.c_double),
                ("rho_c", ctypes.c_double), ("kappa", ctypes.c_double), ("total", ctypes.c_int),
                ("model", ctypes.c_int)]


class InterfaceFit(ctypes.Structure):
    _fields_ = [("rho_l", ctypes.c_double), ("rho_v", ctypes.c_double), ("width", ctypes.c_double),
                ("guess", ctypes.c_double * 2), ("window", ctypes.c_int), ("iterations", ctypes.c_int)]


def interface_fit(rho_l: float, rho_v: float, width: float, guess, window: int = 8,
                  iterations: int = 8) -> InterfaceFit:
    """flb_interface_fit for a stripe with interfaces near rows guess = (lower, upper)."""
    return InterfaceFit(float(rho_l), float(rho_v), float(width), (ctypes.c_double * 2)(*map(float, guess)),
                        int(window), int(iterations))


def landau_width(rho_l: float, rho_v: float, beta: float, kappa: float) -> float:
    """Interface width w = sqrt(8 kappa / beta) / (rho_L - rho_V) of the mean-field
    profile of the Landau double well (Sec. VI, Eq. (interf-width))."""
    return (8.0 * kappa / beta) ** 0.5 / (rho_l - rho_v)


def landau_free_energy(rho_l: float, rho_v: float, beta: float, kappa: float) -> dict:
    """Free-energy parameters of the Landau double well beta (rho - rho_V)^2 (rho - rho_L)^2
    of Sec. VI as the total bulk free energy: psi' = A d + B d^3, d = rho - (rho_L + rho_V)/2,
    with A = -beta (rho_L - rho_V)^2 and B = 4 beta."""
    return dict(A=-beta * (rho_l - rho_v) ** 2, B=4.0 * beta, rho_c=0.5 * (rho_l + rho_v), kappa=kappa,
                total=True)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("rho0", ctypes.c_double), ("replica", ctypes.c_uint32),
                ("noise_rho_local", ctypes.c_int), ("stream", ctypes.c_void_p), ("device", ctypes.c_int),
                ("check_every", ctypes.c_int), ("guard", ctypes.c_int), ("z_chunk", ctypes.c_int)]


_lib = None


def lib():
    """Load libflb.so (raises FLBError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FLBError(FLB_ECUDA, f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, dp, ip, vp = ctypes.POINTER, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p
    sig = {
        "flb_default_options": (None, [P(Options)]),
        "flb_create": (ctypes.c_int, [P(vp), ctypes.c_int, ip, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, P(FreeEnergy), ctypes.c_uint64, P(Options)]),
        "flb_init": (ctypes.c_int, [vp, dp, dp, ctypes.c_int]),
        "flb_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "flb_moments": (ctypes.c_int, [vp, dp, ctypes.c_int]),
        "flb_structure_factor": (ctypes.c_int, [vp, dp, ctypes.c_int, ctypes.c_int]),
        "flb_snapshot_count": (ctypes.c_int, [vp, ctypes.c_int, ip]),
        "flb_reset_accumulators": (ctypes.c_int, [vp]),
        "flb_conservation": (ctypes.c_int, [vp, dp]),
        "flb_get_populations": (ctypes.c_int, [vp, dp]),
        "flb_set_populations": (ctypes.c_int, [vp, dp]),
        "flb_get_sites": (ctypes.c_int, [vp, P(ctypes.c_longlong), ctypes.c_int, dp]),
        "flb_check_guards": (ctypes.c_int, [vp]),
        "flb_z_chunk": (ctypes.c_int, [vp, ip, ip]),
        "flb_adjoint_segment": (ctypes.c_int, [vp, vp, ctypes.c_uint64, ctypes.c_int, vp, vp, vp]),
        "flb_step_sums": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "flb_step_sums_async": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "flb_get_step": (ctypes.c_int, [vp, P(ctypes.c_uint64)]),
        "flb_set_step": (ctypes.c_int, [vp, ctypes.c_uint64]),
        "flb_set_stream": (ctypes.c_int, [vp, vp]),
        "flb_synchronize": (ctypes.c_int, [vp]),
        "flb_get_info": (ctypes.c_int, [vp, ip]),
        "flb_kernel_timing": (ctypes.c_int, [vp, ctypes.c_int]),
        "flb_kernel_times": (ctypes.c_int, [vp, dp, ip]),
        "flb_save": (ctypes.c_int, [vp, ctypes.c_char_p]),
        "flb_load": (ctypes.c_int, [P(vp), ctypes.c_char_p, P(Options)]),
        "flb_error_string": (ctypes.c_char_p, [ctypes.c_int]),
        "flb_last_error": (ctypes.c_char_p, []),
        "flb_destroy": (None, [vp]),
        "flb_structure_factor_noalloc": (ctypes.c_int, [ctypes.c_int, ip, vp, ctypes.c_int, vp, vp]),
        "flb_batch_create": (ctypes.c_int, [P(vp), ctypes.c_int, ctypes.c_int, ip, dp, dp, dp, dp,
                                            P(ctypes.c_uint64), P(Options)]),
        "flb_batch_init": (ctypes.c_int, [vp, ctypes.c_int]),
        "flb_batch_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "flb_batch_autotune": (ctypes.c_int, [vp, ip]),
        "flb_batch_mode_variance": (ctypes.c_int, [vp, dp]),
        "flb_batch_structure_factor": (ctypes.c_int, [vp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int]),
        "flb_batch_get_populations": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "flb_batch_info": (ctypes.c_int, [vp, ip, P(ctypes.c_longlong), P(ctypes.c_uint64)]),
        "flb_batch_synchronize": (ctypes.c_int, [vp]),
        "flb_batch_destroy": (None, [vp]),
        "flb_get_state_device": (ctypes.c_int, [vp, vp]),
        "flb_set_state_device": (ctypes.c_int, [vp, vp]),
        "flb_adjoint_step": (ctypes.c_int, [vp, vp, ctypes.c_uint64, vp, vp, vp]),
        "flb_interface_heights": (ctypes.c_int, [vp, P(InterfaceFit), dp]),
        "flb_height_spectrum": (ctypes.c_int, [vp, P(InterfaceFit), dp, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc: int):
    if rc != FLB_OK:
        L = lib()
        raise FLBError(rc, f"{L.flb_error_string(rc).decode()}: {L.flb_last_error().decode()}")


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, n: int, name: str) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != n:
        raise ValueError(f"{name} must have {n} elements, got {a.size}")
    return a


def options(precision="fp32", rho0=1.0, replica=0, noise_rho_local=True, stream=None, device=-1,
            check_every=0, guard=False, z_chunk=0) -> Options:
    o = Options()
    lib().flb_default_options(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.rho0 = rho0
    o.replica = replica & 0xFFFFFFFF
    o.noise_rho_local = int(bool(noise_rho_local))
    o.stream = stream
    o.device = device
    o.check_every = check_every
    o.guard = int(guard)
    o.z_chunk = int(z_chunk)
    return o


class Context:
    """One periodic lattice on one GPU (``flb_create`` ... ``flb_destroy``)."""

    def __init__(self, lattice: int, dims, omega_shear: float, omega_bulk: float = 1.0,
                 omega_ghost: float = 1.0, kT: float = 0.0, free_energy: dict | None = None, seed: int = 1,
                 _handle=None, **opts):
        L = lib()
        if _handle is not None:
            self._h = _handle
        else:
            dims = list(dims) + [1] * (3 - len(dims))
            d = (ctypes.c_int * 3)(*dims)
            fe = FreeEnergy(0, 0.0, 0.0, 1.0, 0.0, 0, 0)
            if free_energy:
                fe = FreeEnergy(1, free_energy.get("A", 0.0), free_energy.get("B", 0.0),
                                free_energy.get("rho_c", 1.0), free_energy.get("kappa", 0.0),
                                int(bool(free_energy.get("total", False))), int(free_energy.get("model", 0)))
            o = options(**opts)
            h = ctypes.c_void_p()
            _check(L.flb_create(ctypes.byref(h), lattice, d, omega_shear, omega_bulk, omega_ghost, kT,
                                ctypes.byref(fe), seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(o)))
            self._h = h
        info = (ctypes.c_int * 6)()
        _check(L.flb_get_info(self._h, info))
        self.Q, self.D, self.X, self.Y, self.Z, self.precision = list(info)
        self.dims = (self.X, self.Y, self.Z)
        self.V = self.X * self.Y * self.Z

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().flb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state ---------------------------------------------------------------
    def init(self, rho=None, u=None, thermal: bool = False):
        r = None if rho is None else _f64(rho, self.V, "rho")
        uu = None if u is None else _f64(u, self.D * self.V, "u")
        _check(lib().flb_init(self._h, None if r is None else _dptr(r), None if uu is None else _dptr(uu),
                              int(bool(thermal))))

    def step(self, n: int = 1):
        _check(lib().flb_step(self._h, int(n)))

    def step_sums(self, nsteps: int = 1, out: np.ndarray | None = None) -> np.ndarray:
        """nsteps steps; (nsteps, 4) mass and momentum of the state each step starts from."""
        sums = out if out is not None else np.empty((nsteps, 4))
        _check(lib().flb_step_sums(self._h, int(nsteps), _dptr(sums)))
        return sums

    def step_sums_async(self, nsteps: int, out: np.ndarray) -> np.ndarray:
        """nsteps steps whose (nsteps, 4) sums land in `out` (a C-contiguous
        float64 array, ideally in page-locked memory) once the context's
        stream has been synchronised; returns without waiting."""
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size < 4 * nsteps:
            raise ValueError("out must be a C-contiguous float64 array of at least 4 * nsteps elements")
        _check(lib().flb_step_sums_async(self._h, int(nsteps), _dptr(out)))
        return out

    def get_populations(self) -> np.ndarray:
        f = np.empty((self.Q, self.V))
        _check(lib().flb_get_populations(self._h, _dptr(f)))
        return f

    def z_chunk(self):
        """(planes of z per block of the non-ideal D3Q19 step, still tuning?)"""
        n, t = ctypes.c_int(), ctypes.c_int()
        _check(lib().flb_z_chunk(self._h, ctypes.byref(n), ctypes.byref(t)))
        return n.value, bool(t.value)

    def check_guards(self):
        """Raise FLBError (FLB_EBOUNDS) if a kernel wrote outside a guarded buffer."""
        _check(lib().flb_check_guards(self._h))

    def get_sites(self, sites) -> np.ndarray:
        """(Q, n) pre-collision populations at the given site indices."""
        idx = np.ascontiguousarray(sites, dtype=np.int64).ravel()
        f = np.empty((self.Q, idx.size))
        _check(lib().flb_get_sites(self._h, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), idx.size,
                                   _dptr(f)))
        return f

    def set_populations(self, f):
        f = _f64(f, self.Q * self.V, "f")
        _check(lib().flb_set_populations(self._h, _dptr(f)))

    @property
    def step_count(self) -> int:
        s = ctypes.c_uint64()
        _check(lib().flb_get_step(self._h, ctypes.byref(s)))
        return s.value

    @step_count.setter
    def step_count(self, v: int):
        _check(lib().flb_set_step(self._h, int(v)))

    # -- observables ---------------------------------------------------------
    def moments(self, which: int, out: np.ndarray | None = None) -> np.ndarray:
        """Observable `which` of the current state; `out` (float64, C-contiguous,
        e.g. pinned memory) receives it when given."""
        n = {RHO: self.V, U: self.D * self.V, MODES: self.Q * self.V, MODE_VAR: self.Q}[which]
        if out is None:
            out = np.empty(n)
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != n:
            raise ValueError(f"out must be a C-contiguous float64 array of {n} elements")
        _check(lib().flb_moments(self._h, _dptr(out), which))
        out = out.reshape(-1)
        if which == U:
            return out.reshape(self.D, self.V)
        if which == MODES:
            return out.reshape(self.Q, self.V)
        return out

    def structure_factor(self, mode: int = 0, accumulate: bool = False, fetch: bool = True):
        S = np.empty(self.V) if fetch else None
        _check(lib().flb_structure_factor(self._h, None if S is None else _dptr(S), mode, int(bool(accumulate))))
        return S

    def interface_heights(self, fit: InterfaceFit) -> np.ndarray:
        """(2, X) heights of the lower and upper interface of a D2Q9 stripe."""
        h = np.empty(2 * self.dims[0])
        _check(lib().flb_interface_heights(self._h, ctypes.byref(fit), _dptr(h)))
        return h.reshape(2, -1)

    def height_spectrum(self, fit: InterfaceFit, accumulate: bool = False, fetch: bool = True):
        S = np.empty(self.dims[0]) if fetch else None
        _check(lib().flb_height_spectrum(self._h, ctypes.byref(fit), None if S is None else _dptr(S),
                                         int(bool(accumulate))))
        return S

    def snapshot_count(self, mode: int) -> int:
        c = ctypes.c_int()
        _check(lib().flb_snapshot_count(self._h, mode, ctypes.byref(c)))
        return c.value

    def reset_accumulators(self):
        _check(lib().flb_reset_accumulators(self._h))

    def conservation(self) -> np.ndarray:
        out = np.zeros(4)
        _check(lib().flb_conservation(self._h, _dptr(out)))
        return out

    # -- execution -----------------------------------------------------------
    def set_stream(self, stream_ptr: int | None):
        _check(lib().flb_set_stream(self._h, stream_ptr))

    def synchronize(self):
        _check(lib().flb_synchronize(self._h))

    def kernel_timing(self, enable: bool = True):
        _check(lib().flb_kernel_timing(self._h, int(bool(enable))))

    def kernel_times(self):
        ms = np.zeros(NKERNEL_TIMERS)
        n = (ctypes.c_int * NKERNEL_TIMERS)()
        _check(lib().flb_kernel_times(self._h, _dptr(ms), n))
        return ms, np.array(list(n))

    # -- device state and adjoint (pointers are device addresses) -----------
    def get_state_device(self, ptr: int):
        _check(lib().flb_get_state_device(self._h, ctypes.c_void_p(ptr)))

    def set_state_device(self, ptr: int):
        _check(lib().flb_set_state_device(self._h, ctypes.c_void_p(ptr)))

    def adjoint_step(self, g_n: int, step: int, lam_next: int, lam: int, grad: int):
        _check(lib().flb_adjoint_step(self._h, ctypes.c_void_p(g_n), int(step), ctypes.c_void_p(lam_next),
                                      ctypes.c_void_p(lam), ctypes.c_void_p(grad)))

    def adjoint_segment(self, g_start: int, step0: int, n: int, states: int, lam: int, grad: int):
        _check(lib().flb_adjoint_segment(self._h, ctypes.c_void_p(g_start), int(step0), int(n),
                                         ctypes.c_void_p(states), ctypes.c_void_p(lam), ctypes.c_void_p(grad)))

    # -- checkpoints ---------------------------------------------------------
    def save(self, path: str):
        _check(lib().flb_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path: str, **opts) -> "Context":
        h = ctypes.c_void_p()
        o = options(**opts)
        _check(lib().flb_load(ctypes.byref(h), os.fsencode(path), ctypes.byref(o)))
        return cls(0, (1, 1, 1), 1.0, _handle=h)


class Batch:
    """Independent D3Q19 ideal-gas replicas of uneven sizes (``flb_batch_*``)."""

    def __init__(self, dims, omega_shear, kT, seeds, omega_bulk=None, omega_ghost=None, **opts):
        L = lib()
        n = len(dims)
        d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(n, 3))
        f = lambda v: None if v is None else _dptr(_f64(v, n, "per-replica value"))
        self._keep = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) if v is not None else None
                      for v in (omega_shear, omega_bulk, omega_ghost, kT)]
        sd = (ctypes.c_uint64 * n)(*[int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds])
        o = options(**opts)
        h = ctypes.c_void_p()
        oms, omb, omg, kts = self._keep
        _check(L.flb_batch_create(ctypes.byref(h), D3Q19, n, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                  _dptr(oms), None if omb is None else _dptr(omb), None if omg is None else _dptr(omg),
                                  _dptr(kts), sd, ctypes.byref(o)))
        self._h = h
        self.n = n
        self.dims = [tuple(int(v) for v in row) for row in d]

    def close(self):
        if getattr(self, "_h", None):
            lib().flb_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init(self, thermal=False):
        _check(lib().flb_batch_init(self._h, int(bool(thermal))))

    def step(self, n=1):
        _check(lib().flb_batch_step(self._h, int(n)))

    def autotune(self):
        sh = np.zeros((self.n, 3), dtype=np.int32)
        _check(lib().flb_batch_autotune(self._h, sh.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return sh

    def mode_variance(self):
        out = np.zeros((self.n, 19))
        _check(lib().flb_batch_mode_variance(self._h, _dptr(out)))
        return out

    def structure_factor(self, replica, mode=0, accumulate=False, fetch=True):
        """S_a(k) of one replica; with fetch=False (and accumulate=True) the
        snapshot only goes into the device accumulator and None is returned."""
        X, Y, Z = self.dims[replica]
        S = np.empty(X * Y * Z) if fetch else None
        _check(lib().flb_batch_structure_factor(self._h, replica, None if S is None else _dptr(S), mode,
                                                int(bool(accumulate))))
        return S

    def get_populations(self, replica):
        X, Y, Z = self.dims[replica]
        f = np.empty((19, X * Y * Z))
        _check(lib().flb_batch_get_populations(self._h, replica, _dptr(f)))
        return f

    def info(self):
        n = ctypes.c_int()
        s = ctypes.c_longlong()
        st = ctypes.c_uint64()
        _check(lib().flb_batch_info(self._h, ctypes.byref(n), ctypes.byref(s), ctypes.byref(st)))
        return n.value, s.value, st.value

    def synchronize(self):
        _check(lib().flb_batch_synchronize(self._h))


__all__ = ["Context", "Batch", "FLBError", "lib", "options", "EXPORTS", "D2Q9", "D3Q19", "FP64", "FP32", "BF16",
           "RHO", "U", "MODES", "MODE_VAR"]
