"""FP64 CPU oracle of the fluctuating lattice Boltzmann update (arXiv 1012.3632).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library: the arithmetic lives in
``flb_oracle.c`` (plain C, double precision, one site at a time), and this
module only marshals numpy arrays through ctypes.

Arrays use the structure-of-arrays layout ``f[i, s]`` with the site index
``s = x + X*(y + Y*z)`` (x fastest) and hold the paper's pre-collision
populations f^LB(r, t) (Sec. V, Eq. (f-aux)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flb_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")


def build(force: bool = False) -> str:
    """Compile ``flb_oracle.c`` into ``liborc.so`` with gcc (no FMA contraction,
    so that x86 and Arm hosts round alike)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("Q", ctypes.c_int),
        ("X", ctypes.c_int), ("Y", ctypes.c_int), ("Z", ctypes.c_int),
        ("ox", ctypes.c_int), ("oy", ctypes.c_int), ("oz", ctypes.c_int),
        ("wx", ctypes.c_int), ("wy", ctypes.c_int), ("wz", ctypes.c_int),
        ("omega_shear", ctypes.c_double), ("omega_bulk", ctypes.c_double),
        ("omega_ghost", ctypes.c_double),
        ("kT", ctypes.c_double), ("rho0", ctypes.c_double),
        ("noise_rho_local", ctypes.c_int),
        ("nonideal", ctypes.c_int),
        ("A", ctypes.c_double), ("B", ctypes.c_double), ("rho_c", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("total", ctypes.c_int),
        ("model", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("replica", ctypes.c_uint32),
    ]


@dataclass(frozen=True)
class Params:
    """Model parameters.  ``dims`` is the global periodic lattice (X, Y, Z);
    ``origin``/``window`` select the sub-box held in the arrays (default: all
    of it).  Outside a full-lattice window, sites whose update needs data from
    beyond the window come out as NaN."""
    Q: int
    dims: tuple
    omega_shear: float = 1.0
    omega_bulk: float = 1.0
    omega_ghost: float = 1.0
    kT: float = 0.0
    rho0: float = 1.0
    noise_rho_local: bool = True
    nonideal: bool = False
    A: float = 0.0
    B: float = 0.0
    rho_c: float = 1.0
    kappa: float = 0.0
    total: bool = False
    model: int = 0  # 0 force-based, 1 modified equilibrium (D2Q9)
    seed: int = 1
    replica: int = 0
    origin: tuple = (0, 0, 0)
    window: tuple | None = None

    @property
    def wdims(self):
        return tuple(self.window) if self.window is not None else tuple(self.dims)

    @property
    def V(self):
        wx, wy, wz = self.wdims
        return wx * wy * wz

    @property
    def D(self):
        return 2 if self.Q == 9 else 3

    def c_struct(self) -> _Params:
        X, Y, Z = self.dims
        wx, wy, wz = self.wdims
        ox, oy, oz = self.origin
        return _Params(self.Q, X, Y, Z, ox, oy, oz, wx, wy, wz,
                       self.omega_shear, self.omega_bulk, self.omega_ghost,
                       self.kT, self.rho0, int(self.noise_rho_local), int(self.nonideal),
                       self.A, self.B, self.rho_c, self.kappa, int(self.total), int(self.model),
                       self.seed & 0xFFFFFFFFFFFFFFFF, self.replica & 0xFFFFFFFF)

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        L.orc_get_lattice.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp, dp, dp,
                                      ctypes.POINTER(ctypes.c_int)]
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.orc_philox4x32_10.restype = None
        L.orc_normals4.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, dp]
        L.orc_normals4.restype = None
        L.orc_collide_site.argtypes = [pp, dp, dp, ctypes.c_uint32, ctypes.c_uint64, dp]
        L.orc_density_force.argtypes = [pp, dp, dp, dp]
        L.orc_step.argtypes = [pp, ctypes.c_uint64, dp, dp]
        L.orc_run.argtypes = [pp, ctypes.c_uint64, ctypes.c_int, dp]
        L.orc_init.argtypes = [pp, dp, dp, ctypes.c_int, dp]
        L.orc_modes.argtypes = [pp, dp, dp]
        L.orc_velocity.argtypes = [pp, dp, dp]
        L.orc_dft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_structure_factor.argtypes = [pp, dp, ctypes.c_int, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc):
    if rc != 0:
        raise ValueError(f"oracle call failed ({rc})")


@dataclass
class Lattice:
    Q: int
    D: int
    c: np.ndarray      # (Q, 3) int
    w: np.ndarray      # (Q,)
    T: np.ndarray      # (Q, Q), T[a, i]
    N: np.ndarray      # (Q,)
    cls: np.ndarray    # (Q,) 0 conserved, 1 bulk, 2 shear, 3 ghost
    cs2: float = 1.0 / 3.0

    @property
    def Tinv(self):
        """(T^-1)_{ia} = w_i T_ai / N_a, Eq. (moments-inv)."""
        return (self.w[:, None] * self.T.T) / self.N[None, :]


def lattice(Q: int) -> Lattice:
    c = np.zeros(Q * 3, dtype=np.int32)
    w = np.zeros(Q)
    T = np.zeros(Q * Q)
    N = np.zeros(Q)
    cls = np.zeros(Q, dtype=np.int32)
    _check(lib().orc_get_lattice(Q, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w), _dp(T),
                                 _dp(N), cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
    return Lattice(Q, 2 if Q == 9 else 3, c.reshape(Q, 3), w, T.reshape(Q, Q), N, cls)


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def normals4(seed, site, step, call, tag, replica):
    z = np.zeros(4)
    lib().orc_normals4(seed & 0xFFFFFFFFFFFFFFFF, site, step & 0xFFFFFFFF, call, tag, replica, _dp(z))
    return z


def collide_site(p: Params, f, F, site: int, step: int) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    F3 = np.zeros(3)
    F3[: len(F)] = F
    out = np.zeros(p.Q)
    ps = p.c_struct()
    _check(lib().orc_collide_site(ctypes.byref(ps), _dp(f), _dp(F3), site, step, _dp(out)))
    return out


def init(p: Params, rho=None, u=None, thermal: bool = False) -> np.ndarray:
    """Initial pre-collision populations (Q, V): f^eq(rho, u) (+ thermal modes)."""
    V = p.V
    f = np.zeros((p.Q, V))
    r = None if rho is None else np.ascontiguousarray(np.reshape(rho, V), dtype=np.float64)
    uu = None if u is None else np.ascontiguousarray(np.reshape(u, (p.D, V)), dtype=np.float64)
    ps = p.c_struct()
    _check(lib().orc_init(ctypes.byref(ps), None if r is None else _dp(r),
                          None if uu is None else _dp(uu), int(thermal), _dp(f)))
    return f


def step(p: Params, f: np.ndarray, t: int) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    ps = p.c_struct()
    _check(lib().orc_step(ctypes.byref(ps), t, _dp(f), _dp(out)))
    return out


def run(p: Params, f: np.ndarray, step0: int, nsteps: int) -> np.ndarray:
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    ps = p.c_struct()
    _check(lib().orc_run(ctypes.byref(ps), step0, nsteps, _dp(f)))
    return f


def density_force(p: Params, f: np.ndarray):
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros(p.V)
    F = np.zeros((3, p.V))
    ps = p.c_struct()
    _check(lib().orc_density_force(ctypes.byref(ps), _dp(f), _dp(rho), _dp(F)))
    return rho, F


def modes(p: Params, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    m = np.zeros_like(f)
    ps = p.c_struct()
    _check(lib().orc_modes(ctypes.byref(ps), _dp(f), _dp(m)))
    return m


def velocity(p: Params, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    u = np.zeros((p.D, p.V))
    ps = p.c_struct()
    _check(lib().orc_velocity(ctypes.byref(ps), _dp(f), _dp(u)))
    return u


def dft(phi: np.ndarray) -> np.ndarray:
    """Naive separable DFT of a real field of shape (Z, Y, X) (or (Y, X))."""
    phi = np.asarray(phi, dtype=np.float64)
    shp = phi.shape
    phi = phi.reshape((1,) * (3 - phi.ndim) + shp)
    nz, ny, nx = phi.shape
    src = np.ascontiguousarray(phi).reshape(-1)
    re = np.zeros_like(src)
    im = np.zeros_like(src)
    _check(lib().orc_dft(nx, ny, nz, _dp(src), _dp(re), _dp(im)))
    return (re + 1j * im).reshape(shp)


def structure_factor(p: Params, f: np.ndarray, mode: int = 0) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    S = np.zeros(p.V)
    ps = p.c_struct()
    _check(lib().orc_structure_factor(ctypes.byref(ps), _dp(f), mode, _dp(S)))
    return S


__all__ = ["Params", "Lattice", "lattice", "build", "philox4x32_10", "normals4", "collide_site",
           "init", "step", "run", "density_force", "modes", "velocity", "dft", "structure_factor"]
