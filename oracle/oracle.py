"""TEST INFRASTRUCTURE: ctypes front end of the FP64 C oracle (vlbm_oracle.c).

Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
use this module. It never imports the CUDA library, and the CUDA library never
imports it.

Time stepping follows the numerical section of the paper: a^n = 2 lambda^n /
(1 - alpha) (= 4 lambda^n at alpha = 1/2, the critical case of Bouchut's
criterion), Delta t^n = dx / a^n, populations initialised as u_k^0 = M_k(u_0)
with a^0. With a fixed lambda the kinetic speed is held at 2 lambda/(1-alpha)
(the entropy-wave run of Sec. 4.1 uses a = 10.7). With a final time, the last
step is shortened to land on it: Delta t = t_end - t and a = dx / Delta t, which
is still >= the Bouchut speed.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vlbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

LIM_FIRST, LIM_SECOND, LIM_PP, LIM_LMP, LIM_RLMP = range(5)
BC_PERIODIC, BC_ZEROGRAD, BC_REFLECT = range(3)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC[:-2] + ".h"))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               _SRC, "-o", _LIB_PATH, "-lm"])
    return _LIB_PATH


class _Field(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_double * 4), ("out", ctypes.c_double * 4), ("nplanes", ctypes.c_int),
                ("nx", ctypes.c_double * 2), ("ny", ctypes.c_double * 2), ("c0", ctypes.c_double * 2),
                ("c1", ctypes.c_double * 2)]


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("bc", ctypes.c_int * 4),
                ("limiter", ctypes.c_int), ("gamma", ctypes.c_double),
                ("alpha", ctypes.c_double), ("eps", ctypes.c_double), ("sponge", ctypes.c_int),
                ("bc_hi", ctypes.c_int * 4), ("split", ctypes.c_int * 4),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("dx", ctypes.c_double),
                ("field", ctypes.POINTER(_Field))]


_DBG_FIELDS = ["theta_x", "theta_y", "theta_rho_x", "theta_rho_y", "theta_p_x", "theta_p_y",
               "ustar_x", "ustar_y", "dflux_x", "dflux_y", "mu", "nu"]


class _Debug(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_double)) for n in _DBG_FIELDS]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D, P, I = ctypes.c_double, ctypes.c_void_p, ctypes.c_int
        _lib.orc_max_speed.restype = D
        _lib.orc_max_speed.argtypes = [P, P]
        _lib.orc_init_populations.argtypes = [P, D, P]
        _lib.orc_step.argtypes = [P, D, D, P, P, P]
        _lib.orc_step_fv.argtypes = [P, D, D, P, P]
        _lib.orc_fill_ghosts.argtypes = [P, D, D, P, P]
        _lib.orc_theta_p.restype = D
        _lib.orc_theta_p.argtypes = [D, D, P, P]
        _lib.orc_gql_radius.restype = D
        _lib.orc_gql_radius.argtypes = [P, P]
        _lib.orc_theta_rho_pp.restype = D
        _lib.orc_theta_rho_pp.argtypes = [D, D, D, D]
        _lib.orc_theta_rho_lmp.restype = D
        _lib.orc_theta_rho_lmp.argtypes = [D, D, D, D, D, D, D]
        _lib.orc_maxwellians.argtypes = [D, D, D, P, P]
        _lib.orc_flux_x.argtypes = [D, P, P]
        _lib.orc_flux_y.argtypes = [D, P, P]
        _lib.orc_set_threads.argtypes = [I]
        _lib.orc_get_threads.restype = I
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Field:
    """Prescribed boundary field (BC_DIRICHLET parts): at time t the ghost cell with
    centre (x, y) holds conserved state `inside` if nx[k] x + ny[k] y >= c0[k] + c1[k] t
    for every half-plane k, else `outside`."""
    inside: tuple
    outside: tuple
    planes: tuple = ()    # up to two (nx, ny, c0, c1)

    def c(self) -> _Field:
        f = _Field()
        f.in_[:] = [float(v) for v in self.inside]
        f.out[:] = [float(v) for v in self.outside]
        f.nplanes = len(self.planes)
        for k, (a, b, c0, c1) in enumerate(self.planes):
            f.nx[k], f.ny[k], f.c0[k], f.c1[k] = a, b, c0, c1
        return f


@dataclass
class Config:
    nx: int
    ny: int
    bc: tuple = (0, 0, 0, 0)
    limiter: int = LIM_PP
    gamma: float = 1.4
    alpha: float = 0.5
    eps: float = 1e-16
    sponge: int = 0       # Sec. 4.2: theta = 0 within `sponge` cells of a zero-gradient side
    bc_hi: tuple | None = None     # per side: type at and past split[s] (None: = bc)
    split: tuple = (0, 0, 0, 0)    # per side: index along it where the type switches (0: none)
    x0: float = 0.0
    y0: float = 0.0
    dx: float = 1.0
    field: Field | None = None

    def c(self) -> _Cfg:
        hi = self.bc if self.bc_hi is None else self.bc_hi
        cf = _Cfg(self.nx, self.ny, (ctypes.c_int * 4)(*self.bc), self.limiter,
                  self.gamma, self.alpha, self.eps, self.sponge, (ctypes.c_int * 4)(*hi),
                  (ctypes.c_int * 4)(*self.split), self.x0, self.y0, self.dx, None)
        if self.field is not None:
            cf._field_keep = self.field.c()      # keep the struct alive with the config
            cf.field = ctypes.pointer(cf._field_keep)
        return cf


def kinetic_speed(lam: float, alpha: float) -> float:
    """a = 2 lambda / (1 - alpha): the critical case of the Bouchut criterion."""
    return 2.0 * lam / (1.0 - alpha)


def flux_x(u, gamma=1.4):
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.zeros(4)
    lib().orc_flux_x(gamma, _ptr(u), _ptr(f))
    return f


def flux_y(u, gamma=1.4):
    u = np.ascontiguousarray(u, dtype=np.float64)
    g = np.zeros(4)
    lib().orc_flux_y(gamma, _ptr(u), _ptr(g))
    return g


def maxwellians(u, a, gamma=1.4, alpha=0.5) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    M = np.zeros((5, 4))
    lib().orc_maxwellians(gamma, alpha, a, _ptr(u), _ptr(M))
    return M


def theta_p(kappa, eps, ustar, dflux) -> float:
    us = np.ascontiguousarray(ustar, dtype=np.float64)
    df = np.ascontiguousarray(dflux, dtype=np.float64)
    return float(lib().orc_theta_p(kappa, eps, _ptr(us), _ptr(df)))


def gql_radius(ustar, dflux) -> float:
    us = np.ascontiguousarray(ustar, dtype=np.float64)
    df = np.ascontiguousarray(dflux, dtype=np.float64)
    return float(lib().orc_gql_radius(_ptr(us), _ptr(df)))


def theta_rho_pp(kappa, eps, rho_star, dflux_rho) -> float:
    return float(lib().orc_theta_rho_pp(kappa, eps, rho_star, dflux_rho))


def theta_rho_lmp(kappa, rho_star, dflux_rho, mu_l, nu_l, mu_r, nu_r) -> float:
    return float(lib().orc_theta_rho_lmp(kappa, rho_star, dflux_rho, mu_l, nu_l, mu_r, nu_r))


def new_state(cons: np.ndarray) -> np.ndarray:
    """(20, ny, nx) state with the conserved planes set and populations zero."""
    cons = np.asarray(cons, dtype=np.float64)
    s = np.zeros((20,) + cons.shape[1:])
    s[:4] = cons
    return s


def max_speed(cfg: Config, state: np.ndarray) -> float:
    state = np.ascontiguousarray(state)
    c = cfg.c()
    return float(lib().orc_max_speed(ctypes.byref(c), _ptr(state)))


def init_populations(cfg: Config, state: np.ndarray, a: float) -> np.ndarray:
    s = np.ascontiguousarray(state, dtype=np.float64).copy()
    c = cfg.c()
    lib().orc_init_populations(ctypes.byref(c), a, _ptr(s))
    return s


def step(cfg: Config, state: np.ndarray, a: float, debug: bool = False, fv: bool = False, t: float = 0.0):
    """One time step from time t (which only places the Dirichlet field) with kinetic
    speed a. Returns the new state (and a dict of per-face / per-cell intermediate
    values if debug)."""
    s = np.ascontiguousarray(state, dtype=np.float64)
    out = np.empty_like(s)
    c = cfg.c()
    if fv:
        rc = lib().orc_step_fv(ctypes.byref(c), a, t, _ptr(s), _ptr(out))
        if rc:
            raise ValueError("oracle rejected the configuration")
        return out
    dbg_arrays = None
    dbg_ptr = None
    if debug:
        nx, ny = cfg.nx, cfg.ny
        shp = {"theta_x": (ny, nx + 1), "theta_y": (ny + 1, nx),
               "theta_rho_x": (ny, nx + 1), "theta_rho_y": (ny + 1, nx),
               "theta_p_x": (ny, nx + 1), "theta_p_y": (ny + 1, nx),
               "ustar_x": (ny, nx + 1, 4), "ustar_y": (ny + 1, nx, 4),
               "dflux_x": (ny, nx + 1, 4), "dflux_y": (ny + 1, nx, 4),
               "mu": (ny, nx), "nu": (ny, nx)}
        dbg_arrays = {k: np.zeros(v) for k, v in shp.items()}
        d = _Debug(*[dbg_arrays[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
                     for k in _DBG_FIELDS])
        dbg_ptr = ctypes.byref(d)
    rc = lib().orc_step(ctypes.byref(c), a, t, _ptr(s), _ptr(out), dbg_ptr)
    if rc:
        raise ValueError("oracle rejected the configuration")
    return (out, dbg_arrays) if debug else out


def fill_ghosts(cfg: Config, state: np.ndarray, a: float, t: float = 0.0) -> np.ndarray:
    """The ghost fill alone: (20, ny + 4, nx + 4), cell (i, j) at [:, j + 2, i + 2]."""
    s = np.ascontiguousarray(state, dtype=np.float64)
    ext = np.empty((20, cfg.ny + 4, cfg.nx + 4))
    if lib().orc_fill_ghosts(ctypes.byref(cfg.c()), a, t, _ptr(s), _ptr(ext)):
        raise ValueError("oracle rejected the configuration")
    return ext


def run(cfg: Config, cons: np.ndarray, dx: float, nsteps: int | None = None,
        t_end: float | None = None, lam_fixed: float | None = None, fv: bool = False,
        callback=None, max_steps: int = 10 ** 9):
    """Advance initial conserved fields `cons` (4, ny, nx).

    Returns dict(state, t, n, a) with the list of kinetic speeds used. Stops after
    `nsteps`, or on reaching `t_end`; raises FloatingPointError if the state leaves
    the admissible set (lambda undefined)."""
    state = new_state(cons)
    if lam_fixed is not None and lam_fixed > 0:
        a_fixed = kinetic_speed(lam_fixed, cfg.alpha)
    else:
        a_fixed = None

    def speed(s):
        if a_fixed is not None:
            return a_fixed
        lam = max_speed(cfg, s)
        if not np.isfinite(lam):
            raise FloatingPointError("state left the admissible set")
        return kinetic_speed(lam, cfg.alpha)

    a = speed(state)
    state = init_populations(cfg, state, a)
    t, n, hist = 0.0, 0, []
    limit = nsteps if nsteps is not None else max_steps
    while n < limit:
        if n > 0:
            a = speed(state)
        dt = dx / a
        last = False
        if t_end is not None:
            if t >= t_end:
                break
            if t + dt >= t_end:
                dt = t_end - t
                a = dx / dt
                last = True
        state = step(cfg, state, a, fv=fv, t=t)
        hist.append(a)
        t = t + dt
        n += 1
        if callback is not None:
            callback(n, state)
        if last:
            break
    return {"state": state, "t": t, "n": n, "a": hist}
