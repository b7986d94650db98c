"""Thin Python binding of libvlbm (include/vlbm.h).

The functions below carry the C names and only marshal arguments; every step of
the scheme runs in the CUDA library. The `VLBM` class adds PyTorch plumbing:
torch allocates the device workspace and supplies the stream. There is no CPU
fallback: if the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvlbm.so")

OK, E_INVAL, E_CUDA, E_POSITIVITY, E_NONFINITE, E_TIMEOUT, E_UNSUPPORTED, E_NOMEM = 0, -1, -2, -3, -4, -5, -6, -7
LIM_FIRST_ORDER, LIM_NONE, LIM_PP, LIM_LMP, LIM_RLMP = range(5)
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_DIRICHLET = range(4)
FP64, FP32 = 0, 1
ADJOINT_HOLD_A, ADJOINT_DIFF_A = 0, 1
KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_FUSED = range(3)

LIMITERS = {"first": LIM_FIRST_ORDER, "none": LIM_NONE, "pp": LIM_PP, "lmp": LIM_LMP, "rlmp": LIM_RLMP}


class vlbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("bc", ctypes.c_int32 * 4)]


class vlbm_field(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_double * 4), ("out", ctypes.c_double * 4), ("nplanes", ctypes.c_int32),
                ("nx", ctypes.c_double * 2), ("ny", ctypes.c_double * 2), ("c0", ctypes.c_double * 2),
                ("c1", ctypes.c_double * 2)]


class vlbm_boundary(ctypes.Structure):
    _fields_ = [("bc_hi", ctypes.c_int32 * 4), ("split", ctypes.c_int32 * 4), ("x0", ctypes.c_double),
                ("y0", ctypes.c_double), ("field", vlbm_field)]


class vlbm_opts(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("eps", ctypes.c_double), ("kernel", ctypes.c_int32),
                ("sponge", ctypes.c_int32), ("boundary", ctypes.POINTER(vlbm_boundary))]


def make_boundary(bc, bc_hi=None, split=(0, 0, 0, 0), x0=0.0, y0=0.0, field=None):
    """vlbm_boundary from per-side types and an optional prescribed field: `field` is
    (inside, outside, planes) with conserved 4-tuples and up to two half-planes
    (nx, ny, c0, c1), or an object with those attributes."""
    b = vlbm_boundary()
    b.bc_hi[:] = list(bc if bc_hi is None else bc_hi)
    b.split[:] = list(split)
    b.x0, b.y0 = float(x0), float(y0)
    if field is not None:
        inside, outside, planes = ((field.inside, field.outside, field.planes)
                                   if hasattr(field, "inside") else field)
        b.field.in_[:] = [float(v) for v in inside]
        b.field.out[:] = [float(v) for v in outside]
        b.field.nplanes = len(planes)
        for k, (a, c, c0, c1) in enumerate(planes):
            b.field.nx[k], b.field.ny[k], b.field.c0[k], b.field.c1[k] = a, c, c0, c1
    return b


def _opts(alpha, eps, kernel, sponge, boundary):
    o = vlbm_opts(alpha, eps, kernel, sponge, None)
    if boundary is not None:
        o._boundary_keep = boundary          # the struct must outlive the call that reads it
        o.boundary = ctypes.pointer(boundary)
    return o


class vlbm_monitor_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("t", ctypes.c_double), ("a", ctypes.c_double),
                ("dt", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("bad_cells", ctypes.c_int64), ("nonfinite_cells", ctypes.c_int64),
                ("first_bad_step", ctypes.c_int64), ("min_rho", ctypes.c_double),
                ("sum", ctypes.c_double * 4), ("theta_p_fp64_faces", ctypes.c_int64),
                ("done", ctypes.c_int32), ("status", ctypes.c_int32),
                ("min_internal_energy", ctypes.c_double)]


class vlbm_step_result(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("a_next", ctypes.c_double), ("min_rho", ctypes.c_double),
                ("sum", ctypes.c_double * 4), ("bad_cells", ctypes.c_int64),
                ("nonfinite_cells", ctypes.c_int64), ("theta_p_fp64_faces", ctypes.c_int64)]


class vlbm_batch_tuning(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("order", ctypes.c_int32),
                ("items", ctypes.c_int32), ("ctas", ctypes.c_int32)]


ORDER_LPT, ORDER_INDEX, ORDER_GUIDED = 0, 1, 2


class VLBMError(RuntimeError):
    def __init__(self, code: int, detail: str = ""):
        self.code = code
        super().__init__(f"{vlbm_strerror(code)} ({code}): {detail}")


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2411_15001_gb300.build` "
                      "(or __graft_entry__.build()). There is no CPU fallback.")

_lib = ctypes.CDLL(LIB_PATH)
_P, _I32, _I64, _D, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t

_SIGS = {
    "vlbm_workspace_bytes": (_SZ, [ctypes.POINTER(vlbm_grid), _I32]),
    "vlbm_init": (ctypes.c_int, [ctypes.POINTER(vlbm_grid), _D, _D, _I32, _I32, ctypes.POINTER(vlbm_opts),
                                 _P, _SZ, _P, ctypes.POINTER(_P)]),
    "vlbm_set_conserved": (ctypes.c_int, [_P, _P, _P, _P]),
    "vlbm_step": (ctypes.c_int, [_P, _I64]),
    "vlbm_step_to": (ctypes.c_int, [_P, _D, _I64]),
    "vlbm_moments": (ctypes.c_int, [_P, _P, _P, _P]),
    "vlbm_monitors": (ctypes.c_int, [_P, ctypes.POINTER(vlbm_monitor_t)]),
    "vlbm_monitors_raw_bytes": (_SZ, []),
    "vlbm_monitors_async": (ctypes.c_int, [_P, _P]),
    "vlbm_monitors_decode": (ctypes.c_int, [_P, ctypes.POINTER(vlbm_monitor_t)]),
    "vlbm_sync": (ctypes.c_int, [_P]),
    "vlbm_time": (ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "vlbm_checkpoint_bytes": (_SZ, [_P]),
    "vlbm_save": (ctypes.c_int, [_P, _P]),
    "vlbm_load": (ctypes.c_int, [_P, _P]),
    "vlbm_profile": (ctypes.c_int, [_P, _I32]),
    "vlbm_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(_D), ctypes.POINTER(_I64)]),
    "vlbm_step_noalloc": (ctypes.c_int, [ctypes.POINTER(vlbm_grid), _D, _D, _I32, _I32,
                                         ctypes.POINTER(vlbm_opts), _P, _P,
                                         ctypes.POINTER(vlbm_step_result), _P]),
    "vlbm_adjoint_scratch_bytes": (_SZ, [_P, _I64, _I32]),
    "vlbm_rollout": (ctypes.c_int, [_P, _I64, _I32, _P, _SZ]),
    "vlbm_adjoint": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P, _SZ]),
    "vlbm_adjoint_set_mode": (ctypes.c_int, [_P, _I32]),
    "vlbm_batch_workspace_bytes": (_SZ, [_I32, ctypes.POINTER(vlbm_grid), _I32]),
    "vlbm_batch_init": (ctypes.c_int, [_I32, ctypes.POINTER(vlbm_grid), _D, _I32, _I32,
                                       ctypes.POINTER(vlbm_opts), _P, _SZ, _P, ctypes.POINTER(_P)]),
    "vlbm_batch_set_conserved": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "vlbm_batch_step": (ctypes.c_int, [_P, _I64]),
    "vlbm_batch_moments": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "vlbm_batch_save": (ctypes.c_int, [_P, _I32, _P]),
    "vlbm_batch_monitors": (ctypes.c_int, [_P, _I32, ctypes.POINTER(vlbm_monitor_t)]),
    "vlbm_batch_get_tuning": (ctypes.c_int, [_P, ctypes.POINTER(vlbm_batch_tuning)]),
    "vlbm_batch_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(vlbm_batch_tuning)]),
    "vlbm_batch_autotune": (ctypes.c_int, [_P, _I32, ctypes.POINTER(vlbm_batch_tuning), ctypes.POINTER(_D)]),
    "vlbm_batch_destroy": (None, [_P]),
    "vlbm_batch_last_error": (ctypes.c_char_p, [_P]),
    "vlbm_destroy": (None, [_P]),
    "vlbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "vlbm_last_error_detail": (ctypes.c_int, [_P, ctypes.c_char_p, _SZ]),
    # test hooks (include/vlbm_testing.h)
    "vlbm_test_theta_faces": (ctypes.c_int, [_I64, _D, _D, _D, _P, _P, _P, _P]),
    "vlbm_test_wait_probe": (ctypes.c_int, [_P, ctypes.c_uint32]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def library():
    return _lib


# ------------------------------------------------------------------ C-named calls
def vlbm_workspace_bytes(grid: vlbm_grid, precision: int) -> int:
    return int(_lib.vlbm_workspace_bytes(ctypes.byref(grid), precision))


def vlbm_init(grid, gamma, lam, limiter, precision, opts, d_workspace, workspace_bytes, stream):
    out = _P()
    rc = _lib.vlbm_init(ctypes.byref(grid), gamma, lam, limiter, precision,
                        ctypes.byref(opts) if opts is not None else None,
                        d_workspace, workspace_bytes, stream, ctypes.byref(out))
    return rc, out


def vlbm_set_conserved(s, d_rho, d_mom, d_E) -> int:
    return _lib.vlbm_set_conserved(s, d_rho, d_mom, d_E)


def vlbm_step(s, nsteps: int) -> int:
    return _lib.vlbm_step(s, nsteps)


def vlbm_step_to(s, t_end: float, max_steps: int) -> int:
    return _lib.vlbm_step_to(s, t_end, max_steps)


def vlbm_moments(s, d_rho, d_mom, d_E) -> int:
    return _lib.vlbm_moments(s, d_rho, d_mom, d_E)


def vlbm_monitors(s):
    m = vlbm_monitor_t()
    rc = _lib.vlbm_monitors(s, ctypes.byref(m))
    return rc, m


def vlbm_monitors_raw_bytes() -> int:
    return int(_lib.vlbm_monitors_raw_bytes())


def vlbm_monitors_async(s, h_dst) -> int:
    return _lib.vlbm_monitors_async(s, h_dst)


def vlbm_monitors_decode(h_src):
    m = vlbm_monitor_t()
    rc = _lib.vlbm_monitors_decode(h_src, ctypes.byref(m))
    return rc, m


def vlbm_sync(s) -> int:
    return _lib.vlbm_sync(s)


def vlbm_time(s):
    t, n = _D(), _I64()
    rc = _lib.vlbm_time(s, ctypes.byref(t), ctypes.byref(n))
    return rc, t.value, n.value


def vlbm_checkpoint_bytes(s) -> int:
    return int(_lib.vlbm_checkpoint_bytes(s))


def vlbm_save(s, d_dst) -> int:
    return _lib.vlbm_save(s, d_dst)


def vlbm_load(s, d_src) -> int:
    return _lib.vlbm_load(s, d_src)


def vlbm_profile(s, enable: bool) -> int:
    return _lib.vlbm_profile(s, 1 if enable else 0)


def vlbm_profile_read(s):
    ms, n = _D(), _I64()
    rc = _lib.vlbm_profile_read(s, ctypes.byref(ms), ctypes.byref(n))
    return rc, ms.value, n.value


def vlbm_step_noalloc(grid, gamma, a, limiter, precision, opts, d_in, d_out, stream):
    """One workspace-free step (see include/vlbm.h); returns (rc, vlbm_step_result)."""
    r = vlbm_step_result()
    rc = _lib.vlbm_step_noalloc(ctypes.byref(grid), gamma, a, limiter, precision,
                                ctypes.byref(opts) if opts is not None else None, d_in, d_out,
                                ctypes.byref(r), stream)
    return rc, r


def vlbm_adjoint_scratch_bytes(s, nsteps: int, ckpt_every: int) -> int:
    return int(_lib.vlbm_adjoint_scratch_bytes(s, nsteps, ckpt_every))


def vlbm_rollout(s, nsteps: int, ckpt_every: int, d_scratch, scratch_bytes: int) -> int:
    return _lib.vlbm_rollout(s, nsteps, ckpt_every, d_scratch, scratch_bytes)


def vlbm_adjoint_set_mode(s, mode: int) -> int:
    return _lib.vlbm_adjoint_set_mode(s, mode)


def vlbm_adjoint(s, d_u0, nsteps: int, ckpt_every: int, d_dLduN, d_dLdu0, d_scratch, scratch_bytes: int) -> int:
    return _lib.vlbm_adjoint(s, d_u0, nsteps, ckpt_every, d_dLduN, d_dLdu0, d_scratch, scratch_bytes)


def vlbm_batch_workspace_bytes(grids, precision) -> int:
    arr = (vlbm_grid * len(grids))(*grids)
    return int(_lib.vlbm_batch_workspace_bytes(len(grids), arr, precision))


def vlbm_batch_init(grids, gamma, limiter, precision, opts, d_workspace, workspace_bytes, stream):
    arr = (vlbm_grid * len(grids))(*grids)
    out = _P()
    rc = _lib.vlbm_batch_init(len(grids), arr, gamma, limiter, precision,
                              ctypes.byref(opts) if opts is not None else None, d_workspace,
                              workspace_bytes, stream, ctypes.byref(out))
    return rc, out


def vlbm_batch_set_conserved(b, i, d_rho, d_mom, d_E) -> int:
    return _lib.vlbm_batch_set_conserved(b, i, d_rho, d_mom, d_E)


def vlbm_batch_step(b, nsteps: int) -> int:
    return _lib.vlbm_batch_step(b, nsteps)


def vlbm_batch_moments(b, i, d_rho, d_mom, d_E) -> int:
    return _lib.vlbm_batch_moments(b, i, d_rho, d_mom, d_E)


def vlbm_batch_save(b, i, d_dst) -> int:
    return _lib.vlbm_batch_save(b, i, d_dst)


def vlbm_batch_monitors(b, i):
    m = vlbm_monitor_t()
    rc = _lib.vlbm_batch_monitors(b, i, ctypes.byref(m))
    return rc, m


def vlbm_batch_get_tuning(b):
    t = vlbm_batch_tuning()
    rc = _lib.vlbm_batch_get_tuning(b, ctypes.byref(t))
    return rc, t


def vlbm_batch_set_tuning(b, t) -> int:
    return _lib.vlbm_batch_set_tuning(b, ctypes.byref(t))


def vlbm_batch_autotune(b, trial_steps: int):
    t = vlbm_batch_tuning()
    ms = _D()
    rc = _lib.vlbm_batch_autotune(b, trial_steps, ctypes.byref(t), ctypes.byref(ms))
    return rc, t, ms.value


def vlbm_batch_destroy(b) -> None:
    _lib.vlbm_batch_destroy(b)


def vlbm_batch_last_error(b) -> str:
    r = _lib.vlbm_batch_last_error(b)
    return r.decode() if r else ""


def vlbm_destroy(s) -> None:
    _lib.vlbm_destroy(s)


def vlbm_strerror(code: int) -> str:
    return _lib.vlbm_strerror(code).decode()


def vlbm_last_error_detail(s=None) -> str:
    buf = ctypes.create_string_buffer(256)
    _lib.vlbm_last_error_detail(s, buf, 256)
    return buf.value.decode()


THETA_STAGE_NONE, THETA_STAGE_SCREEN, THETA_STAGE_INTERVAL, THETA_STAGE_FP64 = range(4)


def vlbm_test_theta_faces(n: int, a: float, alpha: float, eps: float, d_faces, d_theta, d_stage, stream) -> int:
    """FP32 theta of n caller-supplied faces (test hook, include/vlbm_testing.h)."""
    return _lib.vlbm_test_theta_faces(n, a, alpha, eps, d_faces, d_theta, d_stage, stream)


def vlbm_test_wait_probe(s, limit_ns: int) -> int:
    """Arm (limit_ns > 0) or disarm the row-marching kernel's wait probe (test hook)."""
    return _lib.vlbm_test_wait_probe(s, limit_ns)


def _check(rc: int, s=None) -> int:
    if rc != OK:
        raise VLBMError(rc, vlbm_last_error_detail(s))
    return rc


# ------------------------------------------------------------------ torch front end
class _StreamOrder:
    """Orders a library call on the solver's stream against torch's current stream of
    the device: the solver's stream first waits for the work already enqueued on the
    current stream (so the inputs the caller just produced are complete), and the
    current stream then waits for the call's work (so outputs are complete, and
    inputs and scratch freed afterwards through the caching allocator are not reused
    while the call still reads them). Nothing is done when the two are the same stream."""

    def __init__(self, owner):
        self.owner = owner

    def __enter__(self):
        t = self.owner.torch
        self.cur = t.cuda.current_stream(self.owner.device)
        self.same = self.cur == self.owner.stream
        if not self.same:
            self.owner.stream.wait_stream(self.cur)
        return self

    def __exit__(self, *exc):
        if not self.same:
            self.cur.wait_stream(self.owner.stream)
        return False


class VLBM:
    """One 2D grid advanced by the blended D2Q5 vectorial LBM on a CUDA device.

    Device memory (the workspace, inputs, outputs) is torch-allocated; the stream
    is torch's current stream of `device` unless one is given.
    """

    def __init__(self, nx: int, ny: int, dx: float, bc=(0, 0, 0, 0), gamma: float = 1.4,
                 lam: float = 0.0, limiter=LIM_PP, precision=FP32, alpha: float = 0.5,
                 eps: float = 1e-16, kernel=KERNEL_AUTO, device=None, stream=None, sponge: int = 0,
                 boundary: "vlbm_boundary | None" = None):
        import torch

        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if isinstance(limiter, str):
            limiter = LIMITERS[limiter.lower()]
        self.nx, self.ny, self.dx = nx, ny, dx
        self.precision = precision
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self.grid = vlbm_grid(nx, ny, dx, (ctypes.c_int32 * 4)(*bc))
        self.opts = _opts(alpha, eps, kernel, sponge, boundary)
        nbytes = vlbm_workspace_bytes(self.grid, precision)
        if nbytes == 0:
            raise VLBMError(E_INVAL, "invalid grid")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace.record_stream(self.stream)
        rc, self._s = vlbm_init(self.grid, gamma, lam, limiter, precision, self.opts,
                                self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        _check(rc)

    def _ptr(self, t):
        if t is None:
            return None
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError("tensor must be contiguous, on the solver's device, in its dtype")
        return t.data_ptr()

    def set_conserved(self, rho, mom, E):
        """rho, E: (ny, nx); mom: (2, ny, nx) -- device tensors in the solver's dtype."""
        with _StreamOrder(self):
            _check(vlbm_set_conserved(self._s, self._ptr(rho), self._ptr(mom), self._ptr(E)), self._s)

    def step(self, nsteps: int = 1):
        with _StreamOrder(self):
            _check(vlbm_step(self._s, int(nsteps)), self._s)

    def step_to(self, t_end: float, max_steps: int = 10 ** 9) -> int:
        with _StreamOrder(self):
            rc = vlbm_step_to(self._s, float(t_end), int(max_steps))
        return _check(rc, self._s)

    def moments(self):
        t = self.torch
        rho = t.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        mom = t.empty((2, self.ny, self.nx), dtype=self.dtype, device=self.device)
        E = t.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        with _StreamOrder(self):
            _check(vlbm_moments(self._s, rho.data_ptr(), mom.data_ptr(), E.data_ptr()), self._s)
        return rho, mom, E

    @staticmethod
    def _monitor_dict(m) -> dict:
        return {"status": m.status, "n": m.n, "t": m.t, "a": m.a, "dt": m.dt, "lambda": m.lambda_,
                "bad_cells": m.bad_cells, "nonfinite_cells": m.nonfinite_cells,
                "first_bad_step": m.first_bad_step, "min_rho": m.min_rho, "sum": list(m.sum),
                "theta_p_fp64_faces": m.theta_p_fp64_faces,
                "min_internal_energy": m.min_internal_energy, "done": m.done}

    def monitors(self) -> dict:
        rc, m = vlbm_monitors(self._s)
        if rc == E_CUDA:
            _check(rc, self._s)
        return self._monitor_dict(m)

    def monitor_buffer(self):
        """A pinned host buffer for monitors_async (vlbm_monitors_raw_bytes bytes)."""
        return self.torch.empty(vlbm_monitors_raw_bytes(), dtype=self.torch.uint8).pin_memory()

    def monitors_async(self, buf):
        """Enqueue on the solver's stream a copy of the monitors, as the work enqueued so far
        leaves them, into the pinned buffer `buf` (vlbm_monitors_async); read them with
        decode_monitors(buf) once the copy has completed."""
        with _StreamOrder(self):
            _check(vlbm_monitors_async(self._s, buf.data_ptr()), self._s)

    def decode_monitors(self, buf) -> dict:
        rc, m = vlbm_monitors_decode(buf.data_ptr())
        return self._monitor_dict(m)

    def sync(self) -> int:
        return vlbm_sync(self._s)

    def time(self):
        rc, t, n = vlbm_time(self._s)
        if rc == E_CUDA:
            _check(rc, self._s)
        return t, n

    def save(self):
        buf = self.torch.empty(vlbm_checkpoint_bytes(self._s), dtype=self.torch.uint8, device=self.device)
        with _StreamOrder(self):
            _check(vlbm_save(self._s, buf.data_ptr()), self._s)
        return buf

    def load(self, buf):
        with _StreamOrder(self):
            _check(vlbm_load(self._s, buf.data_ptr()), self._s)

    def state_planes(self):
        """(20, ny, nx) copy of the current state (u, then u_1..u_4) via a checkpoint."""
        buf = self.save()
        return buf[64:].view(self.dtype).view(20, self.ny, self.nx)

    def profile(self, enable: bool = True):
        """Time every step kernel with a CUDA event pair (see vlbm_profile)."""
        _check(vlbm_profile(self._s, enable), self._s)

    def profile_read(self):
        """(summed step-kernel milliseconds, number of timed launches); waits for the stream."""
        rc, ms, n = vlbm_profile_read(self._s)
        _check(rc, self._s)
        return ms, n

    def adjoint_scratch(self, nsteps: int, ckpt_every: int):
        """Device scratch for vlbm_rollout / vlbm_adjoint with these arguments."""
        n = vlbm_adjoint_scratch_bytes(self._s, int(nsteps), int(ckpt_every))
        if n == 0:
            raise VLBMError(E_INVAL, "invalid rollout arguments")
        return self.torch.empty(n, dtype=self.torch.uint8, device=self.device)

    def rollout(self, nsteps: int, ckpt_every: int, scratch):
        """Advance nsteps from the state set_conserved left, checkpointing into scratch."""
        with _StreamOrder(self):
            _check(vlbm_rollout(self._s, int(nsteps), int(ckpt_every), scratch.data_ptr(), scratch.numel()),
                   self._s)

    def set_adjoint_mode(self, mode: int):
        """ADJOINT_HOLD_A (default) or ADJOINT_DIFF_A: whether the adjoint differentiates
        the dynamic kinetic speed a^n = 2 max lambda / (1 - alpha)."""
        _check(vlbm_adjoint_set_mode(self._s, int(mode)), self._s)

    def adjoint(self, dLduN, nsteps: int, ckpt_every: int, scratch, u0=None):
        """dL/du_0 (4, ny, nx) from dL/du^N (4, ny, nx): planes rho, m1, m2, E.

        With u0 the call sets the state from it and runs the rollout itself; without
        it, the checkpoints of the preceding rollout (same arguments) are used."""
        g = self.torch.empty((4, self.ny, self.nx), dtype=self.dtype, device=self.device)
        with _StreamOrder(self):
            _check(vlbm_adjoint(self._s, self._ptr(u0), int(nsteps), int(ckpt_every), self._ptr(dLduN),
                                g.data_ptr(), scratch.data_ptr(), scratch.numel()), self._s)
        return g

    def close(self):
        if getattr(self, "_s", None):
            vlbm_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VLBMBatch:
    """Independent grids of uneven sizes advanced together (vlbm_batch_*)."""

    def __init__(self, grids, gamma: float = 1.4, limiter=LIM_PP, precision=FP32,
                 alpha: float = 0.5, eps: float = 1e-16, device=None, stream=None, sponge: int = 0,
                 boundary: "vlbm_boundary | None" = None):
        """grids: sequence of (nx, ny, dx, bc) tuples; `boundary` applies to every grid."""
        import torch

        self.torch = torch
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if isinstance(limiter, str):
            limiter = LIMITERS[limiter.lower()]
        self.shapes = [(int(g[0]), int(g[1])) for g in grids]
        self.precision = precision
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self._grids = [vlbm_grid(int(g[0]), int(g[1]), float(g[2]), (ctypes.c_int32 * 4)(*g[3]))
                       for g in grids]
        self.opts = _opts(alpha, eps, 0, sponge, boundary)
        nbytes = vlbm_batch_workspace_bytes(self._grids, precision)
        if nbytes == 0:
            raise VLBMError(E_INVAL, "invalid grids")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace.record_stream(self.stream)
        rc, self._b = vlbm_batch_init(self._grids, gamma, limiter, precision, self.opts,
                                      self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        if rc != OK:
            raise VLBMError(rc, vlbm_batch_last_error(None))

    def _chk(self, rc):
        if rc != OK:
            raise VLBMError(rc, vlbm_batch_last_error(self._b))

    def set_conserved(self, i, rho, mom, E):
        for t in (rho, mom, E):
            if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
                raise ValueError("tensor must be contiguous, on the batch's device, in its dtype")
        with _StreamOrder(self):
            self._chk(vlbm_batch_set_conserved(self._b, i, rho.data_ptr(), mom.data_ptr(), E.data_ptr()))

    def step(self, nsteps: int = 1):
        with _StreamOrder(self):
            self._chk(vlbm_batch_step(self._b, int(nsteps)))

    def moments(self, i):
        nx, ny = self.shapes[i]
        t = self.torch
        rho = t.empty((ny, nx), dtype=self.dtype, device=self.device)
        mom = t.empty((2, ny, nx), dtype=self.dtype, device=self.device)
        E = t.empty((ny, nx), dtype=self.dtype, device=self.device)
        with _StreamOrder(self):
            self._chk(vlbm_batch_moments(self._b, i, rho.data_ptr(), mom.data_ptr(), E.data_ptr()))
        return rho, mom, E

    def state_planes(self, i):
        nx, ny = self.shapes[i]
        el = 8 if self.precision == FP64 else 4
        buf = self.torch.empty(64 + 20 * nx * ny * el, dtype=self.torch.uint8, device=self.device)
        with _StreamOrder(self):
            self._chk(vlbm_batch_save(self._b, i, buf.data_ptr()))
        return buf[64:].view(self.dtype).view(20, ny, nx)

    def monitors(self, i) -> dict:
        rc, m = vlbm_batch_monitors(self._b, i)
        return {"status": m.status, "n": m.n, "t": m.t, "a": m.a, "lambda": m.lambda_,
                "bad_cells": m.bad_cells, "nonfinite_cells": m.nonfinite_cells,
                "first_bad_step": m.first_bad_step, "min_rho": m.min_rho, "sum": list(m.sum),
                "theta_p_fp64_faces": m.theta_p_fp64_faces,
                "min_internal_energy": m.min_internal_energy, "done": m.done}

    def tuning(self) -> dict:
        rc, t = vlbm_batch_get_tuning(self._b)
        self._chk(rc)
        return {"chunk": t.chunk, "ctas_per_sm": t.ctas_per_sm, "order": t.order, "items": t.items,
                "ctas": t.ctas}

    def set_tuning(self, chunk, ctas_per_sm, order=ORDER_LPT):
        self._chk(vlbm_batch_set_tuning(self._b, vlbm_batch_tuning(chunk, ctas_per_sm, order, 0, 0)))

    def autotune(self, trial_steps: int = 3):
        with _StreamOrder(self):
            rc, t, ms = vlbm_batch_autotune(self._b, int(trial_steps))
        self._chk(rc)
        return {"chunk": t.chunk, "ctas_per_sm": t.ctas_per_sm, "order": t.order, "items": t.items,
                "ctas": t.ctas, "ms_per_step": ms}

    def close(self):
        if getattr(self, "_b", None):
            vlbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rollout_function():
    import torch

    class VLBMRollout(torch.autograd.Function):
        """u^N = rollout(u_0) through `nsteps` steps of a VLBM solver, differentiable in u_0.

        forward(rho, mom, E, solver, nsteps, ckpt_every) -> (rho^N, mom^N, E^N); the
        backward pass is the library's adjoint (vlbm_adjoint) over the checkpoints
        the forward pass stored; a dynamic a^n is held or differentiated as the
        solver's set_adjoint_mode says. One solver may serve several forwards before
        their backwards: a backward whose forward is no longer the solver's latest
        rollout passes u_0 to vlbm_adjoint, which then runs that rollout again."""

        @staticmethod
        def forward(ctx, rho, mom, E, solver, nsteps, ckpt_every):
            scratch = solver.adjoint_scratch(nsteps, ckpt_every)
            solver.set_conserved(rho.contiguous(), mom.contiguous(), E.contiguous())
            solver.rollout(nsteps, ckpt_every, scratch)
            token = object()
            solver._rollout_token = token
            ctx.solver, ctx.nsteps, ctx.every, ctx.scratch, ctx.token = solver, nsteps, ckpt_every, scratch, token
            ctx.u0 = torch.cat([rho.detach().reshape(1, solver.ny, solver.nx),
                                mom.detach().reshape(2, solver.ny, solver.nx),
                                E.detach().reshape(1, solver.ny, solver.nx)]).to(solver.dtype).contiguous()
            return solver.moments()

        @staticmethod
        def backward(ctx, g_rho, g_mom, g_E):
            s = ctx.solver
            t = torch
            z = lambda g, shape: g if g is not None else t.zeros(shape, dtype=s.dtype, device=s.device)
            dLduN = t.cat([z(g_rho, (s.ny, s.nx)).reshape(1, s.ny, s.nx),
                           z(g_mom, (2, s.ny, s.nx)).reshape(2, s.ny, s.nx),
                           z(g_E, (s.ny, s.nx)).reshape(1, s.ny, s.nx)]).to(s.dtype).contiguous()
            latest = getattr(s, "_rollout_token", None) is ctx.token
            g = s.adjoint(dLduN, ctx.nsteps, ctx.every, ctx.scratch, u0=None if latest else ctx.u0)
            s._rollout_token = ctx.token          # the checkpoints now hold this rollout
            ctx.scratch = ctx.u0 = None
            return g[0], g[1:3], g[3], None, None, None

    return VLBMRollout


def __getattr__(name):
    if name == "VLBMRollout":
        cls = _rollout_function()
        globals()["VLBMRollout"] = cls
        return cls
    raise AttributeError(name)
