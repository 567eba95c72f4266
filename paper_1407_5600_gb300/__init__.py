"""GB300 multiblob inertial-coupling library: Python binding of libmb.so (include/mb.h).

The binding only marshals arguments: every step of the method runs in the CUDA kernels of
libmb.so.  Arrays may be torch tensors (device or host) or numpy arrays (host); they are passed
to the C ABI as raw pointers and must be C-contiguous with the documented dtype.  PyTorch is
used for device memory and streams only.

If the compiled library is missing and cannot be built, every call raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "GridDesc", "MBError", "load_library", "create_grid", "destroy", "set_particles", "step",
    "get_velocities", "get_particle_velocities", "set_velocity_field", "spread", "spread_static",
    "interp",
    "fluid_update", "get_counts", "get_forces", "set_stage_timing", "get_stage_times",
    "get_launch_count", "get_tuning", "set_positions", "adjoint_step", "velocity_adjoint",
    "particle_velocity_adjoint", "last_error", "Multiblob",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libmb.so")
_lib = None

STATUS = {0: "MB_OK", 1: "MB_EINVAL", 2: "MB_ENOMEM", 3: "MB_ECUDA", 4: "MB_ESTATE",
          5: "MB_ETIMEOUT"}


class MBError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("batch", ctypes.c_int), ("h", ctypes.c_double), ("rho", ctypes.c_double),
                ("eta", ctypes.c_double), ("dt", ctypes.c_double), ("precision", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("advection", ctypes.c_int),
                ("mean_mode", ctypes.c_int), ("kT", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("integrator", ctypes.c_int)]


@dataclass
class GridDesc:
    nx: int
    ny: int
    nz: int
    batch: int = 1
    h: float = 1.0
    rho: float = 1.0
    eta: float = 1.0
    dt: float = 0.05
    precision: int = 0        # 0: FP32 grid, 1: FP64
    deterministic: int = 0
    advection: int = 0
    mean_mode: int = 0        # 0: conserve net momentum, 1: hold the mean at zero
    kT: float = 0.0
    seed: int = 0
    integrator: int = 0       # 0: inertial coupling, 1: Stokes limit

    def _c(self):
        return _Desc(self.nx, self.ny, self.nz, self.batch, self.h, self.rho, self.eta, self.dt,
                     self.precision, self.deterministic, self.advection, self.mean_mode,
                     self.kT, self.seed, self.integrator)

    @property
    def grid_dtype(self):
        return np.float64 if self.precision == 1 else np.float32


def load_library(path: str | None = None):
    """Loads libmb.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if path == _LIB_PATH:
        from . import build as _build
        try:
            _build.build()          # no-op when the library is newer than its sources
        except RuntimeError:
            if not os.path.exists(path):
                raise
    lib = ctypes.CDLL(path)
    P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    sig = {
        "mb_create_grid": [ctypes.POINTER(_Desc), P, ctypes.POINTER(P)],
        "mb_destroy": [P],
        "mb_set_particles": [P, I, I64, P, P, I64, P, P, D, D, D],
        "mb_step": [P, I, P, P],
        "mb_get_velocities": [P, P, P, P, P],
        "mb_get_particle_velocities": [P, P, P],
        "mb_set_velocity_field": [P, P],
        "mb_spread": [P, I64, P, P, P],
        "mb_interp": [P, I64, P, P, P],
        "mb_fluid_update": [P, P, P, P, P],
        "mb_get_counts": [P, ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "mb_get_forces": [P, P, P],
        "mb_spread_static": [ctypes.POINTER(_Desc), I64, P, P, P, P],
        "mb_set_stage_timing": [P, I],
        "mb_set_positions": [P, P],
        "mb_get_tuning": [P, P, P],
        "mb_adjoint_step": [P, P, P, P, P, P, P, P],
        "mb_velocity_adjoint": [P, P, P, P, P, P],
        "mb_particle_velocity_adjoint": [P, P, P, P, P, P],
        "mb_get_stage_times": [P, I, P, P, ctypes.POINTER(I)],
        "mb_get_launch_count": [P, ctypes.POINTER(I64)],
        "mb_set_step_index": [P, ctypes.c_uint64],
        "mb_get_step_index": [P, ctypes.POINTER(ctypes.c_uint64)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.mb_stage_name.argtypes = [I]
    lib.mb_stage_name.restype = ctypes.c_char_p
    lib.mb_last_error.argtypes = [P]
    lib.mb_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(x, dtype=None):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != dtype:
            raise TypeError(f"expected dtype {np.dtype(dtype)}, got {x.dtype}")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None:
            import torch
            want = {np.float64: torch.float64, np.float32: torch.float32,
                    np.int32: torch.int32}[np.dtype(dtype).type]
            if x.dtype != want:
                raise TypeError(f"expected {want}, got {x.dtype}")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported array type {type(x)}")


def _check(ctx, status):
    if status != 0:
        raise MBError(status, last_error(ctx))


def last_error(ctx=None) -> str:
    msg = load_library().mb_last_error(ctx)
    return msg.decode() if msg else ""


def create_grid(desc: GridDesc, stream=None):
    """mb_create_grid; stream is a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    lib = load_library()
    handle = ctypes.c_void_p()
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    st = lib.mb_create_grid(ctypes.byref(desc._c()), s, ctypes.byref(handle))
    _check(None, st)
    return handle.value


def destroy(ctx):
    _check(ctx, load_library().mb_destroy(ctx))


def set_particles(ctx, box, pos, particle_id, bonds, rest_len, k_spring, k_rep=0.0, r_cut=0.0):
    n = int(pos.shape[0]) if pos is not None else 0
    m = int(bonds.shape[0]) if bonds is not None and len(bonds.shape) else 0
    _check(ctx, load_library().mb_set_particles(
        ctx, int(box), n, _ptr(pos, np.float64), _ptr(particle_id, np.int32), m,
        _ptr(bonds, np.int32) if m else None, _ptr(rest_len, np.float64) if m else None,
        float(k_spring), float(k_rep), float(r_cut)))


def step(ctx, n_steps, ext_blob_force=None, body_force=None):
    body = None
    if body_force is not None:
        body = np.ascontiguousarray(np.asarray(body_force, dtype=np.float64).reshape(4))
    _check(ctx, load_library().mb_step(ctx, int(n_steps), _ptr(ext_blob_force, np.float64),
                                       _ptr(body)))


def get_velocities(ctx, blob_vel=None, blob_pos=None, particle_U=None, grid_v=None):
    _check(ctx, load_library().mb_get_velocities(ctx, _ptr(blob_vel, np.float64),
                                                 _ptr(blob_pos, np.float64),
                                                 _ptr(particle_U, np.float64), _ptr(grid_v)))


def get_particle_velocities(ctx, particle_U=None, particle_Omega=None):
    _check(ctx, load_library().mb_get_particle_velocities(ctx, _ptr(particle_U, np.float64),
                                                          _ptr(particle_Omega, np.float64)))


def set_velocity_field(ctx, grid_v):
    _check(ctx, load_library().mb_set_velocity_field(ctx, _ptr(grid_v)))


def spread(ctx, pos, F, grid_out):
    _check(ctx, load_library().mb_spread(ctx, int(pos.shape[0]), _ptr(pos, np.float64),
                                         _ptr(F, np.float64), _ptr(grid_out)))


def spread_static(desc: GridDesc, pos, F, grid_out, stream=None):
    """mb_spread_static: spreading without any allocation (device arrays only, no context)."""
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(None, load_library().mb_spread_static(ctypes.byref(desc._c()), int(pos.shape[0]),
                                                 _ptr(pos, np.float64), _ptr(F, np.float64),
                                                 _ptr(grid_out), s))


def interp(ctx, pos, grid_v, u_out):
    _check(ctx, load_library().mb_interp(ctx, int(pos.shape[0]), _ptr(pos, np.float64),
                                         _ptr(grid_v), _ptr(u_out, np.float64)))


def fluid_update(ctx, v_in, f, v_out, body_force=None):
    body = None
    if body_force is not None:
        body = np.ascontiguousarray(np.asarray(body_force, dtype=np.float64).reshape(4))
    _check(ctx, load_library().mb_fluid_update(ctx, _ptr(v_in), _ptr(f), _ptr(body),
                                               _ptr(v_out)))


def get_forces(ctx, blob_force=None, midpoint_pos=None):
    _check(ctx, load_library().mb_get_forces(ctx, _ptr(blob_force, np.float64),
                                             _ptr(midpoint_pos, np.float64)))


def set_stage_timing(ctx, enable=True):
    _check(ctx, load_library().mb_set_stage_timing(ctx, int(bool(enable))))


def get_stage_times(ctx):
    """{stage name: (total ms, calls)} accumulated since timing was enabled."""
    lib = load_library()
    n = ctypes.c_int()
    ms = (ctypes.c_double * 64)()
    calls = (ctypes.c_int64 * 64)()
    _check(ctx, lib.mb_get_stage_times(ctx, 64, ms, calls, ctypes.byref(n)))
    return {lib.mb_stage_name(i).decode(): (ms[i], calls[i]) for i in range(n.value)}


def get_launch_count(ctx):
    n = ctypes.c_int64()
    _check(ctx, load_library().mb_get_launch_count(ctx, ctypes.byref(n)))
    return n.value


def set_positions(ctx, pos):
    _check(ctx, load_library().mb_set_positions(ctx, _ptr(pos, np.float64)))


def set_step_index(ctx, step):
    """mb_set_step_index: the step index keying the next step's thermal stress."""
    _check(ctx, load_library().mb_set_step_index(ctx, int(step)))


def get_step_index(ctx):
    n = ctypes.c_uint64()
    _check(ctx, load_library().mb_get_step_index(ctx, ctypes.byref(n)))
    return n.value


def adjoint_step(ctx, pos_n, grid_v_n, ext_blob_force, body_force, grad_pos, grad_v,
                 grad_k_spring=None):
    """mb_adjoint_step: overwrites grad_pos and grad_v in place, adds to grad_k_spring[0]."""
    body = None
    if body_force is not None:
        body = np.ascontiguousarray(np.asarray(body_force, dtype=np.float64).reshape(4))
    _check(ctx, load_library().mb_adjoint_step(
        ctx, _ptr(pos_n, np.float64), _ptr(grid_v_n), _ptr(ext_blob_force, np.float64),
        _ptr(body), _ptr(grad_pos, np.float64), _ptr(grad_v),
        _ptr(grad_k_spring, np.float64) if grad_k_spring is not None else None))


def velocity_adjoint(ctx, pos, grid_v, grad_u, grad_pos, grad_v):
    """mb_velocity_adjoint: grad_pos += (du/dq)^T grad_u, grad_v += J^T grad_u."""
    _check(ctx, load_library().mb_velocity_adjoint(
        ctx, _ptr(pos, np.float64), _ptr(grid_v), _ptr(grad_u, np.float64),
        _ptr(grad_pos, np.float64), _ptr(grad_v)))


def particle_velocity_adjoint(ctx, pos, grid_v, grad_U, grad_pos, grad_v):
    """mb_particle_velocity_adjoint: grad_pos += (dU0/dq)^T grad_U, grad_v += (dU0/dv)^T grad_U."""
    _check(ctx, load_library().mb_particle_velocity_adjoint(
        ctx, _ptr(pos, np.float64), _ptr(grid_v), _ptr(grad_U, np.float64),
        _ptr(grad_pos, np.float64), _ptr(grad_v)))


def get_tuning(ctx):
    """(spreading tile (tx, ty, tz), milliseconds of one spreading launch when tuned)."""
    tile = (ctypes.c_int * 3)()
    ms = ctypes.c_float()
    _check(ctx, load_library().mb_get_tuning(ctx, tile, ctypes.byref(ms)))
    return tuple(tile), ms.value


def get_counts(ctx):
    nb, np_ = ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, load_library().mb_get_counts(ctx, ctypes.byref(nb), ctypes.byref(np_)))
    return nb.value, np_.value


class Multiblob:
    """Owning wrapper around one mb_ctx, with torch tensors for device memory.

    Example:
        sim = Multiblob(GridDesc(32, 32, 32, precision=1))
        sim.set_particles(0, pos, pid, bonds, rest, k_spring=100.0)
        sim.step(200, ext_blob_force=ext)
        u = sim.blob_velocities()
    """

    def __init__(self, desc: GridDesc, stream=None, device="cuda"):
        import torch
        self.torch = torch
        self.desc = desc
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = create_grid(desc, self.stream)
        self.grid_dtype = torch.float64 if desc.precision == 1 else torch.float32

    def close(self):
        if self.ctx:
            destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, x, dtype):
        t = self.torch
        if x is None:
            return None
        if not isinstance(x, t.Tensor):
            x = t.as_tensor(np.ascontiguousarray(x))
        return x.to(device=self.device, dtype=dtype).contiguous()

    def grid_shape(self, boxes=None):
        d = self.desc
        b = d.batch if boxes is None else boxes
        return (b, 3, d.nz, d.ny, d.nx)

    def set_particles(self, box, pos, particle_id, bonds, rest_len, k_spring, k_rep=0.0,
                      r_cut=0.0):
        t = self.torch
        set_particles(self.ctx, box, self._dev(pos, t.float64), self._dev(particle_id, t.int32),
                      self._dev(np.asarray(bonds).reshape(-1, 2), t.int32),
                      self._dev(rest_len, t.float64), k_spring, k_rep, r_cut)

    def step(self, n_steps, ext_blob_force=None, body_force=None):
        step(self.ctx, n_steps, self._dev(ext_blob_force, self.torch.float64)
             if ext_blob_force is not None else None, body_force)

    def counts(self):
        return get_counts(self.ctx)

    def blob_velocities(self):
        nb, _ = self.counts()
        out = self.torch.empty((nb, 3), dtype=self.torch.float64, device=self.device)
        get_velocities(self.ctx, blob_vel=out)
        return out

    def last_forces(self):
        """(F, q_half) of the last step, each [total blobs][3]."""
        nb, _ = self.counts()
        F = self.torch.empty((nb, 3), dtype=self.torch.float64, device=self.device)
        qh = self.torch.empty((nb, 3), dtype=self.torch.float64, device=self.device)
        get_forces(self.ctx, F, qh)
        return F, qh

    def blob_positions(self):
        nb, _ = self.counts()
        out = self.torch.empty((nb, 3), dtype=self.torch.float64, device=self.device)
        get_velocities(self.ctx, blob_pos=out)
        return out

    def particle_velocities(self):
        _, npart = self.counts()
        U = self.torch.empty((npart, 3), dtype=self.torch.float64, device=self.device)
        W = self.torch.empty((npart, 3), dtype=self.torch.float64, device=self.device)
        get_particle_velocities(self.ctx, U, W)
        return U, W

    def velocity_field(self):
        out = self.torch.empty(self.grid_shape(), dtype=self.grid_dtype, device=self.device)
        get_velocities(self.ctx, grid_v=out)
        return out

    def set_positions(self, pos):
        set_positions(self.ctx, self._dev(pos, self.torch.float64))

    def set_velocity_field(self, v):
        set_velocity_field(self.ctx, self._dev(v, self.grid_dtype))

    @property
    def step_index(self):
        """Index keying the next step's thermal stress (settable, for resuming a run)."""
        return get_step_index(self.ctx)

    @step_index.setter
    def step_index(self, n):
        set_step_index(self.ctx, n)

    def spread(self, pos, F):
        out = self.torch.empty(self.grid_shape(1), dtype=self.grid_dtype, device=self.device)
        spread(self.ctx, self._dev(pos, self.torch.float64), self._dev(F, self.torch.float64), out)
        return out

    def interp(self, pos, v):
        pos = self._dev(pos, self.torch.float64)
        out = self.torch.empty((pos.shape[0], 3), dtype=self.torch.float64, device=self.device)
        interp(self.ctx, pos, self._dev(v, self.grid_dtype), out)
        return out

    def fluid_update(self, v, f=None, body_force=None):
        out = self.torch.empty(self.grid_shape(1), dtype=self.grid_dtype, device=self.device)
        fluid_update(self.ctx, self._dev(v, self.grid_dtype) if v is not None else None,
                     self._dev(f, self.grid_dtype) if f is not None else None, out, body_force)
        return out
