"""mbref — FP64 CPU oracle of the multiblob ICM step (arXiv:1407.5600).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this module.  The product library never does, and the two
share no code: this wrapper loads ``oracle/_build/libmbref.so`` built from ``mbref.c`` with
plain gcc (``-O2 -ffp-contract=off``, no fast-math, OpenMP over independent loops when the
compiler has it), and marshals numpy arrays into it.

Parity status of each routine (what pins it) is listed in the tests under
``tests/test_oracle_*.py``; every routine here has at least one independent pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbref.c")
_LIB = os.path.join(_HERE, "_build", "libmbref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile mbref.c into a shared library (gcc, FP64, no contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mbref.h"))
    ):
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                "-o", tmp, _SRC, "-lm"]
        try:   # OpenMP threads over independent loops; results do not depend on them
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("rho", ctypes.c_double), ("eta", ctypes.c_double),
                ("dt", ctypes.c_double), ("mean_mode", ctypes.c_int),
                ("advection", ctypes.c_int)]


class _Noise(ctypes.Structure):
    _fields_ = [("kT", ctypes.c_double), ("seed", ctypes.c_uint64), ("step0", ctypes.c_uint64),
                ("box", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        G = ctypes.POINTER(_Grid)
        lib.mbref_phi.restype = D
        lib.mbref_phi.argtypes = [D]
        lib.mbref_set_threads.restype = ctypes.c_int
        lib.mbref_set_threads.argtypes = [ctypes.c_int]
        lib.mbref_philox4x64.restype = None
        lib.mbref_philox4x64.argtypes = [P, P, P]
        for name, args in {
            "mbref_spread": [G, I64, P, P, P],
            "mbref_interp": [G, I64, P, P, P],
            "mbref_dft3": [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int],
            "mbref_fluid_update": [G, P, P, P, P],
            "mbref_stokes_solve": [G, P, P],
            "mbref_bond_forces": [G, I64, P, I64, P, P, D, P],
            "mbref_pair_forces": [G, I64, P, P, D, D, P],
            "mbref_pair_forces_brute": [G, I64, P, P, D, D, P],
            "mbref_pair_forces_subset": [G, I64, P, P, D, D, I64, P, P],
            "mbref_step": [G, ctypes.c_int, I64, P, P, P, I64, P, P, D, D, D, P, P,
                           ctypes.POINTER(_Noise)],
            "mbref_stress_normals": [G, ctypes.c_uint64, ctypes.c_uint64, I64, P],
            "mbref_stress_div": [G, P, P],
            "mbref_advection": [G, P, P],
            "mbref_stokes_step": [G, ctypes.c_int, I64, P, P, P, I64, P, P, D, D, D, P, P],
            "mbref_particle_velocities": [G, I64, P, P, P, I64, P, P],
        }.items():
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = args
        _lib = lib
    return _lib


@dataclass
class Grid:
    """Periodic MAC grid and fluid parameters (mirrors the oracle's C struct)."""
    nx: int
    ny: int
    nz: int
    h: float = 1.0
    rho: float = 1.0
    eta: float = 1.0
    dt: float = 0.05
    mean_mode: int = 0   # 0: mean momentum follows the net force; 1: mean held at zero
    advection: int = 0   # 1: the convective stress rho v v, explicit at v^n

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def L(self):
        return np.array([self.nx * self.h, self.ny * self.h, self.nz * self.h])

    def _c(self):
        return ctypes.byref(_Grid(self.nx, self.ny, self.nz, self.h, self.rho, self.eta,
                                  self.dt, self.mean_mode, self.advection))

    def zeros(self):
        return np.zeros((3,) + self.shape)


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} returned {rc}")


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's parallel loops (n <= 0: leave unchanged); returns the number
    in effect.  No result depends on it."""
    return _load().mbref_set_threads(int(n))


def phi(r: float) -> float:
    """Three-point kernel Phi(r) of Eq. (delta)."""
    return _load().mbref_phi(float(r))


def spread(g: Grid, q, F):
    """f = S F on the MAC grid; returns [3][nz][ny][nx]."""
    q, qp = _d(q)
    F, Fp = _d(F)
    f = g.zeros()
    _check(_load().mbref_spread(g._c(), len(q), qp, Fp, f.ctypes.data_as(ctypes.c_void_p)),
           "spread")
    return f


def interp(g: Grid, q, v):
    """u = J v at the blobs; returns [n][3]."""
    q, qp = _d(q)
    v, vp = _d(v)
    u = np.zeros((len(q), 3))
    _check(_load().mbref_interp(g._c(), len(q), qp, vp, u.ctypes.data_as(ctypes.c_void_p)),
           "interp")
    return u


def dft3(x, inverse=False):
    """Unnormalised 3-D DFT of a complex array [nz][ny][nx]."""
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real)
    im = np.ascontiguousarray(x.imag)
    nz, ny, nx = x.shape
    _check(_load().mbref_dft3(nx, ny, nz, re.ctypes.data_as(ctypes.c_void_p),
                              im.ctypes.data_as(ctypes.c_void_p), int(inverse)), "dft3")
    return re + 1j * im


def _body(body):
    if body is None:
        return None, None
    return _d(np.asarray(body, dtype=np.float64).reshape(4))


def fluid_update(g: Grid, v, f, body=None):
    """One CN + projection fluid update; returns the new [3][nz][ny][nx] velocity."""
    v, vp = _d(v)
    f, fp = _d(f)
    b, bp = _body(body)
    out = g.zeros()
    _check(_load().mbref_fluid_update(g._c(), vp, fp, bp, out.ctypes.data_as(ctypes.c_void_p)),
           "fluid_update")
    return out


def stokes_solve(g: Grid, f):
    """Steady Stokes velocity P (-eta L)^-1 f (mean mode zero)."""
    f, fp = _d(f)
    out = g.zeros()
    _check(_load().mbref_stokes_solve(g._c(), fp, out.ctypes.data_as(ctypes.c_void_p)),
           "stokes_solve")
    return out


def bond_forces(g: Grid, q, bonds, rest, k):
    q, qp = _d(q)
    b, bp = _i32(np.asarray(bonds).reshape(-1, 2))
    r, rp = _d(rest)
    F = np.zeros((len(q), 3))
    _check(_load().mbref_bond_forces(g._c(), len(q), qp, len(b), bp, rp, float(k),
                                     F.ctypes.data_as(ctypes.c_void_p)), "bond_forces")
    return F


def pair_forces(g: Grid, q, pid, k_rep, r_cut):
    q, qp = _d(q)
    p, pp = _i32(pid)
    F = np.zeros((len(q), 3))
    _check(_load().mbref_pair_forces(g._c(), len(q), qp, pp, float(k_rep), float(r_cut),
                                     F.ctypes.data_as(ctypes.c_void_p)), "pair_forces")
    return F


def pair_forces_brute(g: Grid, q, pid, k_rep, r_cut):
    """The repulsion by its definition (all pairs); pair_forces equals it to the bit."""
    q, qp = _d(q)
    p, pp = _i32(pid)
    F = np.zeros((len(q), 3))
    _check(_load().mbref_pair_forces_brute(g._c(), len(q), qp, pp, float(k_rep), float(r_cut),
                                           F.ctypes.data_as(ctypes.c_void_p)),
           "pair_forces_brute")
    return F


def pair_forces_subset(g: Grid, q, pid, k_rep, r_cut, idx):
    q, qp = _d(q)
    p, pp = _i32(pid)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    F = np.zeros((len(idx), 3))
    _check(_load().mbref_pair_forces_subset(
        g._c(), len(q), qp, pp, float(k_rep), float(r_cut), len(idx),
        idx.ctypes.data_as(ctypes.c_void_p), F.ctypes.data_as(ctypes.c_void_p)),
        "pair_forces_subset")
    return F


def philox4x64(counter, key):
    """Philox4x64-10 block: four uint64 words of Philox(counter[4], key[2])."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, dtype=np.uint64)
    _load().mbref_philox4x64(c.ctypes.data_as(ctypes.c_void_p), k.ctypes.data_as(ctypes.c_void_p),
                             out.ctypes.data_as(ctypes.c_void_p))
    return out


def stress_normals(g: Grid, seed, step, box=0):
    """The standard normals W [9][nz][ny][nx] of the thermal stress at one step."""
    W = np.zeros((9,) + g.shape)
    _check(_load().mbref_stress_normals(g._c(), int(seed), int(step), int(box),
                                        W.ctypes.data_as(ctypes.c_void_p)), "stress_normals")
    return W


def stress_div(g: Grid, W):
    """D.W on the MAC faces for a stress field W [9][nz][ny][nx]; returns [3][nz][ny][nx]."""
    W, Wp = _d(np.asarray(W).reshape((9,) + g.shape))
    f = g.zeros()
    _check(_load().mbref_stress_div(g._c(), Wp, f.ctypes.data_as(ctypes.c_void_p)), "stress_div")
    return f


def advection(g: Grid, v):
    """D.(v v), the convective term on the MAC faces; returns [3][nz][ny][nx]."""
    v, vp = _d(v)
    out = g.zeros()
    _check(_load().mbref_advection(g._c(), vp, out.ctypes.data_as(ctypes.c_void_p)), "advection")
    return out


def step(g: Grid, nsteps, q, v, pid, bonds, rest, k_spring, k_rep=0.0, r_cut=0.0,
         ext=None, body=None, kT=0.0, seed=0, step0=0, box=0):
    """Run nsteps ICM steps; returns new (q, v) (inputs are not modified).  kT > 0 adds the
    thermal stress of steps step0, step0 + 1, ... of box `box` drawn with `seed`."""
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    p, pp = _i32(pid)
    b, bp = _i32(np.asarray(bonds).reshape(-1, 2))
    r, rp = _d(rest)
    e, ep = _d(ext) if ext is not None else (None, None)
    bb, bbp = _body(body)
    _check(_load().mbref_step(g._c(), int(nsteps), len(q), q.ctypes.data_as(ctypes.c_void_p),
                              v.ctypes.data_as(ctypes.c_void_p), pp, len(b), bp, rp,
                              float(k_spring), float(k_rep), float(r_cut), ep, bbp,
                              ctypes.byref(_Noise(float(kT), int(seed), int(step0), int(box)))),
           "step")
    return q, v


def stokes_step(g: Grid, nsteps, q, pid, bonds, rest, k_spring, k_rep=0.0, r_cut=0.0,
                ext=None, body=None):
    """Run nsteps Stokes-limit steps (explicit midpoint, steady zero-mean Stokes flow of the
    current forces); returns new (q, v) with v the last flow (inputs are not modified)."""
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    v = g.zeros()
    p, pp = _i32(pid)
    b, bp = _i32(np.asarray(bonds).reshape(-1, 2))
    r, rp = _d(rest)
    e, ep = _d(ext) if ext is not None else (None, None)
    bb, bbp = _body(body)
    _check(_load().mbref_stokes_step(g._c(), int(nsteps), len(q),
                                     q.ctypes.data_as(ctypes.c_void_p),
                                     v.ctypes.data_as(ctypes.c_void_p), pp, len(b), bp, rp,
                                     float(k_spring), float(k_rep), float(r_cut), ep, bbp),
           "stokes_step")
    return q, v


def particle_velocities(g: Grid, q, u, pid, n_particles):
    """(U0, Omega) per particle, each [np][3]."""
    q, qp = _d(q)
    u, up = _d(u)
    p, pp = _i32(pid)
    U = np.zeros((n_particles, 3))
    W = np.zeros((n_particles, 3))
    _check(_load().mbref_particle_velocities(g._c(), len(q), qp, up, pp, n_particles,
                                             U.ctypes.data_as(ctypes.c_void_p),
                                             W.ctypes.data_as(ctypes.c_void_p)),
           "particle_velocities")
    return U, W
