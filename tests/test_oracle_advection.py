"""Pins of the oracle's convective term D.(v v) (the rho v v stress of Eq. vf on the MAC grid)
against what the mathematics fixes (no GPU).

- Conservative form: every component sums to zero over the box (momentum).
- The centred staggered divergence form conserves kinetic energy for a discretely
  divergence-free field, sum v . D.(v v) = 0, and does not for a general one.
- Linearised about a uniform flow U it is the centred derivative U . grad w (exactly).
- A unidirectional shear flow has no convective term, so its fluid update is unchanged.
- For the 2-D Taylor-Green vortex, (v . grad) v is a pure gradient, and so is the discrete
  term sampled on the MAC grid: its projection vanishes to rounding.
"""
import numpy as np

import oracle as mb
from paper_1407_5600_gb300 import workloads as wl


def _project(shape, f):
    nz, ny, nx = shape
    g0 = mb.Grid(nx, ny, nz, rho=1.0, eta=0.0, dt=1.0)
    return mb.fluid_update(g0, g0.zeros(), f)


def _roll(u, axis_xyz, s):
    """u at index i + s along x (0), y (1) or z (2), periodic."""
    return np.roll(u, -s, axis=2 - axis_xyz)


def test_momentum_and_energy_conservation():
    shape = (8, 16, 4)
    g = mb.Grid(4, 16, 8, h=0.7)
    v = _project(shape, wl.random_field(shape, 3))
    A = mb.advection(g, v)
    scale = np.max(np.abs(A)) * A[0].size
    assert np.max(np.abs(A.sum(axis=(1, 2, 3)))) < 1e-13 * scale
    assert abs(np.sum(v * A)) < 1e-13 * np.sum(np.abs(v * A))
    w = wl.random_field(shape, 4)                      # not divergence-free
    assert abs(np.sum(w * mb.advection(g, w))) > 1e-3 * np.sum(np.abs(w * mb.advection(g, w)))


def test_linearisation_about_uniform_flow_is_centred_derivative():
    shape = (8, 8, 16)
    g = mb.Grid(16, 8, 8, h=0.9)
    w = _project(shape, wl.random_field(shape, 5))
    U = np.array([0.7, -1.3, 0.4])
    eps = 1e-3
    v = U[:, None, None, None] + eps * w
    lin = (mb.advection(g, v) - eps ** 2 * mb.advection(g, w)) / eps
    want = np.zeros_like(w)
    for a in range(3):
        for b in range(3):
            want[a] += U[b] * (_roll(w[a], b, 1) - _roll(w[a], b, -1)) / (2 * g.h)
    assert np.max(np.abs(lin - want)) < 1e-9 * np.max(np.abs(want))
    assert np.max(np.abs(mb.advection(g, U[:, None, None, None] + 0 * w))) < 1e-14


def test_shear_flow_has_no_convective_term():
    n, L = 16, 16.0
    g = mb.Grid(n, n, n, rho=1.0, eta=0.6, dt=0.3, mean_mode=0)
    ga = mb.Grid(n, n, n, rho=1.0, eta=0.6, dt=0.3, mean_mode=0, advection=1)
    v = g.zeros()
    z = (np.arange(n) + 0.5)
    v[0] = (0.4 * np.sin(2 * np.pi * z / L) + 0.1)[:, None, None]
    assert np.max(np.abs(mb.advection(g, v))) == 0.0
    assert np.array_equal(mb.fluid_update(g, v, g.zeros()), mb.fluid_update(ga, v, g.zeros()))


def test_taylor_green_term_is_a_gradient():
    errs = []
    for n in (16, 32):
        h = 2 * np.pi / n
        g = mb.Grid(n, n, 4, h=h)
        x_face = np.arange(n) * h
        c = (np.arange(n) + 0.5) * h
        v = g.zeros()
        # v_x on (i h, (j + 1/2) h), v_y on ((i + 1/2) h, j h); uniform in z
        v[0] = (np.sin(x_face)[None, :] * np.cos(c)[:, None])[None, :, :] * np.ones((4, 1, 1))
        v[1] = (-np.cos(c)[None, :] * np.sin(x_face)[:, None])[None, :, :] * np.ones((4, 1, 1))
        A = mb.advection(g, v)
        errs.append(np.max(np.abs(_project((4, n, n), A))) / np.max(np.abs(A)))
    assert max(errs) < 1e-13, errs
