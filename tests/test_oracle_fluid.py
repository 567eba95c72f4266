"""Pins of the oracle's DFT and fluid update (no GPU).

- DFT: the O(n^3)-per-axis definition via explicit DFT matrices, numpy.fft, round trip.
- Fluid update (Eq. vf, viscous stress only, Crank-Nicolson in time): the output is
  divergence-free (P v = v), and the residual of the discrete momentum balance
  (rho/dt - eta/2 L) v' - (rho/dt + eta/2 L) v - f is a discrete gradient (its MAC curl
  vanishes), which together characterise the projected solve without re-using it.
- Closed forms: decay factor of one shear mode per step, the steady sinusoidal profile of the
  viscosity protocol (Sec. 10, eta = f0/(k^2 v_x) with the discrete k^2), and momentum
  bookkeeping rho h^3 sum(v' - v) = dt sum F (zeroth moment of S).
"""
import numpy as np
import pytest

import oracle as mb
from paper_1407_5600_gb300 import workloads as wl


def _dft_matrix(n, sign):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 5, 3), (8, 4, 2)])
def test_dft_matches_definition(shape):
    rng = np.random.default_rng(1)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    nz, ny, nx = shape
    ref = np.einsum("ab,kjb->kja", _dft_matrix(nx, -1), x)
    ref = np.einsum("ab,kbi->kai", _dft_matrix(ny, -1), ref)
    ref = np.einsum("ab,bji->aji", _dft_matrix(nz, -1), ref)
    out = mb.dft3(x)
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))
    back = mb.dft3(out, inverse=True) / x.size
    assert np.max(np.abs(back - x)) < 1e-14 * np.max(np.abs(x)) * 10


@pytest.mark.parametrize("shape", [(32, 32, 32), (12, 10, 6), (16, 8, 64)])
def test_dft_matches_numpy(shape):
    rng = np.random.default_rng(2)
    x = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    out = mb.dft3(x)
    ref = np.fft.fftn(x)
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))
    inv = mb.dft3(x, inverse=True)
    assert np.max(np.abs(inv - np.fft.ifftn(x) * x.size)) < 1e-13 * np.max(np.abs(inv))


def _div(v, h):
    vx, vy, vz = v
    return ((np.roll(vx, -1, 2) - vx) + (np.roll(vy, -1, 1) - vy) + (np.roll(vz, -1, 0) - vz)) / h


def _lap(c, h):
    return sum(np.roll(c, s, a) for a in range(3) for s in (1, -1)) / h ** 2 - 6 * c / h ** 2


def _curl(r, h):
    """MAC curl on edges: a discrete gradient (face values p[i] - p[i-1]) has zero curl."""
    rx, ry, rz = r
    cz = (rx - np.roll(rx, 1, 1)) - (ry - np.roll(ry, 1, 2))
    cx = (ry - np.roll(ry, 1, 0)) - (rz - np.roll(rz, 1, 1))
    cy = (rz - np.roll(rz, 1, 2)) - (rx - np.roll(rx, 1, 0))
    return np.stack([cx, cy, cz]) / h


@pytest.mark.parametrize("shape,h,mean_mode", [((16, 16, 16), 1.0, 0), ((8, 12, 16), 0.5, 1),
                                              ((6, 10, 4), 2.0, 0)])
def test_fluid_update_characterisation(shape, h, mean_mode):
    g = mb.Grid(shape[2], shape[1], shape[0], h=h, rho=1.3, eta=0.7, dt=0.05,
                mean_mode=mean_mode)
    v = mb.fluid_update(mb.Grid(g.nx, g.ny, g.nz, h=h, rho=1.0, eta=0.0, dt=1.0),
                        g.zeros(), wl.random_field(g.shape, 3))          # P of a random field
    assert np.max(np.abs(_div(v, h))) < 1e-12 * np.max(np.abs(v)) / h
    f = wl.random_field(g.shape, 4, scale=0.3)
    vn = mb.fluid_update(g, v, f)
    scale = np.max(np.abs(vn)) / h
    assert np.max(np.abs(_div(vn, h))) < 1e-12 * scale
    res = np.stack([(g.rho / g.dt) * vn[a] - 0.5 * g.eta * _lap(vn[a], h)
                    - (g.rho / g.dt) * v[a] - 0.5 * g.eta * _lap(v[a], h) - f[a]
                    for a in range(3)])
    big = np.max(np.abs(f)) + g.rho / g.dt * np.max(np.abs(v))
    assert np.max(np.abs(_curl(res, h))) < 1e-11 * big / h
    if mean_mode == 0:
        # mean mode follows the net force: rho (mean v' - mean v) = dt mean f
        assert np.allclose(g.rho * (vn.mean((1, 2, 3)) - v.mean((1, 2, 3))),
                           g.dt * f.mean((1, 2, 3)), rtol=0, atol=1e-12 * big * g.dt)
    else:
        assert np.max(np.abs(vn.mean((1, 2, 3)))) < 1e-13 * np.max(np.abs(vn))


def test_stokes_solution_characterisation():
    g = mb.Grid(12, 16, 8, h=1.0, eta=2.5)
    f = wl.random_field(g.shape, 7)
    f -= f.mean((1, 2, 3), keepdims=True)
    v = mb.stokes_solve(g, f)
    assert np.max(np.abs(_div(v, g.h))) < 1e-12 * np.max(np.abs(v))
    res = np.stack([g.eta * _lap(v[a], g.h) + f[a] for a in range(3)])
    assert np.max(np.abs(_curl(res, g.h))) < 1e-12 * np.max(np.abs(f))
    assert np.max(np.abs(v.mean((1, 2, 3)))) < 1e-14


@pytest.mark.parametrize("n,h,j", [(32, 1.0, 1), (16, 0.5, 3)])
def test_shear_mode_decay_closed_form(n, h, j):
    g = mb.Grid(n, n, n, h=h, rho=1.0, eta=1.0, dt=0.05)
    L = n * h
    z = (np.arange(n) + 0.5) * h              # v_x nodes sit at z = (k + 1/2) h
    v = g.zeros()
    v[0] = np.sin(2 * np.pi * j * z / L)[:, None, None] * np.ones((n, n, n))
    lam = 4.0 / h ** 2 * np.sin(np.pi * j * h / L) ** 2
    nu = g.eta / g.rho
    factor = (1 - g.dt * nu * lam / 2) / (1 + g.dt * nu * lam / 2)
    vn = mb.fluid_update(g, v, g.zeros())
    assert np.max(np.abs(vn - factor * v)) < 1e-13


def test_viscosity_protocol_steady_profile():
    """Sec. 10: body force f0 sin(k z) x_hat; the discrete steady profile v = f0/(eta k_eff^2)
    with k_eff^2 = (4/h^2) sin^2(k h/2) is a fixed point of the update, and the estimator
    eta = f0/(k_eff^2 v_x) returns the fluid viscosity."""
    n, h, j, f0 = 32, 1.0, 1, 1e-4
    g = mb.Grid(n, n, n, h=h, rho=1.0, eta=1.7, dt=0.05)
    L = n * h
    z = (np.arange(n) + 0.5) * h
    k2 = 4.0 / h ** 2 * np.sin(np.pi * j * h / L) ** 2
    v = g.zeros()
    v[0] = (f0 / (g.eta * k2) * np.sin(2 * np.pi * j * z / L))[:, None, None]
    vn = mb.fluid_update(g, v, g.zeros(), body=(f0, 0, 2, j))
    assert np.max(np.abs(vn - v)) < 1e-12 * np.max(np.abs(v))
    amp = 2.0 / n * np.sum(vn[0][:, 0, 0] * np.sin(2 * np.pi * j * z / L))
    assert abs(f0 / (k2 * amp) - g.eta) < 1e-10 * g.eta


def test_momentum_bookkeeping_with_spread_forces():
    g = mb.Grid(16, 16, 16, h=0.8, rho=2.0, eta=1.0, dt=0.1, mean_mode=0)
    q, F, _ = wl.random_blobs(30, g.shape, seed=8, h=g.h)
    v = wl.random_field(g.shape, 9, scale=0.01)
    vn = mb.fluid_update(g, v, mb.spread(g, q, F))
    dP = g.rho * g.h ** 3 * (vn.sum((1, 2, 3)) - v.sum((1, 2, 3)))
    assert np.max(np.abs(dP - g.dt * F.sum(0))) < 1e-12 * np.max(np.abs(F.sum(0))) * 10


def test_time_stepping_converges_to_the_steady_stokes_flow():
    """A constant force density (a spread point force) held on the fluid: the Crank-Nicolson
    steps converge to the steady zero-mean Stokes flow of the same force, the solve that the
    mobility pins use (each mode relaxes by (1 - eta lam dt/(2 rho))/(1 + ...) per step)."""
    g = mb.Grid(16, 8, 16, h=0.9, rho=1.0, eta=1.0, dt=1.0, mean_mode=1)
    F = np.array([[0.3, -0.2, 0.5]])
    f = mb.spread(g, np.array([[3.3, 2.1, 7.7]]), F)
    v = g.zeros()
    for _ in range(300):
        v = mb.fluid_update(g, v, f)
    ref = mb.stokes_solve(g, f)
    assert np.linalg.norm(v - ref) < 1e-10 * np.linalg.norm(ref)


def test_transient_viscosity_estimator_returns_eta_for_the_pure_fluid():
    """Sec. 10 protocol before steady state: the Crank-Nicolson transient of the driven shear
    mode, solved for eta, returns the fluid's viscosity after any number of oracle steps (the
    mode is an eigenvector of L and unchanged by the projection)."""
    from helpers import eta_from_transient, shear_amplitude
    n, f0 = 16, 1e-3
    for eta, rho, nsteps in ((1.0, 1.0, 40), (2.5, 5.0, 7), (0.3, 1.0, 120)):
        g = mb.Grid(n, n, n, rho=rho, eta=eta, dt=0.05, mean_mode=0)
        q, v = mb.step(g, nsteps, np.zeros((0, 3)), g.zeros(), np.zeros(0, dtype=np.int32),
                       np.zeros((0, 2), dtype=np.int32), np.zeros(0), 0.0, body=(f0, 0, 2, 1))
        lam = 4.0 * np.sin(np.pi / n) ** 2
        est = eta_from_transient(shear_amplitude(v[0], n), f0, lam, rho, g.dt, nsteps)
        assert abs(est / eta - 1.0) < 1e-10, (eta, est)
