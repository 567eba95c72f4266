"""GPU path on boxes with 256-cell sides (the fluctuating 256^3 suspension and its
oracle-sized stand-ins).

Sides above 128 cells run the fluid solve as five one-axis passes.  Long thin boxes with one
256-cell side are small enough for the oracle, so the 256-point transforms, the thermal stress
and both integrators are compared element by element there; the full 256^3 fluctuating
suspension (36,669 particles, 476,697 blobs, kT = 1e-3) is checked on sampled blob forces and
on properties of the flow.
"""
import numpy as np
import pytest

import oracle
from helpers import TOL, min_image, assert_positions, rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1407_5600_gb300 as mb  # noqa: E402
from paper_1407_5600_gb300 import workloads as wl  # noqa: E402

LONG = [(8, 8, 256), (8, 256, 8), (256, 8, 8)]          # (nz, ny, nx)


def _oracle_grid(d: mb.GridDesc):
    return oracle.Grid(d.nx, d.ny, d.nz, h=d.h, rho=d.rho, eta=d.eta, dt=d.dt,
                       mean_mode=d.mean_mode)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape", LONG)
def test_fluid_update_parity_on_256_sides(prec, shape):
    nz, ny, nx = shape
    d = mb.GridDesc(nx, ny, nz, h=0.9, rho=1.1, eta=0.8, dt=0.07, precision=prec, mean_mode=0)
    g = _oracle_grid(d)
    v = oracle.fluid_update(oracle.Grid(nx, ny, nz, rho=1.0, eta=0.0, dt=1.0), g.zeros(),
                            wl.random_field(shape, 3))
    v = v.astype(d.grid_dtype).astype(np.float64)
    f = wl.random_field(shape, 4, scale=0.3).astype(d.grid_dtype).astype(np.float64)
    axis = int(np.argmax([nx, ny, nz]))
    body = (0.2, (axis + 1) % 3, axis, 2)
    with mb.Multiblob(d) as sim:
        vn = to_np(sim.fluid_update(v[None].astype(d.grid_dtype), f[None].astype(d.grid_dtype),
                                    body_force=body))[0]
    assert rel_l2(vn, oracle.fluid_update(g, v, f, body=body)) < TOL[prec]


def _particle_in(shape, seed, stretch=0.05):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    L = np.array([nx, ny, nz], dtype=np.float64)
    s = wl.build_particles(rng.uniform(0, 1, size=3) * L, 1.0, rng, L)
    s.pos = np.mod(s.pos + rng.normal(scale=stretch, size=s.pos.shape), L)
    s.ext = rng.normal(scale=1e-3, size=s.pos.shape)
    return s


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape", LONG)
def test_thermal_step_parity_on_256_sides(prec, shape):
    nz, ny, nx = shape
    s = _particle_in(shape, 7)
    d = mb.GridDesc(nx, ny, nz, dt=0.05, precision=prec, mean_mode=0, kT=1e-3, seed=13)
    nsteps = 4
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        sim.step(nsteps, ext_blob_force=s.ext)
        q, v = to_np(sim.blob_positions()), to_np(sim.velocity_field()).astype(np.float64)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest,
                               s.k_spring, ext=s.ext, kT=d.kT, seed=d.seed)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]


@pytest.mark.parametrize("prec,stretch,tol", [(1, 0.05, TOL[1]), (0, 0.0, TOL[0]),
                                               (0, 0.05, 5e-5)])
def test_stokes_step_parity_on_a_256_side(prec, stretch, tol):
    """A particle in an 8 x 256 x 8 box.  In the Stokes limit the flow answers the forces
    directly, and in a long thin periodic box the response to a net force grows with the box
    length.  The springs' internal forces cancel exactly only in exact arithmetic: stretched
    by 0.05h (forces ~ k 0.05 against external forces of 1e-3), their FP32 rounding leaves a
    spurious net force whose amplified flow reaches ~2e-5 of the field, so the FP32 grid is
    held to 5e-5 there and to the usual 1e-5 with the particle at rest shape."""
    shape = (8, 256, 8)
    nz, ny, nx = shape
    s = _particle_in(shape, 8, stretch)
    d = mb.GridDesc(nx, ny, nz, dt=0.05, precision=prec, mean_mode=1, integrator=1)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        sim.step(3, ext_blob_force=s.ext)
        q, v = to_np(sim.blob_positions()), to_np(sim.velocity_field()).astype(np.float64)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.stokes_step(g, 3, s.pos, s.pid, s.bonds, s.rest, s.k_spring,
                                      ext=s.ext)
    assert_positions(q, q_ref, s.pos, g.L, 3, tol)
    assert rel_l2(v[0], v_ref) < tol


@pytest.fixture(scope="module")
def thermal256():
    return wl.fluctuating_suspension(n=256, a=3.2, phi=0.30, kT=1e-3, seed=5)


def test_full_size_fluctuating_suspension(thermal256):
    """256^3, 476,697 blobs, kT = 1e-3, FP32 grid: sampled blob forces against the oracle,
    a divergence-free zero-mean flow of thermal size, and bounded blob motion."""
    spec, s = thermal256
    assert s.n_particles == 36669 and len(s.pos) == 476697
    n = spec.nx
    d = mb.GridDesc(n, n, n, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt, precision=0,
                    mean_mode=spec.mean_mode, kT=spec.kT, seed=17)
    nsteps = 4
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(nsteps)
        assert sim.step_index == nsteps
        F, qh = (to_np(x) for x in sim.last_forces())
        q = to_np(sim.blob_positions())
        v = to_np(sim.velocity_field())[0].astype(np.float64)
    g = oracle.Grid(n, n, n, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt)
    # blob forces at the last midpoints, on a sample of blobs
    idx = np.random.default_rng(0).choice(len(qh), size=1500, replace=False)
    F_ref = oracle.bond_forces(g, qh, s.bonds, s.rest, s.k_spring)[idx] \
        + oracle.pair_forces_subset(g, qh, s.pid, s.k_rep, s.r_cut, idx)
    assert np.max(np.abs(F[idx] - F_ref)) < TOL[0] * max(np.max(np.abs(F_ref)), 1e-30)
    # the flow: finite, divergence-free to FP32 rounding, no net momentum
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(q))
    div = sum(np.roll(v[a], -1, axis=2 - a) - v[a] for a in range(3)) / spec.h
    assert np.max(np.abs(div)) < 1e-4 * np.max(np.abs(v)) / spec.h
    assert np.max(np.abs(v.mean(axis=(1, 2, 3)))) < 1e-5 * np.sqrt(spec.kT)
    # thermal size: below the equipartition level (the slow modes have not filled yet) and
    # far from zero
    var = (v ** 2).mean()
    assert 0.05 * (2.0 / 3.0) * spec.kT < var < 1.05 * (2.0 / 3.0) * spec.kT
    disp = np.abs(min_image(q - s.pos, n * spec.h))
    assert np.max(disp) < 0.5 * spec.h



def test_full_size_fluctuating_steps_match_oracle(thermal256):
    """The 256^3 fluctuating suspension (476,697 blobs, kT = 1e-3, FP32 grid, five-pass FFT),
    element by element: two steps, positions, fluid and blob velocities against two oracle steps
    drawing the same thermal stress (Philox keyed by seed 17, steps 0 and 1)."""
    spec, s = thermal256
    n = spec.nx
    d = mb.GridDesc(n, n, n, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt, precision=0,
                    mean_mode=spec.mean_mode, kT=spec.kT, seed=17)
    nsteps = 2
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(nsteps)
        q = to_np(sim.blob_positions())
        v = to_np(sim.velocity_field())[0].astype(np.float64)
        u = to_np(sim.blob_velocities())
    g = oracle.Grid(n, n, n, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt,
                    mean_mode=spec.mean_mode)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, kT=spec.kT, seed=17)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[0])
    assert rel_l2(v, v_ref) < TOL[0]
    assert rel_l2(u, oracle.interp(g, q_ref, v_ref)) < TOL[0]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape", [(16, 16, 16), (8, 16, 128), (4, 4, 4), (32, 8, 64),
                                   (128, 4, 8)])
def test_five_pass_fluid_update_parity(monkeypatch, prec, shape):
    """The five-pass pipeline (the one sides above 128 take) on ordinary shapes, selected with
    MB_FFT_PASSES=5."""
    monkeypatch.setenv("MB_FFT_PASSES", "5")
    nz, ny, nx = shape
    d = mb.GridDesc(nx, ny, nz, h=1.1, rho=0.9, eta=0.7, dt=0.05, precision=prec, mean_mode=0)
    g = _oracle_grid(d)
    v = oracle.fluid_update(oracle.Grid(nx, ny, nz, rho=1.0, eta=0.0, dt=1.0), g.zeros(),
                            wl.random_field(shape, 5))
    v = v.astype(d.grid_dtype).astype(np.float64)
    f = wl.random_field(shape, 6, scale=0.3).astype(d.grid_dtype).astype(np.float64)
    body = (0.1, 0, 2, 1)
    with mb.Multiblob(d) as sim:
        vn = to_np(sim.fluid_update(v[None].astype(d.grid_dtype), f[None].astype(d.grid_dtype),
                                    body_force=body))[0]
    assert rel_l2(vn, oracle.fluid_update(g, v, f, body=body)) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
def test_five_pass_step_parity(monkeypatch, prec):
    monkeypatch.setenv("MB_FFT_PASSES", "5")
    spec, s = wl.dense_suspension(n=32, a=2.2, phi=0.40, seed=5, mc_sweeps=3)
    d = mb.GridDesc(32, 32, 32, dt=spec.dt, precision=prec, mean_mode=0, kT=1e-3, seed=3)
    rng = np.random.default_rng(4)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(3, ext_blob_force=ext, body_force=s.body)
        q, v = to_np(sim.blob_positions()), to_np(sim.velocity_field()).astype(np.float64)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, 3, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, ext=ext, body=s.body, kT=d.kT, seed=d.seed)
    assert_positions(q, q_ref, s.pos, g.L, 3, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]
