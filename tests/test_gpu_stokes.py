"""GPU parity of the Stokes-limit integrator (integrator 1: the steady zero-mean Stokes flow of
the current forces, blobs advanced by the explicit midpoint rule) against the FP64 oracle.

Tolerances as for the inertial steps: relative L2 1e-10 (FP64 grid), 1e-5 (FP32 grid with
FP64 blob positions).
"""
import numpy as np
import pytest

import oracle
from helpers import TOL, assert_positions, rel_l2, to_np

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1407_5600_gb300 as mb  # noqa: E402
from paper_1407_5600_gb300 import workloads as wl  # noqa: E402


def _desc(n, prec, **kw):
    nx, ny, nz = n
    kw.setdefault("mean_mode", 1)
    return mb.GridDesc(nx, ny, nz, precision=prec, integrator=1, **kw)


def _oracle_grid(d: mb.GridDesc):
    return oracle.Grid(d.nx, d.ny, d.nz, h=d.h, rho=d.rho, eta=d.eta, dt=d.dt,
                       mean_mode=d.mean_mode)


def _run(d, susp_list, nsteps, ext=None, body=None):
    with mb.Multiblob(d) as sim:
        for b, s in enumerate(susp_list):
            sim.set_particles(b, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(nsteps, ext_blob_force=ext, body_force=body)
        q = to_np(sim.blob_positions())
        v = to_np(sim.velocity_field()).astype(np.float64)
        u = to_np(sim.blob_velocities())
        U, _ = sim.particle_velocities()
        return q, v, u, to_np(U)


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("n,h", [((16, 16, 16), 1.0), ((32, 8, 16), 0.7), ((8, 64, 128), 1.0)])
def test_stokes_solve_parity(prec, n, h):
    d = _desc(n, prec, h=h, eta=1.3)
    shape = (n[2], n[1], n[0])
    f = wl.random_field(shape, 31, scale=0.5).astype(d.grid_dtype).astype(np.float64)
    with mb.Multiblob(d) as sim:
        v = to_np(sim.fluid_update(None, f[None].astype(d.grid_dtype)))[0].astype(np.float64)
    ref = oracle.stokes_solve(_oracle_grid(d), f)
    assert rel_l2(v, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
def test_stokes_step_single_particle(prec):
    spec, s = wl.single_particle(n=32, a=1.0, seed=1)
    d = _desc((32, 32, 32), prec, h=spec.h, eta=spec.eta, dt=spec.dt)
    nsteps = 10
    q, v, u, U = _run(d, [s], nsteps, ext=s.ext)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.stokes_step(g, nsteps, s.pos, s.pid, s.bonds, s.rest, s.k_spring,
                                      ext=s.ext)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]
    # the blob velocities read back are J(q^{n+1}) of the last flow
    assert rel_l2(u, oracle.interp(g, q_ref, v_ref)) < TOL[prec]
    U_ref, _ = oracle.particle_velocities(g, q_ref, oracle.interp(g, q_ref, v_ref), s.pid, 1)
    assert rel_l2(U, U_ref) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
def test_stokes_step_dense_with_repulsion_and_body_force(prec):
    spec, s = wl.dense_suspension(n=32, a=2.2, phi=0.40, seed=5, mc_sweeps=3)
    d = _desc((spec.nx, spec.ny, spec.nz), prec, h=spec.h, eta=spec.eta, dt=spec.dt)
    rng = np.random.default_rng(19)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    s.pos = np.mod(s.pos + rng.normal(scale=0.05, size=s.pos.shape), s.L)
    nsteps = 3
    q, v, _, _ = _run(d, [s], nsteps, ext=ext, body=s.body)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.stokes_step(g, nsteps, s.pos, s.pid, s.bonds, s.rest, s.k_spring,
                                      s.k_rep, s.r_cut, ext=ext, body=s.body)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]
    assert np.max(np.abs(oracle.pair_forces(g, q_ref, s.pid, s.k_rep, s.r_cut))) > 0


def test_stokes_step_full_size_dense_fp32():
    """The benchmark's dense 128^3 suspension (244,504 blobs), two Stokes-limit steps in FP32
    grid mode: the solve divides by eta lambda down to lambda_min, so FP32 errors of the
    spread forces reach the lowest modes amplified; the tile's fixed-point scale keeps them
    within 1e-5 of the oracle."""
    spec, s = wl.dense_suspension(n=128)
    d = _desc((spec.nx, spec.ny, spec.nz), 0, h=spec.h, eta=spec.eta, dt=spec.dt)
    nsteps = 2
    q, v, _, _ = _run(d, [s], nsteps, body=s.body)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.stokes_step(g, nsteps, s.pos, s.pid, s.bonds, s.rest, s.k_spring,
                                      s.k_rep, s.r_cut, body=s.body)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[0])
    assert rel_l2(v[0], v_ref) < TOL[0]


@pytest.mark.parametrize("prec", [1, 0])
def test_stokes_batched_boxes_match_independent_runs(prec):
    B = 3
    boxes = [wl.gap_sweep_box(b, n_boxes=B, n=16, a=1.6)[1] for b in range(B)]
    d = _desc((16, 16, 16), prec, batch=B, dt=0.05)
    nsteps = 6
    q, v, _, _ = _run(d, boxes, nsteps, ext=np.concatenate([s.ext for s in boxes]))
    g = _oracle_grid(d)
    off = 0
    for b, s in enumerate(boxes):
        q_ref, v_ref = oracle.stokes_step(g, nsteps, s.pos, s.pid, s.bonds, s.rest, s.k_spring,
                                          ext=s.ext)
        assert_positions(q[off:off + s.n_blobs], q_ref, s.pos, g.L, nsteps, TOL[prec])
        assert rel_l2(v[b], v_ref) < TOL[prec]
        off += s.n_blobs


def test_stokes_empty_box_and_single_blob_with_body_force():
    """Box 0 holds no blobs, so its flow is the steady flow of the body force alone (the
    closed form of the oracle pins); box 1 holds one forced blob on the periodic seam."""
    body = (0.3, 0, 2, 1)
    L = np.array([16.0, 16, 16])
    empty = wl.Suspension(pos=np.zeros((0, 3)), pid=np.zeros(0, dtype=np.int32),
                          bonds=np.zeros((0, 2), dtype=np.int32), rest=np.zeros(0),
                          n_particles=0, a=0.0, L=L)
    single = wl.Suspension(pos=np.array([[15.999999999, 0.0, 7.5]]),
                           pid=np.zeros(1, dtype=np.int32),
                           bonds=np.zeros((0, 2), dtype=np.int32), rest=np.zeros(0),
                           n_particles=1, a=0.0, L=L)
    ext = np.array([[0.1, -0.2, 0.05]])
    g = oracle.Grid(16, 16, 16, eta=1.7, dt=0.1, mean_mode=1)
    none = dict(pid=np.zeros(1, np.int32), bonds=np.zeros((0, 2), np.int32), rest=np.zeros(0),
                k_spring=0.0)
    _, v0_ref = oracle.stokes_step(g, 3, np.array([[1.0, 2.0, 3.0]]), body=body, **none)
    q1_ref, v1_ref = oracle.stokes_step(g, 3, single.pos, ext=ext, body=body, **none)
    for prec in (1, 0):
        d = _desc((16, 16, 16), prec, batch=2, eta=1.7, dt=0.1)
        q, v, _, _ = _run(d, [empty, single], 3, ext=ext, body=body)
        assert rel_l2(v[0], v0_ref) < TOL[prec]
        assert rel_l2(v[1], v1_ref) < TOL[prec]
        assert_positions(q, q1_ref, single.pos, g.L, 3, TOL[prec])


def test_stokes_invalid_configurations():
    with pytest.raises(mb.MBError, match="mean_mode"):
        mb.Multiblob(_desc((8, 8, 8), 1, mean_mode=0))
    with pytest.raises(mb.MBError, match="integrator"):
        mb.Multiblob(mb.GridDesc(8, 8, 8, integrator=2))
    spec, s = wl.single_particle(n=16, a=1.0, seed=2)
    with mb.Multiblob(_desc((16, 16, 16), 1)) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        v = np.zeros((3, 16, 16, 16))
        with pytest.raises(mb.MBError, match="inertial coupling"):
            mb.adjoint_step(sim.ctx, s.pos.copy(), v, None, None, np.zeros_like(s.pos),
                            np.zeros_like(v))


@pytest.mark.parametrize("prec", [1, 0])
def test_torque_driven_rotation_parity(prec):
    """A couple of blob forces on a d = 2h icosahedron (the rotlet experiment): the particle
    angular velocity Omega and drift U0 follow the oracle."""
    n = 32
    rng = np.random.default_rng(3)
    a = 2.0 * np.sqrt(10 + 2 * np.sqrt(5)) / 4
    s = wl.build_particles(np.array([13.3, 15.1, 16.7]), a, rng, np.array([32.0] * 3))
    r = s.pos - s.pos.mean(axis=0)
    T = np.array([2e-4, -5e-4, 1e-3])
    F = np.cross(T, r) / np.sum(r ** 2) * 1.5            # a couple (zero net force)
    d = _desc((n, n, n), prec, dt=0.05)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, 200.0)
        sim.step(12, ext_blob_force=F)
        U, W = (to_np(x) for x in sim.particle_velocities())
        q = to_np(sim.blob_positions())
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.stokes_step(g, 12, s.pos, s.pid, s.bonds, s.rest, 200.0, ext=F)
    U_ref, W_ref = oracle.particle_velocities(g, q_ref, oracle.interp(g, q_ref, v_ref), s.pid, 1)
    assert_positions(q, q_ref, s.pos, g.L, 12, TOL[prec])
    assert rel_l2(W, W_ref) < TOL[prec]
    assert np.max(np.abs(U - U_ref)) < TOL[prec] * np.max(np.abs(W_ref)) * a
