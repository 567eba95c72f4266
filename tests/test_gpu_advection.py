"""GPU parity of the convective stress (advection = 1: rho v v of Eq. vf, explicit at v^n)
against the FP64 oracle: the standalone fluid update and whole ICM steps with blobs, body
force and thermal stress.  Tolerances: relative L2 1e-10 (FP64 grid), 1e-5 (FP32 grid).
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


def _oracle_grid(d: mb.GridDesc):
    return oracle.Grid(d.nx, d.ny, d.nz, h=d.h, rho=d.rho, eta=d.eta, dt=d.dt,
                       mean_mode=d.mean_mode, advection=d.advection)


def _field(shape, seed, scale):
    nz, ny, nx = shape
    g0 = oracle.Grid(nx, ny, nz, rho=1.0, eta=0.0, dt=1.0)
    return oracle.fluid_update(g0, g0.zeros(), wl.random_field(shape, seed, scale))


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape,h,mean_mode", [((16, 16, 16), 1.0, 0), ((8, 16, 32), 0.6, 1),
                                               ((8, 8, 256), 1.0, 0)])
def test_fluid_update_with_advection_parity(prec, shape, h, mean_mode):
    nz, ny, nx = shape
    d = mb.GridDesc(nx, ny, nz, h=h, rho=1.3, eta=0.4, dt=0.2, precision=prec,
                    mean_mode=mean_mode, advection=1)
    v = _field(shape, 7, 0.5).astype(d.grid_dtype).astype(np.float64)
    f = wl.random_field(shape, 8, scale=0.1).astype(d.grid_dtype).astype(np.float64)
    body = (0.05, 1, 2, 1)
    g = _oracle_grid(d)
    ref = oracle.fluid_update(g, v, f, body=body)
    ref_no_f = oracle.fluid_update(g, v, g.zeros())
    with mb.Multiblob(d) as sim:
        out = to_np(sim.fluid_update(v[None].astype(d.grid_dtype), f[None].astype(d.grid_dtype),
                                     body_force=body))[0]
        out_no_f = to_np(sim.fluid_update(v[None].astype(d.grid_dtype)))[0]
    assert rel_l2(out, ref) < TOL[prec]
    assert rel_l2(out_no_f, ref_no_f) < TOL[prec]
    # the convective term changed the result
    g0 = oracle.Grid(nx, ny, nz, h=h, rho=1.3, eta=0.4, dt=0.2, mean_mode=mean_mode)
    assert rel_l2(oracle.fluid_update(g0, v, f, body=body), ref) > 1e-3


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("kT", [0.0, 1e-3])
def test_step_with_advection_parity(prec, kT):
    spec, s = wl.dense_suspension(n=32, a=2.2, phi=0.40, seed=5, mc_sweeps=3)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, h=spec.h, rho=spec.rho, eta=0.2, dt=spec.dt,
                    precision=prec, mean_mode=spec.mean_mode, advection=1, kT=kT, seed=4)
    rng = np.random.default_rng(3)
    ext = rng.normal(scale=1e-2, size=s.pos.shape)
    s.pos = np.mod(s.pos + rng.normal(scale=0.05, size=s.pos.shape), s.L)
    body = (0.05, 0, 2, 1)
    v0 = _field((32, 32, 32), 9, 0.3)
    nsteps = 4
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.set_velocity_field(v0[None].astype(d.grid_dtype))
        sim.step(nsteps, ext_blob_force=ext, body_force=body)
        q, v = to_np(sim.blob_positions()), to_np(sim.velocity_field()).astype(np.float64)
    g = _oracle_grid(d)
    v0r = v0.astype(d.grid_dtype).astype(np.float64)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, v0r, s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, ext=ext, body=body, kT=kT, seed=d.seed)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]


def test_stokes_integrator_rejects_advection():
    with pytest.raises(mb.MBError, match="convective"):
        mb.Multiblob(mb.GridDesc(8, 8, 8, integrator=1, mean_mode=1, advection=1))


@pytest.mark.parametrize("kw", [dict(advection=1), dict(kT=1e-3)])
def test_step_adjoint_rejects_convective_and_thermal_stress(kw):
    spec, s = wl.single_particle(n=16, a=1.0, seed=2)
    with mb.Multiblob(mb.GridDesc(16, 16, 16, precision=1, **kw)) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        v = np.zeros((3, 16, 16, 16))
        with pytest.raises(mb.MBError, match="thermal and convective"):
            mb.adjoint_step(sim.ctx, s.pos.copy(), v, None, None, np.zeros_like(s.pos),
                            np.zeros_like(v))
