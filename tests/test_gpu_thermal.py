"""GPU parity of the fluctuating ICM step (kT > 0: the thermal stress of Sec. 3 / Eq. vf)
against the FP64 oracle, drawing the same Philox noise on both sides.

Tolerances as for the deterministic steps: relative L2 1e-10 (FP64 grid), 1e-5 (FP32 grid).
The equipartition check of Eq. (ef) runs on the GPU path alone (statistical).
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
                       mean_mode=d.mean_mode)


def _empty(L):
    return wl.Suspension(pos=np.zeros((0, 3)), pid=np.zeros(0, dtype=np.int32),
                         bonds=np.zeros((0, 2), dtype=np.int32), rest=np.zeros(0),
                         n_particles=0, a=0.0, L=np.asarray(L, dtype=np.float64))


def _run(d, susp_list, nsteps, ext=None, body=None, calls=1):
    with mb.Multiblob(d) as sim:
        for b, s in enumerate(susp_list):
            sim.set_particles(b, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        for _ in range(calls):
            sim.step(nsteps // calls, ext_blob_force=ext, body_force=body)
        return (to_np(sim.blob_positions()), to_np(sim.velocity_field()).astype(np.float64),
                sim.step_index)


@pytest.mark.parametrize("prec", [1, 0])
def test_fluid_noise_parity_per_box(prec):
    """No blobs: the fluid is driven by the thermal stress alone; each box draws its own
    stream (the box index is part of the Philox counter)."""
    d = mb.GridDesc(16, 8, 32, batch=2, h=0.8, rho=1.2, eta=0.9, dt=0.1, precision=prec,
                    mean_mode=0, kT=1e-3, seed=7)
    g = _oracle_grid(d)
    empty = _empty(g.L)
    _, v, idx = _run(d, [empty, empty], 3)
    assert idx == 3
    none = dict(pid=np.zeros(0, np.int32), bonds=np.zeros((0, 2), np.int32), rest=np.zeros(0),
                k_spring=0.0)
    for b in range(2):
        _, v_ref = oracle.step(g, 3, np.zeros((0, 3)), g.zeros(), kT=d.kT, seed=d.seed,
                               step0=0, box=b, **none)
        assert rel_l2(v[b], v_ref) < TOL[prec]
    assert rel_l2(v[0], v[1]) > 0.5          # independent streams


@pytest.mark.parametrize("prec", [1, 0])
def test_thermal_step_parity_single_particle(prec):
    spec, s = wl.single_particle(n=32, a=1.0, seed=1)
    d = mb.GridDesc(32, 32, 32, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt,
                    precision=prec, mean_mode=spec.mean_mode, kT=1e-3, seed=11)
    nsteps = 8
    q, v, _ = _run(d, [s], nsteps, ext=s.ext)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest,
                               s.k_spring, ext=s.ext, kT=d.kT, seed=d.seed)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
def test_thermal_step_parity_dense_with_repulsion_and_body_force(prec):
    spec, s = wl.dense_suspension(n=32, a=2.2, phi=0.40, seed=5, mc_sweeps=3)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, h=spec.h, rho=spec.rho, eta=spec.eta,
                    dt=spec.dt, precision=prec, mean_mode=spec.mean_mode, kT=1e-3, seed=2)
    rng = np.random.default_rng(9)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    s.pos = np.mod(s.pos + rng.normal(scale=0.05, size=s.pos.shape), s.L)
    nsteps = 3
    q, v, _ = _run(d, [s], nsteps, ext=ext, body=s.body)
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest,
                               s.k_spring, s.k_rep, s.r_cut, ext=ext, body=s.body, kT=d.kT,
                               seed=d.seed)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
def test_step_index_resumes_the_noise(prec):
    """Run 6 steps in one go; then 3 steps, a checkpoint (positions, field, step index) and
    3 more steps in a fresh context: the same state.  Also one call of 6 steps against six
    calls of one (captured graphs must draw fresh noise on every replay)."""
    spec, s = wl.single_particle(n=16, a=1.0, seed=3)
    d = mb.GridDesc(16, 16, 16, dt=0.05, precision=prec, mean_mode=1, kT=2e-3, seed=5)
    q6, v6, i6 = _run(d, [s], 6, ext=s.ext)
    q6b, v6b, i6b = _run(d, [s], 6, ext=s.ext, calls=6)
    assert i6 == i6b == 6
    tol = 1e-12 if prec == 1 else 1e-6
    assert rel_l2(v6b, v6) < tol
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        sim.step(3, ext_blob_force=s.ext)
        q3, v3 = to_np(sim.blob_positions()), to_np(sim.velocity_field())
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        sim.set_positions(q3)
        sim.set_velocity_field(v3)
        sim.step_index = 3
        sim.step(3, ext_blob_force=s.ext)
        qr, vr = to_np(sim.blob_positions()), to_np(sim.velocity_field()).astype(np.float64)
        assert sim.step_index == 6
    assert rel_l2(vr, v6) < tol
    assert_positions(qr, q6, s.pos, np.array([16.0] * 3), 6, tol)


def test_fluid_equipartition_fp32():
    """Eq. (ef) on the FP32 path: the per-component variance of the fluid velocity is
    (kT / (rho h^3)) (1/N) sum over k != 0 of P_aa(k)."""
    n, kT = 32, 1e-3
    d = mb.GridDesc(n, n, n, dt=0.5, precision=0, mean_mode=0, kT=kT, seed=21)
    acc = np.zeros(3)
    m = 0
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, np.zeros((0, 3)), np.zeros(0, np.int32),
                          np.zeros((0, 2), np.int32), np.zeros(0), 0.0)
        sim.step(60)
        for _ in range(200):
            sim.step(3)
            v = sim.velocity_field()[0].double()
            acc += (v ** 2).mean(dim=(1, 2, 3)).cpu().numpy()
            m += 1
    var = acc / m
    s2 = 4.0 * np.sin(np.pi * np.arange(n) / n) ** 2
    Sx, Sy, Sz = np.meshgrid(s2, s2, s2, indexing="ij")
    lam = Sx + Sy + Sz
    lam[0, 0, 0] = 1.0
    frac = []
    for Sa in (Sx, Sy, Sz):
        P = 1.0 - Sa / lam
        P[0, 0, 0] = 0.0
        frac.append(P.sum() / lam.size)
    want = kT * np.array(frac)
    assert np.all(np.abs(var / want - 1.0) < 0.02), (var, want)


def test_stokes_integrator_rejects_kT():
    with pytest.raises(mb.MBError, match="deterministic"):
        mb.Multiblob(mb.GridDesc(8, 8, 8, integrator=1, mean_mode=1, kT=1e-3))


@pytest.mark.parametrize("prec", [1, 0])
def test_particle_velocity_autocorrelation_matches_oracle(prec):
    """Thermal 32^3 run (the small-box check of the fluctuating suspension): the particle
    velocities U0(t), and so their autocorrelation, follow the oracle step by step with the
    same Philox stream."""
    spec, s = wl.dilute_random(n=32, n_particles=6, a=2.0, seed=12)
    d = mb.GridDesc(32, 32, 32, dt=0.05, precision=prec, mean_mode=0, kT=1e-3, seed=31)
    T = 60
    U_gpu = []
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        for _ in range(T):
            sim.step(1)
            U_gpu.append(to_np(sim.particle_velocities()[0]))
    g = _oracle_grid(d)
    q, v = s.pos.copy(), g.zeros()
    U_ref = []
    for t in range(T):
        q, v = oracle.step(g, 1, q, v, s.pid, s.bonds, s.rest, s.k_spring, kT=d.kT,
                           seed=d.seed, step0=t)
        U_ref.append(oracle.particle_velocities(g, q, oracle.interp(g, q, v), s.pid,
                                                s.n_particles)[0])
    U_gpu, U_ref = np.array(U_gpu), np.array(U_ref)
    assert rel_l2(U_gpu, U_ref) < TOL[prec]

    def vaf(U):
        return np.array([np.mean(np.sum(U[:T - k] * U[k:], axis=-1)) for k in range(T // 2)])
    assert rel_l2(vaf(U_gpu), vaf(U_ref)) < 4 * TOL[prec]
