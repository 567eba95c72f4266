"""Pins of the oracle's forces, time step and particle observables (no GPU).

- Bond and repulsion forces equal minus the gradient of their energies (central differences)
  and sum to zero (action-reaction); repulsion acts only between different particles.
- The step conserves momentum bookkeeping rho h^3 sum v = t sum F_ext (internal forces cancel),
  is invariant under a shift of everything by one mesh cell, and keeps the stiff icosahedron
  rigid (bond lengths within O(F/k) of rest, Sec. 2 and Sec. 4 on stiff springs).
- Particle velocities of an exactly rigid blob velocity field u_i = U + Omega x s_i
  return U and Omega (Sec. 2 and Sec. 3.2).
"""
import numpy as np
import pytest

import oracle as mb
from paper_1407_5600_gb300 import workloads as wl


def _min_img(d, L):
    return d - L * np.round(d / L)


def _bond_energy(g, q, bonds, rest, k):
    r = _min_img(q[bonds[:, 0]] - q[bonds[:, 1]], g.L)
    return 0.5 * k * np.sum((np.linalg.norm(r, axis=1) - rest) ** 2)


def _rep_energy(g, q, pid, krep, rcut):
    e = 0.0
    for i in range(len(q)):
        d = _min_img(q[i] - q[i + 1:], g.L)
        r = np.linalg.norm(d, axis=1)
        m = (r < rcut) & (pid[i + 1:] != pid[i])
        e += 0.5 * krep * np.sum((rcut - r[m]) ** 2)
    return e


def test_bond_forces_gradient_and_balance():
    g = mb.Grid(16, 16, 16)
    rng = np.random.default_rng(4)
    s = wl.build_particles(rng.uniform(0, 16, size=(3, 3)), 1.6, rng, g.L)
    q = s.pos + rng.normal(scale=0.05, size=s.pos.shape)
    q = np.mod(q, g.L)
    F = mb.bond_forces(g, q, s.bonds, s.rest, 100.0)
    assert np.max(np.abs(F.sum(0))) < 1e-12
    eps = 1e-6
    for b in rng.choice(len(q), 8, replace=False):
        for a in range(3):
            qp, qm = q.copy(), q.copy()
            qp[b, a] += eps
            qm[b, a] -= eps
            dE = (_bond_energy(g, qp, s.bonds, s.rest, 100.0)
                  - _bond_energy(g, qm, s.bonds, s.rest, 100.0)) / (2 * eps)
            assert abs(F[b, a] + dE) < 1e-6 * max(1.0, abs(dE))


def test_pair_forces_gradient_balance_and_subset():
    g = mb.Grid(8, 8, 8)
    rng = np.random.default_rng(5)
    q = rng.uniform(0, 8, size=(60, 3))
    pid = (np.arange(60) // 13).astype(np.int32)
    F = mb.pair_forces(g, q, pid, 50.0, 1.2)
    assert np.max(np.abs(F.sum(0))) < 1e-12
    assert np.any(np.abs(F) > 0)
    eps = 1e-6
    for b in rng.choice(60, 8, replace=False):
        for a in range(3):
            qp, qm = q.copy(), q.copy()
            qp[b, a] += eps
            qm[b, a] -= eps
            dE = (_rep_energy(g, qp, pid, 50.0, 1.2) - _rep_energy(g, qm, pid, 50.0, 1.2)) / (2 * eps)
            assert abs(F[b, a] + dE) < 1e-5 * max(1.0, abs(dE))
    idx = np.array([3, 17, 59, 0])
    assert np.array_equal(mb.pair_forces_subset(g, q, pid, 50.0, 1.2, idx), F[idx])
    # same-particle pairs never repel
    F1 = mb.pair_forces(g, q, np.zeros(60, dtype=np.int32), 50.0, 1.2)
    assert np.all(F1 == 0.0)


@pytest.mark.parametrize("shape,h,r_cut,nblob", [
    ((16, 16, 16), 1.0, 1.0, 3000),      # many bins, dense
    ((8, 12, 20), 0.7, 1.3, 1500),       # non-cubic, h != 1
    ((8, 8, 8), 1.0, 2.9, 400),          # two bins along each axis: the definition is used
    ((32, 4, 16), 1.0, 0.5, 2000),       # thin box
])
def test_binned_repulsion_equals_all_pairs_to_the_bit(shape, h, r_cut, nblob):
    """The bins only skip pairs farther apart than r_cut; the sum over the rest runs in the
    definition's order, so the two agree exactly, also for blobs on and outside the box faces."""
    nz, ny, nx = shape
    g = mb.Grid(nx, ny, nz, h=h)
    rng = np.random.default_rng(nblob)
    q = rng.uniform(0, 1, size=(nblob, 3)) * g.L
    q[:40] = q[:40] * 1e-3                                   # a cluster at the origin corner
    q[40:60] = g.L - q[40:60] * 1e-3                         # and just below the far faces
    q[60:70] += g.L                                          # outside the box
    q[70:80] -= 2 * g.L
    q[80:90, 0] = np.round(q[80:90, 0] / (r_cut * 1.000001)) * r_cut * 1.000001   # on bin faces
    pid = (np.arange(nblob) // 13).astype(np.int32)
    Fb = mb.pair_forces(g, q, pid, 75.0, r_cut)
    Fa = mb.pair_forces_brute(g, q, pid, 75.0, r_cut)
    assert np.count_nonzero(Fa) > 0
    assert np.array_equal(Fa, Fb)
    idx = rng.choice(nblob, 50, replace=False)
    assert np.array_equal(mb.pair_forces_subset(g, q, pid, 75.0, r_cut, idx), Fa[idx])


def _single(n=16, a=1.0, seed=1):
    spec, s = wl.single_particle(n=n, a=a, seed=seed)
    g = mb.Grid(spec.nx, spec.ny, spec.nz, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt,
                mean_mode=0)
    return g, s


def test_step_momentum_and_rigidity():
    g, s = _single()
    v0 = np.zeros((3,) + g.shape)
    nsteps = 20
    q, v = mb.step(g, nsteps, s.pos, v0, s.pid, s.bonds, s.rest, s.k_spring, ext=s.ext)
    P = g.rho * g.h ** 3 * v.sum((1, 2, 3))
    expect = nsteps * g.dt * s.ext.sum(0)
    assert np.max(np.abs(P - expect)) < 1e-12 * np.max(np.abs(expect))
    r = np.linalg.norm(_min_img(q[s.bonds[:, 0]] - q[s.bonds[:, 1]], g.L), axis=1)
    assert np.max(np.abs(r - s.rest) / s.rest) < 1e-3
    # the particle moved along +x
    dq = _min_img(q - s.pos, g.L).mean(0)
    assert dq[0] > 0 and abs(dq[1]) < 0.05 * dq[0] and abs(dq[2]) < 0.05 * dq[0]


def test_step_shift_by_one_cell_invariance():
    g, s = _single(n=12)
    rng = np.random.default_rng(7)
    v0 = mb.fluid_update(mb.Grid(12, 12, 12, rho=1.0, eta=0.0, dt=1.0), g.zeros(),
                         wl.random_field(g.shape, 3, scale=1e-3))
    q1, v1 = mb.step(g, 3, s.pos, v0, s.pid, s.bonds, s.rest, s.k_spring, ext=s.ext)
    shift = np.array([g.h, 0, 0])
    qs = np.mod(s.pos + shift, g.L)
    vs = np.roll(v0, 1, axis=3)
    q2, v2 = mb.step(g, 3, qs, vs, s.pid, s.bonds, s.rest, s.k_spring, ext=s.ext)
    assert np.max(np.abs(_min_img(q2 - (q1 + shift), g.L))) < 1e-12
    assert np.max(np.abs(np.roll(v1, 1, axis=3) - v2)) < 1e-13
    del rng


def test_step_mean_mode_zero_frame():
    """With no convection, J of a constant is that constant: holding the mean at zero changes
    the first step's blob velocities only by the mean flow of the conserving run."""
    g, s = _single(n=12)
    g0 = mb.Grid(12, 12, 12, dt=g.dt, mean_mode=0)
    g1 = mb.Grid(12, 12, 12, dt=g.dt, mean_mode=1)
    v0 = g.zeros()
    qa, va = mb.step(g0, 1, s.pos, v0, s.pid, s.bonds, s.rest, s.k_spring, ext=s.ext)
    qb, vb = mb.step(g1, 1, s.pos, v0, s.pid, s.bonds, s.rest, s.k_spring, ext=s.ext)
    vbar = va.mean((1, 2, 3))
    assert np.max(np.abs(va - vbar[:, None, None, None] - vb)) < 1e-15
    # corrector uses (v^n + v^{n+1})/2, whose mean is vbar/2
    assert np.max(np.abs(_min_img(qa - qb, g.L) - g.dt * vbar / 2)) < 1e-15


def test_particle_velocities_rigid_motion():
    g = mb.Grid(32, 32, 32)
    rng = np.random.default_rng(12)
    s = wl.build_particles(rng.uniform(0, 32, size=(4, 3)), 2.0, rng, g.L)
    U = rng.normal(size=(4, 3))
    W = rng.normal(size=(4, 3))
    u = np.empty_like(s.pos)
    for p in range(4):
        sl = slice(13 * p, 13 * p + 13)
        c = s.pos[13 * p] + _min_img(s.pos[sl] - s.pos[13 * p], g.L).mean(0)
        sp = _min_img(s.pos[sl] - c, g.L)
        u[sl] = U[p] + np.cross(W[p], sp)
    U2, W2 = mb.particle_velocities(g, s.pos, u, s.pid, 4)
    assert np.max(np.abs(U2 - U)) < 1e-12 and np.max(np.abs(W2 - W)) < 1e-12


def _stretched_particle_in_flow(g):
    """One particle of vertex radius 1.5h with every spring stretched by 10% (position-dependent
    internal forces), a constant external pull, in a shear mode plus a projected random flow."""
    rng = np.random.default_rng(11)
    s = wl.build_particles(np.array([5.3, 6.1, 4.7]), 1.5, rng, g.L)
    c = s.pos[0]
    q0 = np.mod(c + 1.1 * _min_img(s.pos - c, g.L), g.L)
    z = np.arange(g.nz) + 0.5
    v0 = g.zeros()
    v0[0] += 0.05 * np.sin(2 * np.pi * z / g.nz)[:, None, None]
    v0 += mb.fluid_update(mb.Grid(g.nx, g.ny, g.nz, rho=1.0, eta=0.0, dt=1.0), g.zeros(),
                          wl.random_field(g.shape, 3, scale=2e-2))
    ext = np.zeros_like(q0)
    ext[:, 1] = 2e-2
    return s, q0, v0, ext


def test_step_is_second_order_in_time():
    """The midpoint predictor/corrector with Crank-Nicolson is second order in dt: halving dt
    divides the change of the end state by 4.  Evaluating the forces or the corrector's J at q^n
    instead of q^{n+1/2}, a full predictor step, or v^{n+1} alone in the corrector each make it
    first order (ratio 2), so this pins where the step places its midpoint."""
    T = 0.32
    q, v = {}, {}
    for dt in (0.02, 0.01, 0.005):
        g = mb.Grid(12, 12, 12, dt=dt, mean_mode=0)
        s, q0, v0, ext = _stretched_particle_in_flow(g)
        q[dt], v[dt] = mb.step(g, int(round(T / dt)), q0, v0, s.pid, s.bonds, s.rest, 100.0,
                               ext=ext)
    L = g.L
    dq1 = np.linalg.norm(_min_img(q[0.02] - q[0.01], L))
    dq2 = np.linalg.norm(_min_img(q[0.01] - q[0.005], L))
    dv1 = np.linalg.norm(v[0.02] - v[0.01])
    dv2 = np.linalg.norm(v[0.01] - v[0.005])
    assert 3.6 < dq1 / dq2 < 4.4, dq1 / dq2
    assert 3.6 < dv1 / dv2 < 4.4, dv1 / dv2
    # the particle moved by much more than the time-discretisation change
    assert np.linalg.norm(_min_img(q[0.005] - q0, L)) > 1e3 * dq2


def test_step_midpoint_uniform_flow_shift():
    """A uniform flow U with U dt/2 = h carries the predictor exactly one cell, because J of a
    constant field is that constant (the weights sum to one).  The step from (q, v = U) is then
    the step from (q + h x_hat, v = 0) shifted by h x_hat in q and by U in v: the blob forces and
    S act at q^{n+1/2}, the fluid update is linear with constant fields unchanged, and the
    corrector applies J(q^{n+1/2}) to (v^n + v^{n+1})/2.  Forces or the corrector's J taken at
    q^n, or a full-step predictor, break the relation."""
    g = mb.Grid(12, 12, 12, dt=0.05, mean_mode=0)
    s, q0, v0, ext = _stretched_particle_in_flow(g)
    U = 2.0 * g.h / g.dt
    vU = g.zeros()
    vU[0] = U
    qa, va = mb.step(g, 1, q0, vU, s.pid, s.bonds, s.rest, 100.0, ext=ext)
    shift = np.array([g.h, 0.0, 0.0])
    qb, vb = mb.step(g, 1, np.mod(q0 + shift, g.L), g.zeros(), s.pid, s.bonds, s.rest, 100.0,
                     ext=ext)
    vb[0] += U
    scale = np.max(np.abs(vb - vU))
    assert scale > 1e-4
    assert np.max(np.abs(va - vb)) < 1e-10 * U
    assert np.max(np.abs(_min_img(qa - (qb + shift), g.L))) < 1e-12 * U * g.dt * 10
