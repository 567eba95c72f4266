"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances are relative L2 errors: 1e-10 for the FP64 grid path and 1e-5 for the FP32 grid
(FP64 blobs) path.  Sizes span several spreading tiles and ragged blob counts; the full 128^3
dense workload is checked operator by operator and through properties of one step.
"""
import dataclasses

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


def _desc(shape, prec, **kw):
    nz, ny, nx = shape
    return mb.GridDesc(nx, ny, nz, precision=prec, **kw)


def _oracle_grid(d: mb.GridDesc):
    return oracle.Grid(d.nx, d.ny, d.nz, h=d.h, rho=d.rho, eta=d.eta, dt=d.dt,
                       mean_mode=d.mean_mode)


# ------------------------------------------------------------------------------------------
# Operators

SHAPES = [((8, 8, 8), 1.0, 300), ((16, 16, 16), 0.7, 5003), ((16, 32, 64), 1.0, 20011),
          ((4, 4, 4), 2.0, 37), ((8, 16, 128), 1.0, 7777)]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape,h,n", SHAPES)
def test_spread_parity(prec, shape, h, n):
    d = _desc(shape, prec, h=h)
    q, F, _ = wl.random_blobs(n, shape, seed=n, h=h)
    q[0] = 0.0
    q[1] = [0.5 * h, h, 1.5 * h]
    q[2] = np.array([shape[2], shape[1], shape[0]]) * h - 1e-12   # just inside the box
    q[3] = [-0.3 * h, 1e3 * h, -2.5 * h]                              # outside: wrapped
    with mb.Multiblob(d) as sim:
        f_gpu = to_np(sim.spread(q, F))[0]
    f_ref = oracle.spread(_oracle_grid(d), np.mod(q, _oracle_grid(d).L), F)
    assert rel_l2(f_gpu, f_ref) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape,h,n", SHAPES)
def test_interp_parity(prec, shape, h, n):
    d = _desc(shape, prec, h=h)
    q, _, _ = wl.random_blobs(n, shape, seed=n + 1, h=h)
    v = wl.random_field(shape, seed=n + 2)
    with mb.Multiblob(d) as sim:
        u_gpu = to_np(sim.interp(q, v[None].astype(d.grid_dtype)))
    u_ref = oracle.interp(_oracle_grid(d), q, v.astype(d.grid_dtype).astype(np.float64))
    assert rel_l2(u_gpu, u_ref) < TOL[prec]


def test_spread_interp_adjoint_on_gpu():
    shape = (16, 16, 32)
    d = _desc(shape, 1, h=0.9)
    q, F, _ = wl.random_blobs(3001, shape, seed=3, h=d.h)
    v = wl.random_field(shape, seed=4)
    with mb.Multiblob(d) as sim:
        f = to_np(sim.spread(q, F))[0]
        u = to_np(sim.interp(q, v[None]))
    lhs = d.h ** 3 * np.sum(f * v)
    rhs = np.sum(F * u)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def _projected_field(shape, seed, scale=1.0):
    nz, ny, nx = shape
    g = oracle.Grid(nx, ny, nz, rho=1.0, eta=0.0, dt=1.0)
    return oracle.fluid_update(g, g.zeros(), wl.random_field(shape, seed, scale))


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("shape,h,mean_mode,body", [
    ((16, 16, 16), 1.0, 0, None), ((8, 16, 32), 0.5, 1, None),
    ((32, 32, 32), 1.0, 0, (1e-2, 0, 2, 1)), ((16, 8, 64), 1.3, 1, (0.3, 1, 0, 3)),
    ((4, 8, 4), 2.0, 0, (1.0, 2, 1, 1)),
    ((8, 16, 128), 0.8, 0, (1e-2, 1, 0, 2)), ((4, 64, 128), 1.0, 1, (0.5, 0, 1, 1)),
])
def test_fluid_update_parity(prec, shape, h, mean_mode, body):
    d = _desc(shape, prec, h=h, rho=1.3, eta=0.7, dt=0.05, mean_mode=mean_mode)
    v = _projected_field(shape, 11).astype(d.grid_dtype).astype(np.float64)
    f = wl.random_field(shape, 12, scale=0.5).astype(d.grid_dtype).astype(np.float64)
    with mb.Multiblob(d) as sim:
        vn = to_np(sim.fluid_update(v[None].astype(d.grid_dtype), f[None].astype(d.grid_dtype),
                                    body_force=body))[0]
    ref = oracle.fluid_update(_oracle_grid(d), v, f, body=body)
    assert rel_l2(vn, ref) < TOL[prec]


def test_fp64_fluid_update_on_tiny_fields():
    """FP64 grids transform in double-float arithmetic; values below 2^-74 in magnitude take a
    float-only path and keep 24 bits (documented in include/mb.h).  A field scaled into that
    range matches the oracle to float precision, and the same field at unit scale to 1e-10."""
    shape = (16, 16, 16)
    d = _desc(shape, 1, rho=1.3, eta=0.7, dt=0.05, mean_mode=0)
    v = _projected_field(shape, 31)
    f = wl.random_field(shape, 32, scale=0.5)
    g = _oracle_grid(d)
    for scale, tol in ((1.0, TOL[1]), (2.0 ** -90, 1e-6)):
        with mb.Multiblob(d) as sim:
            vn = to_np(sim.fluid_update((scale * v)[None], (scale * f)[None]))[0]
        ref = oracle.fluid_update(g, scale * v, scale * f)
        err = rel_l2(vn, ref)
        assert err < tol, (scale, err)
        if scale < 1.0:
            assert err > 1e-12      # the float-only path is in use: not FP64 accuracy


# ------------------------------------------------------------------------------------------
# Full step

def _run_gpu(d, susp_list, nsteps, ext_list=None, body=None, v0=None):
    with mb.Multiblob(d) as sim:
        for b, s in enumerate(susp_list):
            sim.set_particles(b, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        if v0 is not None:
            sim.set_velocity_field(v0.astype(d.grid_dtype))
        ext = None
        if ext_list is not None:
            ext = np.concatenate(ext_list, axis=0)
        sim.step(nsteps, ext_blob_force=ext, body_force=body)
        q = to_np(sim.blob_positions())
        v = to_np(sim.velocity_field()).astype(np.float64)
        u = to_np(sim.blob_velocities())
        U, W = sim.particle_velocities()
        return q, v, u, to_np(U), to_np(W)


@pytest.mark.parametrize("prec", [1, 0])
def test_step_parity_single_particle(prec):
    spec, s = wl.single_particle(n=32, a=1.0, seed=1)
    d = mb.GridDesc(32, 32, 32, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt,
                    precision=prec, mean_mode=spec.mean_mode)
    nsteps = 20
    q, v, u, U, W = _run_gpu(d, [s], nsteps, ext_list=[s.ext])
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               ext=s.ext)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]
    u_ref = oracle.interp(g, q_ref, v_ref)
    assert rel_l2(u, u_ref) < TOL[prec]
    U_ref, W_ref = oracle.particle_velocities(g, q_ref, u_ref, s.pid, 1)
    assert rel_l2(U, U_ref) < TOL[prec]
    assert np.max(np.abs(W - W_ref)) < TOL[prec] * max(np.max(np.abs(W_ref)), np.max(np.abs(U_ref)))


def _dense_small(seed=5, n=32, a=2.2, phi=0.40):
    spec, s = wl.dense_suspension(n=n, a=a, phi=phi, seed=seed, mc_sweeps=3)
    return spec, s


@pytest.mark.parametrize("prec", [1, 0])
def test_step_parity_dense_with_repulsion(prec):
    spec, s = _dense_small()
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, h=spec.h, rho=spec.rho, eta=spec.eta,
                    dt=spec.dt, precision=prec, mean_mode=spec.mean_mode)
    rng = np.random.default_rng(9)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    # start slightly off the rest shape so springs and repulsion both act
    s.pos = np.mod(s.pos + rng.normal(scale=0.05, size=s.pos.shape), s.L)
    nsteps = 3
    v0 = _projected_field((spec.nz, spec.ny, spec.nx), 21, scale=1e-3)
    q, v, u, U, W = _run_gpu(d, [s], nsteps, ext_list=[ext], body=s.body, v0=v0[None])
    g = _oracle_grid(d)
    v0r = v0.astype(d.grid_dtype).astype(np.float64)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, v0r, s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, ext=ext, body=s.body)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[prec])
    assert rel_l2(v[0], v_ref) < TOL[prec]


@pytest.mark.parametrize("prec", [1, 0])
def test_forces_parity_after_step(prec):
    """FP64 mode: the oracle's own operation order, so the forces agree to the last bit in
    practice (1e-12 bound); FP32-grid mode: FP64 differences, FP32 magnitudes."""
    spec, s = _dense_small(seed=6)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, precision=prec, dt=spec.dt)
    rng = np.random.default_rng(2)
    s.pos = np.mod(s.pos + rng.normal(scale=0.1, size=s.pos.shape), s.L)
    ext = rng.normal(size=s.pos.shape)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(1, ext_blob_force=ext)
        F, qh = (to_np(x) for x in sim.last_forces())
    g = _oracle_grid(d)
    F_ref = ext + oracle.bond_forces(g, qh, s.bonds, s.rest, s.k_spring) \
        + oracle.pair_forces(g, qh, s.pid, s.k_rep, s.r_cut)
    assert np.max(np.abs(F - F_ref)) < (1e-12 if prec == 1 else TOL[0]) * np.max(np.abs(F_ref))
    # repulsion was active
    assert np.max(np.abs(oracle.pair_forces(g, qh, s.pid, s.k_rep, s.r_cut))) > 0


def test_fp32_springs_with_and_without_a_common_bond_pattern():
    """FP32 grid: the icosahedra in particle order share one bond pattern (stored once); the same
    suspension with its blobs shuffled has none (per-blob bond lists).  Both give the oracle's
    forces and trajectory."""
    spec, s = _dense_small(seed=7)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, h=spec.h, rho=spec.rho, eta=spec.eta,
                    dt=spec.dt, precision=0, mean_mode=spec.mean_mode)
    rng = np.random.default_rng(13)
    s.pos = np.mod(s.pos + rng.normal(scale=0.08, size=s.pos.shape), s.L)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    perm = rng.permutation(s.n_blobs)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(s.n_blobs)
    shuffled = dataclasses.replace(s, pos=s.pos[perm].copy(), pid=s.pid[perm].copy(),
                                   bonds=inv[s.bonds].astype(s.bonds.dtype))
    g = _oracle_grid(d)
    nsteps = 3
    for susp, e, back in ((s, ext, np.arange(s.n_blobs)), (shuffled, ext[perm], inv)):
        with mb.Multiblob(d) as sim:
            sim.set_particles(0, susp.pos, susp.pid, susp.bonds, susp.rest, susp.k_spring,
                              susp.k_rep, susp.r_cut)
            sim.step(1, ext_blob_force=e)
            F, qh = (to_np(x)[back] for x in sim.last_forces())
            sim.step(nsteps - 1, ext_blob_force=e, body_force=s.body)
            q = to_np(sim.blob_positions())[back]
        F_ref = ext + oracle.bond_forces(g, qh, s.bonds, s.rest, s.k_spring) \
            + oracle.pair_forces(g, qh, s.pid, s.k_rep, s.r_cut)
        assert np.max(np.abs(F - F_ref)) < TOL[0] * np.max(np.abs(F_ref))
        q_ref1, v_ref1 = oracle.step(g, 1, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                                     s.k_rep, s.r_cut, ext=ext)
        q_ref, _ = oracle.step(g, nsteps - 1, q_ref1, v_ref1, s.pid, s.bonds, s.rest,
                               s.k_spring, s.k_rep, s.r_cut, ext=ext, body=s.body)
        assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[0])


def test_fp64_springs_pattern_matches_per_blob_sums_bitwise():
    """FP64 grid: with a bond pattern shared by all particles the springs are evaluated once per
    bond and summed in each blob's adjacency order, which gives the bits of the per-blob
    evaluation (the shuffled copy of the suspension has no pattern and takes that path).
    No repulsion, so the forces are the external forces plus the springs alone."""
    spec, s = _dense_small(seed=8)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, h=spec.h, rho=spec.rho, eta=spec.eta,
                    dt=spec.dt, precision=1, mean_mode=spec.mean_mode)
    rng = np.random.default_rng(29)
    s.pos = np.mod(s.pos + rng.normal(scale=0.08, size=s.pos.shape), s.L)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    perm = rng.permutation(s.n_blobs)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(s.n_blobs)
    shuffled = dataclasses.replace(s, pos=s.pos[perm].copy(), pid=s.pid[perm].copy(),
                                   bonds=inv[s.bonds].astype(s.bonds.dtype))
    out = []
    for susp, e, back in ((s, ext, np.arange(s.n_blobs)), (shuffled, ext[perm], inv)):
        with mb.Multiblob(d) as sim:
            sim.set_particles(0, susp.pos, susp.pid, susp.bonds, susp.rest, susp.k_spring)
            sim.step(1, ext_blob_force=e)
            F, qh = (to_np(x)[back] for x in sim.last_forces())
            sim.step(2, ext_blob_force=e)
            q = to_np(sim.blob_positions())[back]
        out.append((F, qh, q))
    assert np.array_equal(out[0][1], out[1][1])           # same midpoints
    assert np.array_equal(out[0][0], out[1][0])           # same forces, bit for bit
    g = _oracle_grid(d)
    F_ref = ext + oracle.bond_forces(g, out[0][1], s.bonds, s.rest, s.k_spring)
    assert np.max(np.abs(out[0][0] - F_ref)) < 1e-12 * np.max(np.abs(F_ref))
    q_ref, _ = oracle.step(g, 3, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring, ext=ext)
    assert_positions(out[0][2], q_ref, s.pos, g.L, 3, TOL[1])


def test_fp32_step_with_clustered_blobs():
    """FP32 grid: 40 icosahedra overlapping inside a 3h cube (520 blobs in a few bin cells, no
    repulsion) with random external forces.  The spreading's fixed-point scale must stay a
    bound on every node of a tile that holds them all; the step matches the oracle."""
    rng = np.random.default_rng(23)
    n = 16
    L = np.array([float(n)] * 3)
    centres = 6.5 + rng.uniform(0.0, 3.0, size=(40, 3))
    s = wl.build_particles(centres, 1.0, rng, L)
    ext = rng.normal(scale=1e-2, size=s.pos.shape)
    d = mb.GridDesc(n, n, n, precision=0, dt=0.05, mean_mode=0)
    nsteps = 2
    q, v, u, U, W = _run_gpu(d, [s], nsteps, ext_list=[ext])
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               ext=ext)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[0])
    assert rel_l2(v[0], v_ref) < TOL[0]


@pytest.mark.parametrize("prec", [1, 0])
def test_batched_boxes_match_independent_runs(prec):
    B = 4
    boxes = []
    for b in range(B):
        spec, s = wl.gap_sweep_box(b, n_boxes=B, n=16, a=1.6)
        boxes.append(s)
    d = mb.GridDesc(16, 16, 16, batch=B, precision=prec, dt=0.05, mean_mode=0)
    nsteps = 8
    q, v, u, U, W = _run_gpu(d, boxes, nsteps, ext_list=[s.ext for s in boxes])
    g = _oracle_grid(d)
    off = 0
    for b, s in enumerate(boxes):
        q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest,
                                   s.k_spring, ext=s.ext)
        qb = q[off:off + s.n_blobs]
        assert_positions(qb, q_ref, s.pos, g.L, nsteps, TOL[prec])
        assert rel_l2(v[b], v_ref) < TOL[prec]
        off += s.n_blobs


# ------------------------------------------------------------------------------------------
# Edge cases

def test_empty_box_and_single_blob():
    d = mb.GridDesc(8, 8, 8, batch=2, precision=1)
    single = wl.Suspension(pos=np.array([[7.999999999, 0.0, 3.5]]),
                           pid=np.zeros(1, dtype=np.int32),
                           bonds=np.zeros((0, 2), dtype=np.int32), rest=np.zeros(0),
                           n_particles=1, a=0.0, L=np.array([8.0, 8, 8]))
    empty = wl.Suspension(pos=np.zeros((0, 3)), pid=np.zeros(0, dtype=np.int32),
                          bonds=np.zeros((0, 2), dtype=np.int32), rest=np.zeros(0),
                          n_particles=0, a=0.0, L=np.array([8.0, 8, 8]))
    ext = np.array([[0.1, -0.2, 0.05]])
    q, v, u, U, W = _run_gpu(d, [single, empty], 4, ext_list=[ext, np.zeros((0, 3))])
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, 4, single.pos, g.zeros(), single.pid, single.bonds,
                               single.rest, 0.0, ext=ext)
    assert_positions(q, q_ref, single.pos, g.L, 4, 1e-10)
    assert rel_l2(v[0], v_ref) < 1e-10
    assert np.all(v[1] == 0.0)


def test_invalid_calls_leave_state_and_report():
    d = mb.GridDesc(8, 8, 8, precision=1)
    with mb.Multiblob(d) as sim:
        with pytest.raises(mb.MBError) as ei:
            sim.step(1)
        assert ei.value.status == 4
        with pytest.raises(mb.MBError) as ei:
            sim.set_particles(0, np.zeros((2, 3)), np.zeros(2, dtype=np.int32),
                              np.array([[0, 5]], dtype=np.int32), np.ones(1), 1.0)
        assert ei.value.status == 1
        with pytest.raises(mb.MBError) as ei:
            sim.set_particles(1, np.zeros((2, 3)), np.zeros(2, dtype=np.int32),
                              np.zeros((0, 2), dtype=np.int32), np.zeros(0), 1.0)
        assert ei.value.status == 1
        with pytest.raises(mb.MBError):
            sim.step(1, body_force=(1.0, 3, 0, 1))


def test_host_buffers_through_the_abi():
    """The same call with host (numpy) arrays stages through device buffers."""
    shape = (16, 16, 16)
    d = _desc(shape, 1)
    q, F, _ = wl.random_blobs(999, shape, seed=77)
    ctx = mb.create_grid(d)
    try:
        out = np.zeros((1, 3) + shape)
        mb.spread(ctx, q, F, out)
        u = np.zeros((999, 3))
        mb.interp(ctx, q, out, u)
    finally:
        mb.destroy(ctx)
    g = _oracle_grid(d)
    f_ref = oracle.spread(g, q, F)
    assert rel_l2(out[0], f_ref) < 1e-12
    assert rel_l2(u, oracle.interp(g, q, f_ref)) < 1e-12


@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
def test_fp32_step_external_forces_from_any_memory(kind):
    """FP32-grid steps with external forces given in pageable host, page-locked host (read by
    the kernel directly) or device memory, and blob velocities read back to the same kind of
    memory: all three agree with the oracle."""
    spec, s = _dense_small(seed=19)
    rng = np.random.default_rng(19)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, precision=0, dt=spec.dt, mean_mode=spec.mean_mode)
    if kind == "pageable":
        e_in, u_out = ext.copy(), np.zeros_like(ext)
    elif kind == "pinned":
        e_in = torch.tensor(ext).pin_memory().numpy()
        u_out = torch.zeros(ext.shape, dtype=torch.float64).pin_memory().numpy()
    else:
        e_in = torch.tensor(ext, device="cuda")
        u_out = torch.zeros(ext.shape, dtype=torch.float64, device="cuda")
    nsteps = 3
    ctx = mb.create_grid(d)
    try:
        mb.set_particles(ctx, 0, np.ascontiguousarray(s.pos, dtype=np.float64),
                         np.ascontiguousarray(s.pid, dtype=np.int32),
                         np.ascontiguousarray(s.bonds, dtype=np.int32),
                         np.ascontiguousarray(s.rest, dtype=np.float64), s.k_spring, s.k_rep,
                         s.r_cut)
        for _ in range(nsteps):
            mb.step(ctx, 1, e_in, s.body)
        mb.get_velocities(ctx, blob_vel=u_out)
        q = np.zeros_like(ext)
        mb.get_velocities(ctx, blob_pos=q)
    finally:
        mb.destroy(ctx)
    u = to_np(u_out) if kind == "device" else u_out
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, ext=ext, body=s.body)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[0])
    assert rel_l2(u, oracle.interp(g, q_ref, v_ref)) < TOL[0]


# ------------------------------------------------------------------------------------------
# Full-size dense workload (128^3, 18,808 particles, 244,504 blobs): operators against the
# oracle element by element, and one step in the benchmark's configuration through properties.

@pytest.fixture(scope="module")
def dense128():
    return wl.dense_suspension()


def test_full_size_spread_and_interp(dense128):
    spec, s = dense128
    d = mb.GridDesc(128, 128, 128, precision=0)
    rng = np.random.default_rng(1)
    F = rng.normal(size=s.pos.shape)
    with mb.Multiblob(d) as sim:
        f = to_np(sim.spread(s.pos, F))[0]
        v = _projected_field((128, 128, 128), 3)
        u = to_np(sim.interp(s.pos, v[None].astype(np.float32)))
    g = _oracle_grid(d)
    assert rel_l2(f, oracle.spread(g, s.pos, F)) < 1e-5
    assert rel_l2(u, oracle.interp(g, s.pos, v.astype(np.float32).astype(np.float64))) < 1e-5


def test_full_size_fluid_update():
    d = mb.GridDesc(128, 128, 128, precision=0, mean_mode=0)
    v = _projected_field((128, 128, 128), 5).astype(np.float32)
    f = wl.random_field((128, 128, 128), 6, scale=0.1).astype(np.float32)
    body = (1e-4, 0, 2, 1)
    with mb.Multiblob(d) as sim:
        vn = to_np(sim.fluid_update(v[None], f[None], body_force=body))[0]
    ref = oracle.fluid_update(_oracle_grid(d), v.astype(np.float64), f.astype(np.float64), body)
    assert rel_l2(vn, ref) < 1e-5


def test_full_size_step_properties(dense128):
    spec, s = dense128
    d = mb.GridDesc(128, 128, 128, precision=0, mean_mode=0, dt=spec.dt)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(2, body_force=s.body)
        F, qh = (to_np(x) for x in sim.last_forces())
        v = to_np(sim.velocity_field())[0].astype(np.float64)
        q = to_np(sim.blob_positions())
    g = _oracle_grid(d)
    # divergence-free fluid (FP32 grid)
    div = ((np.roll(v[0], -1, 2) - v[0]) + (np.roll(v[1], -1, 1) - v[1])
           + (np.roll(v[2], -1, 0) - v[2]))
    assert np.max(np.abs(div)) < 1e-5 * np.max(np.abs(v))
    # mean momentum: internal forces cancel and the body force has zero mean
    assert np.max(np.abs(v.mean((1, 2, 3)))) < 1e-5 * np.max(np.abs(v))
    # forces at the midpoint positions, on a sample of blobs, against the brute-force oracle
    idx = np.random.default_rng(0).choice(len(qh), 200, replace=False)
    Fb = oracle.bond_forces(g, qh, s.bonds, s.rest, s.k_spring)[idx]
    Fp = oracle.pair_forces_subset(g, qh, s.pid, s.k_rep, s.r_cut, idx)
    # FP32-grid mode evaluates the force magnitudes in FP32 after the FP64 differences
    assert np.max(np.abs(F[idx] - Fb - Fp)) < TOL[0] * np.max(np.abs(Fb + Fp))
    # the stiff particles stay rigid and every blob moved by a finite amount
    r = np.linalg.norm(min_image(q[s.bonds[:, 0]] - q[s.bonds[:, 1]], g.L), axis=1)
    assert np.all(np.isfinite(q)) and np.max(np.abs(r - s.rest) / s.rest) < 1e-2


def test_full_size_bench_steps_match_oracle(dense128):
    """The benchmarked workload itself, element by element: 128^3 FP32 grid, 244,504 blobs,
    repulsion and body force, run as the benchmark runs it (first step direct with the spreading
    tile autotuned after it, then graph replays of both velocity-buffer parities with the fused
    corrector/predictor interpolation).  Positions, the fluid velocity, the blob velocities and
    the particle velocities after three steps against three FP64 oracle steps."""
    spec, s = dense128
    assert s.n_blobs == 244504
    nsteps = 3
    d = mb.GridDesc(128, 128, 128, precision=0, mean_mode=0, dt=spec.dt)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(nsteps, body_force=s.body)
        q = to_np(sim.blob_positions())
        v = to_np(sim.velocity_field())[0].astype(np.float64)
        u = to_np(sim.blob_velocities())
        U, _ = (to_np(x) for x in sim.particle_velocities())
        tile, _ = mb.get_tuning(sim.ctx)
    assert tile in [(32, 8, 8), (16, 8, 8), (32, 16, 8), (16, 16, 8), (64, 8, 8)]
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, body=s.body)
    u_ref = oracle.interp(g, q_ref, v_ref)
    U_ref, _ = oracle.particle_velocities(g, q_ref, u_ref, s.pid, s.n_particles)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[0])
    assert rel_l2(v, v_ref) < TOL[0]
    assert rel_l2(u, u_ref) < TOL[0]
    assert rel_l2(U, U_ref) < TOL[0]


def test_single_step_calls_with_changing_external_forces():
    """FP32 steps called one at a time with new external forces every step, from page-locked
    host memory (converted inside the step graph, beside the binning), from pageable host
    memory, from device memory, and from a multi-step call, against oracle steps with the
    same forces."""
    spec, s = _dense_small(seed=21)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, precision=0, dt=spec.dt, mean_mode=0)
    g = _oracle_grid(d)
    rng = np.random.default_rng(22)
    forces = [rng.normal(scale=1e-3, size=s.pos.shape) for _ in range(7)]
    pinned = [torch.empty(s.pos.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        for k in range(5):                       # same page-locked buffer, then the other one
            buf = pinned[0] if k < 3 else pinned[1]
            buf.copy_(torch.from_numpy(forces[k]))
            mb.step(sim.ctx, 1, buf.numpy(), s.body)
        mb.step(sim.ctx, 1, np.ascontiguousarray(forces[5]), s.body)      # pageable
        mb.step(sim.ctx, 1, torch.from_numpy(forces[6]).cuda(), s.body)   # device
        mb.step(sim.ctx, 2, torch.from_numpy(forces[6]).cuda(), s.body)   # two steps, one call
        q = to_np(sim.blob_positions())
        v = to_np(sim.velocity_field())[0].astype(np.float64)
    q_ref, v_ref = s.pos, g.zeros()
    for k in list(range(7)) + [6, 6]:
        q_ref, v_ref = oracle.step(g, 1, q_ref, v_ref, s.pid, s.bonds, s.rest, s.k_spring,
                                   s.k_rep, s.r_cut, ext=forces[k], body=s.body)
    assert_positions(q, q_ref, s.pos, g.L, 9, TOL[0])
    assert rel_l2(v, v_ref) < TOL[0]


def test_graph_replay_matches_direct_launches(monkeypatch):
    """Steps replayed from the captured CUDA graph equal directly launched steps."""
    spec, s = _dense_small(seed=7)
    out = []
    for no_graph in ("1", "0"):
        monkeypatch.setenv("MB_NO_GRAPH", no_graph)
        d = mb.GridDesc(spec.nx, spec.ny, spec.nz, precision=0, dt=spec.dt,
                        mean_mode=spec.mean_mode)
        with mb.Multiblob(d) as sim:
            sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
            sim.step(3, body_force=s.body)
            sim.step(1, body_force=s.body)
            sim.step(4, body_force=s.body)
            out.append((to_np(sim.blob_positions()), to_np(sim.velocity_field())))
    # FP32 shared-memory atomics add in a run-dependent order: the two runs agree to the
    # FP32-grid tolerance, not bitwise
    L = np.array([spec.nx, spec.ny, spec.nz], dtype=float)
    assert_positions(out[0][0], out[1][0], s.pos, L, 8, TOL[0])
    assert rel_l2(out[0][1], out[1][1]) < TOL[0]


def test_fast_translation_in_uniform_flow():
    """FP32-grid steps in a uniform flow that carries every blob about two mesh widths (one bin
    cell) per step, so that blobs change bin cells and spreading tiles every step."""
    spec, s = _dense_small(seed=13)
    shape = (spec.nz, spec.ny, spec.nx)
    v0 = np.zeros((3,) + shape)
    # uniform flow of (2, 1.25, -0.9) mesh widths per step; the workload's own time step keeps
    # the springs and the repulsion stable
    v0[0], v0[1], v0[2] = np.array([2.0, 1.25, -0.9]) * spec.h / spec.dt
    nsteps = 6
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, precision=0, dt=spec.dt, mean_mode=0)
    q, v, *_ = _run_gpu(d, [s], nsteps, body=s.body, v0=v0[None])
    g = _oracle_grid(d)
    q_ref, v_ref = oracle.step(g, nsteps, s.pos, v0, s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, body=s.body)
    assert_positions(q, q_ref, s.pos, g.L, nsteps, TOL[0])
    assert rel_l2(v[0], v_ref) < TOL[0]


@pytest.mark.parametrize("fuse", ["1", "0"])
def test_state_set_between_fp32_steps(monkeypatch, fuse):
    """FP32-grid steps whose predictor is computed by the previous step's corrector pass: a
    velocity field or positions set between steps must reach the next predictor.  Checked
    against the oracle with the same interruptions, with and without the fused pass."""
    monkeypatch.setenv("MB_NO_FUSE_INTERP", "0" if fuse == "1" else "1")
    spec, s = _dense_small(seed=17)
    shape = (spec.nz, spec.ny, spec.nx)
    d = mb.GridDesc(spec.nx, spec.ny, spec.nz, precision=0, dt=spec.dt, mean_mode=spec.mean_mode)
    g = _oracle_grid(d)
    v_mid = _projected_field(shape, 23, scale=1e-3).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(17)
    kick = rng.normal(scale=0.02, size=s.pos.shape)
    q_ref, _ = oracle.step(g, 3, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                           s.k_rep, s.r_cut, body=s.body)
    q_ref5, v_ref5 = oracle.step(g, 2, q_ref, v_mid, s.pid, s.bonds, s.rest, s.k_spring,
                                 s.k_rep, s.r_cut, body=s.body)
    q_set = np.mod(q_ref5 + kick, s.L)          # positions set from outside (oracle-derived)
    q_ref, v_ref = oracle.step(g, 2, q_set, v_ref5, s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, body=s.body)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        sim.step(3, body_force=s.body)
        sim.set_velocity_field(v_mid[None].astype(np.float32))
        sim.step(2, body_force=s.body)
        q5 = to_np(sim.blob_positions())
        sim.set_positions(q_set)
        sim.step(2, body_force=s.body)
        q = to_np(sim.blob_positions())
        v = to_np(sim.velocity_field()).astype(np.float64)
    assert_positions(q5, q_ref5, s.pos, g.L, 5, TOL[0])
    assert_positions(q, q_ref, q_set, g.L, 2, TOL[0])
    assert rel_l2(v[0], v_ref) < TOL[0]


def test_deterministic_fp64_runs_are_bitwise_identical():
    """deterministic = 1 with FP64: two runs of the dense case give the same bits, and match the
    oracle."""
    spec, s = _dense_small(seed=12)
    rng = np.random.default_rng(12)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    outs = []
    for _ in range(2):
        d = mb.GridDesc(spec.nx, spec.ny, spec.nz, precision=1, deterministic=1, dt=spec.dt,
                        mean_mode=spec.mean_mode)
        q, v, u, U, W = _run_gpu(d, [s], 4, ext_list=[ext], body=s.body)
        outs.append((q, v))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    g = _oracle_grid(mb.GridDesc(spec.nx, spec.ny, spec.nz, dt=spec.dt, mean_mode=spec.mean_mode))
    q_ref, v_ref = oracle.step(g, 4, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                               s.k_rep, s.r_cut, ext=ext, body=s.body)
    assert_positions(outs[0][0], q_ref, s.pos, g.L, 4, TOL[1])
    assert rel_l2(outs[0][1][0], v_ref) < TOL[1]


def test_single_particle_full_run_fp64_deterministic():
    """The single-particle Stokeslet run at full length (32^3, 200 steps, FP64, deterministic):
    the whole trajectory equals the oracle's (1e-10), and the drift approaches the
    Hasimoto-corrected Stokes drift of Table rad's radius from below (the t^-1/2 approach of a
    suddenly forced sphere is still under way at t = 10)."""
    import json
    import os
    spec, s = wl.single_particle(n=32, a=1.0, seed=1)
    d = mb.GridDesc(32, 32, 32, h=spec.h, rho=spec.rho, eta=spec.eta, dt=spec.dt,
                    precision=1, deterministic=1, mean_mode=spec.mean_mode)
    Us = []
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring)
        for _ in range(4):
            sim.step(50, ext_blob_force=s.ext)
            Us.append(to_np(sim.particle_velocities()[0])[0, 0])
        q = to_np(sim.blob_positions())
    g = _oracle_grid(d)
    q_ref, _ = oracle.step(g, 200, s.pos, g.zeros(), s.pid, s.bonds, s.rest, s.k_spring,
                           ext=s.ext)
    assert_positions(q, q_ref, s.pos, g.L, 200, TOL[1])
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table_rad.json")))
    RH = dict((r[0], r[1]) for r in gold["rows"])[1.0]
    U_inf = 1e-3 * (1.0 - 2.84 * RH / 32.0) / (6 * np.pi * spec.eta * RH)
    assert np.all(np.diff(Us) > 0)
    assert 0.6 * U_inf < Us[-1] < 1.05 * U_inf, (Us, U_inf)
