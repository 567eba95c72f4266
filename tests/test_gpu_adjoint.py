"""Adjoint of the ICM step and of K-step rollouts against FP64 central finite differences.

The gradient of a scalar loss with respect to every blob coordinate and the spring stiffness
comes from the hand-written adjoint (mb_adjoint_step, mb_particle_velocity_adjoint) through
torch.autograd; it is checked along seeded random directions against central differences of
the FP64 GPU forward (step 1e-6 for positions, 1e-3 relative for the stiffness) and against
central differences of the FP64 CPU oracle.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1407_5600_gb300 as mb  # noqa: E402
from paper_1407_5600_gb300 import workloads as wl  # noqa: E402
from paper_1407_5600_gb300.autograd import rollout_particle_velocities  # noqa: E402

EPS = 1e-6


def _two_particles(n=16, a=1.6, gap=0.4, seed=11):
    rng = np.random.default_rng(seed)
    L = float(n)
    c = np.array([L / 2, L / 2 + 0.3, L / 2 - 0.2])
    sep = 2 * a + gap
    s = wl.build_particles(np.array([c - [sep / 2, 0, 0], c + [sep / 2, 0, 0]]), a, rng,
                           np.array([L, L, L]))
    s.pos = np.mod(s.pos + rng.normal(scale=0.02, size=s.pos.shape), s.L)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    return s, ext


def test_single_step_adjoint_against_finite_differences():
    s, ext = _two_particles()
    d = mb.GridDesc(16, 16, 16, precision=1, dt=0.05, mean_mode=0)
    rng = np.random.default_rng(3)
    cq = torch.tensor(rng.normal(size=s.pos.shape), device="cuda")
    cv = torch.tensor(rng.normal(size=(1, 3, 16, 16, 16)), device="cuda")
    v0 = torch.tensor(rng.normal(scale=1e-3, size=(1, 3, 16, 16, 16)), device="cuda")
    body = (1e-3, 0, 2, 1)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, 100.0, 50.0, 1.0)
        q0 = sim.blob_positions().clone()
        ext_d = torch.tensor(ext, device="cuda")

        def loss(q, v):
            sim.set_positions(q)
            sim.set_velocity_field(v)
            sim.step(1, ext_blob_force=ext_d, body_force=body)
            dq = sim.blob_positions() - q0
            dq -= torch.round(dq / 16.0) * 16.0
            return float((cq * dq).sum() + (cv * sim.velocity_field()).sum())

        gq = cq.clone()
        gv = cv.clone()
        gk = np.zeros(1)
        mb.adjoint_step(sim.ctx, q0, v0, ext_d, body, gq, gv, gk)
        dq_dir = torch.tensor(rng.normal(size=s.pos.shape), device="cuda")
        fd_q = (loss(q0 + EPS * dq_dir, v0) - loss(q0 - EPS * dq_dir, v0)) / (2 * EPS)
        # gq is dL/dq^n of L = cq.(q^{n+1} - q0) + cv.v^{n+1}; the shift by q0 adds cq.(dq)
        an_q = float((gq * dq_dir).sum())
        assert abs(an_q - fd_q) < 1e-6 * max(1.0, abs(fd_q)), (an_q, fd_q)
        dv_dir = torch.tensor(rng.normal(size=(1, 3, 16, 16, 16)), device="cuda")
        fd_v = (loss(q0, v0 + EPS * dv_dir) - loss(q0, v0 - EPS * dv_dir)) / (2 * EPS)
        an_v = float((gv * dv_dir).sum())
        assert abs(an_v - fd_v) < 1e-6 * max(1.0, abs(fd_v)), (an_v, fd_v)


def test_particle_velocity_adjoint_against_oracle_differences():
    """mb_particle_velocity_adjoint: the transpose of U0 = (1/N_p) sum J_i(q) v along random
    directions in q and v, against central differences of the oracle's interpolation and
    particle mean."""
    s, _ = _two_particles()
    d = mb.GridDesc(16, 16, 16, precision=1, dt=0.05, mean_mode=0)
    g = oracle.Grid(16, 16, 16)
    rng = np.random.default_rng(8)
    v = rng.normal(size=(3, 16, 16, 16))
    gU = rng.normal(size=(s.n_particles, 3))
    dq = rng.normal(size=s.pos.shape)
    dv = rng.normal(size=v.shape)

    def U0(q, vv):
        return oracle.particle_velocities(g, q, oracle.interp(g, q, vv), s.pid,
                                          s.n_particles)[0]

    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, 100.0)
        gq = torch.zeros(s.pos.shape, dtype=torch.float64, device="cuda")
        gv = torch.zeros((1, 3, 16, 16, 16), dtype=torch.float64, device="cuda")
        mb.particle_velocity_adjoint(sim.ctx, torch.tensor(s.pos, device="cuda"),
                                     torch.tensor(v[None], device="cuda"),
                                     torch.tensor(gU, device="cuda"), gq, gv)
        gq, gv = gq.cpu().numpy(), gv.cpu().numpy()[0]
    fd_q = np.sum(gU * (U0(s.pos + EPS * dq, v) - U0(s.pos - EPS * dq, v))) / (2 * EPS)
    fd_v = np.sum(gU * (U0(s.pos, v + dv) - U0(s.pos, v - dv))) / 2.0
    assert abs(np.sum(gq * dq) - fd_q) < 1e-6 * max(1.0, abs(fd_q))
    assert abs(np.sum(gv * dv) - fd_v) < 1e-12 * max(1.0, abs(fd_v))


def _rollout_setup(n, seed):
    s, ext = _two_particles(n=n, seed=seed)
    return s, ext


@pytest.mark.parametrize("K,chk", [(6, 2), (5, 10)])
def test_rollout_gradient_against_gpu_finite_differences(K, chk):
    s, ext = _rollout_setup(16, 5)
    d = mb.GridDesc(16, 16, 16, precision=1, dt=0.05, mean_mode=0)
    rng = np.random.default_rng(7)
    target = torch.tensor(rng.normal(scale=1e-4, size=(2, 3)), device="cuda")
    with mb.Multiblob(d) as sim:
        def L(q, k):
            U = rollout_particle_velocities(sim, q, k, s.pid, s.bonds, s.rest, K, chk,
                                            ext_blob_force=ext, k_rep=50.0, r_cut=1.0)
            return ((U - target) ** 2).sum()

        q0 = torch.tensor(s.pos, device="cuda", requires_grad=True)
        k0 = torch.tensor(100.0, dtype=torch.float64, device="cuda", requires_grad=True)
        loss = L(q0, k0)
        loss.backward()
        gq, gk = q0.grad.clone(), float(k0.grad)
        with torch.no_grad():
            dq = torch.tensor(rng.normal(size=s.pos.shape), device="cuda")
            fd_q = (float(L(q0 + EPS * dq, k0)) - float(L(q0 - EPS * dq, k0))) / (2 * EPS)
            fd_k = (float(L(q0, k0 + 0.1)) - float(L(q0, k0 - 0.1))) / 0.2
        an_q = float((gq * dq).sum())
        assert abs(an_q - fd_q) < 1e-5 * abs(fd_q) + 1e-18, (an_q, fd_q)
        assert abs(gk - fd_k) < 1e-5 * abs(fd_k) + 1e-20, (gk, fd_k)


def test_rollout_gradient_against_oracle_finite_differences():
    """The oracle's gradient: central differences of the FP64 CPU oracle rollout."""
    s, ext = _rollout_setup(16, 9)
    K = 4
    d = mb.GridDesc(16, 16, 16, precision=1, dt=0.05, mean_mode=0)
    g = oracle.Grid(16, 16, 16, dt=0.05, mean_mode=0)
    rng = np.random.default_rng(8)
    target = rng.normal(scale=1e-4, size=(2, 3))

    def oracle_loss(q):
        qK, vK = oracle.step(g, K, q, g.zeros(), s.pid, s.bonds, s.rest, 100.0, 50.0, 1.0, ext=ext)
        U, _ = oracle.particle_velocities(g, qK, oracle.interp(g, qK, vK), s.pid, 2)
        return float(((U - target) ** 2).sum())

    with mb.Multiblob(d) as sim:
        q0 = torch.tensor(s.pos, device="cuda", requires_grad=True)
        k0 = torch.tensor(100.0, dtype=torch.float64, device="cuda")
        U = rollout_particle_velocities(sim, q0, k0, s.pid, s.bonds, s.rest, K, 2,
                                        ext_blob_force=ext, k_rep=50.0, r_cut=1.0)
        ((U - torch.tensor(target, device="cuda")) ** 2).sum().backward()
        gq = q0.grad.cpu().numpy()
    for trial in range(2):
        dq = rng.normal(size=s.pos.shape)
        fd = (oracle_loss(s.pos + EPS * dq) - oracle_loss(s.pos - EPS * dq)) / (2 * EPS)
        an = float((gq * dq).sum())
        assert abs(an - fd) < 1e-5 * abs(fd) + 1e-18, (trial, an, fd)


def test_differentiable_workload_64cube_k50():
    """64^3 box, 64 particles of radius 2h, K = 50 steps, checkpoints every 10 steps."""
    spec, s = wl.dilute_random(n=64, n_particles=64, a=2.0, seed=4)
    rng = np.random.default_rng(4)
    ext = rng.normal(scale=1e-3, size=s.pos.shape)
    # targets: particle velocities of a seeded perturbed configuration
    d = mb.GridDesc(64, 64, 64, precision=1, dt=0.05, mean_mode=0)
    with mb.Multiblob(d) as sim:
        k0 = torch.tensor(100.0, dtype=torch.float64, device="cuda", requires_grad=True)
        with torch.no_grad():
            qp = torch.tensor(np.mod(s.pos + rng.normal(scale=0.1, size=s.pos.shape), s.L),
                              device="cuda")
            target = rollout_particle_velocities(sim, qp, k0.detach(), s.pid, s.bonds, s.rest, 50,
                                                 10, ext_blob_force=ext).clone()
        q0 = torch.tensor(s.pos, device="cuda", requires_grad=True)

        def L(q, k):
            U = rollout_particle_velocities(sim, q, k, s.pid, s.bonds, s.rest, 50, 10,
                                            ext_blob_force=ext)
            return ((U - target) ** 2).sum()

        loss = L(q0, k0)
        loss.backward()
        assert torch.isfinite(q0.grad).all()
        with torch.no_grad():
            dq = torch.tensor(rng.normal(size=s.pos.shape), device="cuda")
            fd = (float(L(q0 + EPS * dq, k0)) - float(L(q0 - EPS * dq, k0))) / (2 * EPS)
            # k enters through bond extensions ~1e-6 of the bond length: a relative step of
            # 1e-3 keeps the loss difference far above the forward's rounding reproducibility
            hk = 0.5     # fourth-order central difference
            fdk = (-float(L(q0, k0 + 2 * hk)) + 8 * float(L(q0, k0 + hk))
                   - 8 * float(L(q0, k0 - hk)) + float(L(q0, k0 - 2 * hk))) / (12 * hk)
        an = float((q0.grad * dq).sum())
        assert abs(an - fd) < 1e-5 * abs(fd), (an, fd)
        assert abs(float(k0.grad) - fdk) < 1e-5 * abs(fdk), (float(k0.grad), fdk)
