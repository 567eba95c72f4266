"""The viscosity protocol of Sec. 10 on the GPU path (Stokes limit, FP32 grid): a suspension
driven by the body force f0 sin(2 pi z / L) x_hat relaxes, the x-velocity profile is averaged,
and eta_eff = f0 / (lambda v_hat) with the discrete wavenumber lambda = (4/h^2) sin^2(pi h / L)
(the estimator that returns eta exactly for the pure fluid, pinned in the oracle tests).

- Pure fluid: eta_eff = eta.
- A dilute suspension (geometric phi = 0.05, a = 2.2h): the relative viscosity rises by
  Einstein's 2.5 phi to first order, with phi counted at an effective radius between the
  particles' vertex radius and their hydrodynamic radius (Table rad); the second-order
  (Batchelor) term adds a few percent.  The check is a band, not a fit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected on CPU hosts too
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1407_5600_gb300 as mb  # noqa: E402
from paper_1407_5600_gb300 import workloads as wl  # noqa: E402


def _eta_eff(sim, n, h, f0, steps_relax, steps_avg):
    sim.step(steps_relax, body_force=(f0, 0, 2, 1))
    z = (np.arange(n) + 0.5) * h
    mode = np.sin(2 * np.pi * z / (n * h))
    amp = []
    for _ in range(steps_avg):
        sim.step(1, body_force=(f0, 0, 2, 1))
        vx = sim.velocity_field()[0, 0].double().mean(dim=(1, 2)).cpu().numpy()
        amp.append(2.0 / n * np.sum(vx * mode))
    lam = 4.0 / h ** 2 * np.sin(np.pi * h / (n * h)) ** 2
    return f0 / (lam * np.mean(amp))


def test_viscosity_protocol_pure_fluid_and_dilute_suspension():
    n, f0, eta = 64, 1e-4, 1.0
    empty = wl.Suspension(pos=np.zeros((0, 3)), pid=np.zeros(0, dtype=np.int32),
                          bonds=np.zeros((0, 2), dtype=np.int32), rest=np.zeros(0),
                          n_particles=0, a=0.0, L=np.array([64.0] * 3))
    d = mb.GridDesc(n, n, n, eta=eta, dt=0.05, precision=0, mean_mode=1, integrator=1)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, empty.pos, empty.pid, empty.bonds, empty.rest, 0.0)
        eta0 = _eta_eff(sim, n, 1.0, f0, 1, 3)
    assert abs(eta0 / eta - 1.0) < 1e-5
    spec, s = wl.dense_suspension(n=n, a=2.2, phi=0.05, seed=11, mc_sweeps=2)
    with mb.Multiblob(d) as sim:
        sim.set_particles(0, s.pos, s.pid, s.bonds, s.rest, s.k_spring, s.k_rep, s.r_cut)
        eta_s = _eta_eff(sim, n, 1.0, f0, 400, 100)
    phi_a = s.n_particles * 4.0 / 3.0 * np.pi * 2.2 ** 3 / n ** 3
    phi_h = phi_a * (2.59 / 2.2) ** 3          # R_H at d = 2.31h, between Table rad's rows
    rise = eta_s / eta - 1.0
    print(f"viscosity protocol: pure fluid eta {eta0:.6f}; phi_a {phi_a:.4f} phi_h {phi_h:.4f} "
          f"relative viscosity {eta_s / eta:.4f}")
    assert 2.5 * phi_a * 0.9 < rise < (2.5 * phi_h + 6.2 * phi_h ** 2) * 1.25, (rise, phi_a, phi_h)
