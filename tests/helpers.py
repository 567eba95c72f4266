"""Shared test helpers (comparison metrics only; no method arithmetic)."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def min_image(d, L):
    return d - L * np.round(d / L)


def to_np(x):
    return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)


# Tolerances (relative L2 against the FP64 oracle) for the two grid precisions.
TOL = {0: 1e-5, 1: 1e-10}


def position_error(q, q_ref, q0, L, nsteps):
    """(|d|, |ref|, floor) for the displacement error d = q - q_ref (minimum image) against the
    reference displacement ref = q_ref - q0, and the rounding floor of the positions: each step
    rounds a coordinate of magnitude <= L once, in FP64 in the oracle and in FP64 or split
    float pairs (finer than FP64 at these box sizes) on the GPU, so a few ulps of L per step
    are representation error, not method error.  The floor does not depend on the tolerance."""
    L = np.asarray(L, dtype=np.float64)
    d = min_image(np.asarray(q) - q_ref, L)
    ref = min_image(np.asarray(q_ref) - q0, L)
    floor = 4.0 * max(nsteps, 1) * np.finfo(np.float64).eps * np.max(L) * np.sqrt(d.size)
    return np.linalg.norm(d), np.linalg.norm(ref), floor


def assert_positions(q, q_ref, q0, L, nsteps, tol):
    """Assert |q - q_ref| <= tol |q_ref - q0| + floor (relative L2 on the displacement, plus the
    FP64 rounding floor of position_error)."""
    err, ref, floor = position_error(q, q_ref, q0, L, nsteps)
    assert err <= tol * ref + floor, (
        f"position error {err:.3e} > {tol:.1e} x |displacement| {ref:.3e} + floor {floor:.2e}"
        f" (relative {err / max(ref, 1e-300):.3e})")


# Viscosity protocol (Sec. 10): a body force f0 sin(2 pi z / L) x_hat drives a shear flow whose
# amplitude A = (2/n) sum_k <v_x>_{xy}(k) sin(2 pi (k + 1/2) / n) gives the viscosity.  In steady
# state eta = f0 / (lambda A), lambda = (4/h^2) sin^2(pi h / L) the discrete wavenumber squared.
# From rest the Crank-Nicolson step advances this mode as A_{m+1} = (a A_m + f0) / b,
# a = rho/dt - eta lambda/2, b = rho/dt + eta lambda/2, so after n steps
# A_n = f0 / (eta lambda) (1 - (a/b)^n): solving that for eta gives the viscosity of a run that
# has not reached steady state yet, and eta exactly for the pure fluid.

def shear_amplitude(vx, n):
    """A of a v_x field [nz][ny][nx] (z the wave direction)."""
    prof = np.asarray(vx, dtype=np.float64).mean(axis=(1, 2))
    return 2.0 / n * np.sum(prof * np.sin(2 * np.pi * (np.arange(n) + 0.5) / n))


def transient_amplitude(eta, f0, lam, rho, dt, nsteps):
    a = rho / dt - 0.5 * eta * lam
    b = rho / dt + 0.5 * eta * lam
    return f0 / (eta * lam) * (1.0 - (a / b) ** nsteps)


def eta_from_transient(A, f0, lam, rho, dt, nsteps):
    """The eta whose Crank-Nicolson transient reaches amplitude A after nsteps (bisection on
    log eta; A decreases monotonically with eta)."""
    lo, hi = -12.0, 12.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if transient_amplitude(np.exp(mid), f0, lam, rho, dt, nsteps) > A:
            lo = mid
        else:
            hi = mid
    return float(np.exp(0.5 * (lo + hi)))
