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
    """Relative L2 error of the displacement q - q0 against q_ref - q0 (minimum image), with
    the rounding floor of FP64 positions: each step rounds a coordinate of magnitude <= L once,
    so differences of a few ulps of L per step are representation error, not method error."""
    L = np.asarray(L, dtype=np.float64)
    d = min_image(np.asarray(q) - q_ref, L)
    ref = min_image(np.asarray(q_ref) - q0, L)
    floor = 4.0 * max(nsteps, 1) * np.finfo(np.float64).eps * np.max(L) * np.sqrt(d.size)
    return np.linalg.norm(d) / (np.linalg.norm(ref) + floor / 1e-10)
