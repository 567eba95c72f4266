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
