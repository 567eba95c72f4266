"""Pins of the oracle's kernel, spreading and interpolation (no GPU).

Each check is fixed by the paper or by mathematics, not by the oracle itself:
kernel moments (Sec. 2 after Eq. delta), the Faxen second moment (Sec. 9, Eq. jblob2),
brute-force dense spreading over every node (Sec. 2: f_i(r) = delta_h(r - q_i) F_i),
adjointness of S and J and J_i S_i = 1/(8h^3) (Sec. 2), exactness of J on constant and
linear fields (zeroth and first moments).
"""
import json
import os

import numpy as np
import pytest

import oracle as mb
from paper_1407_5600_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _phi_vec(r):
    return np.vectorize(mb.phi)(r)


def test_phi_moments_every_offset():
    gold = json.load(open(os.path.join(GOLD, "kernel_properties.json")))
    for x in np.linspace(0.0, 1.0, 257):
        j = np.arange(-3, 5)
        w = _phi_vec(j - x)
        assert abs(w.sum() - gold["sum_phi"]) < 1e-15
        assert abs(((j - x) * w).sum() - gold["first_moment"]) < 1e-15
        assert abs((w * w).sum() - gold["sum_phi_squared"]) < 1e-15


def test_phi_support_and_continuity():
    assert mb.phi(1.5) == 0.0 and mb.phi(-1.5) == 0.0 and mb.phi(2.0) == 0.0
    for r0 in (0.5, 1.5):
        lo, hi = mb.phi(r0 - 1e-12), mb.phi(r0 + 1e-12)
        assert abs(lo - hi) < 1e-10
    # symmetric
    for r in np.linspace(0, 1.6, 33):
        assert mb.phi(r) == mb.phi(-r)


def test_faxen_second_moment_range():
    """a_F^2 = 3 sum r^2 Phi lies in [0.75, 1] h^2: 1 at a node, 3/4 at a midpoint, so
    a_F in [0.866, 1] h, consistent with the printed (0.95 +- 0.05) h."""
    gold = json.load(open(os.path.join(GOLD, "kernel_properties.json")))["faxen_radius"]
    vals = []
    for x in np.linspace(0.0, 1.0, 129):
        j = np.arange(-3, 5)
        vals.append(3.0 * (((j - x) ** 2) * _phi_vec(j - x)).sum())
    vals = np.array(vals)
    assert abs(vals[0] - 1.0) < 1e-14 and abs(vals[64] - 0.75) < 1e-14
    assert vals.min() >= 0.75 - 1e-14 and vals.max() <= 1.0 + 1e-14
    aF = np.sqrt(vals)
    assert np.all(np.abs(aF - gold["a_F"]) <= gold["spread"] + 0.04)


def _dense_spread(g, q, F):
    """Brute force: every node of every component against every blob, minimum image."""
    nz, ny, nx = g.shape
    L = g.L
    f = np.zeros((3, nz, ny, nx))
    n = np.array([nx, ny, nz])
    for comp in range(3):
        shift = np.array([0.5, 0.5, 0.5])
        shift[comp] = 0.0
        ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        nodes = (np.stack([ii, jj, kk], -1).reshape(-1, 3) + shift) * g.h
        for b in range(len(q)):
            d = nodes - q[b]
            d -= L * np.round(d / L)
            w = _phi_vec(d[:, 0] / g.h) * _phi_vec(d[:, 1] / g.h) * _phi_vec(d[:, 2] / g.h)
            w = w.reshape(nx, ny, nz).transpose(2, 1, 0)
            f[comp] += w * F[b, comp] / g.h ** 3
    del n
    return f


@pytest.mark.parametrize("shape,h", [((4, 4, 4), 1.0), ((7, 6, 5), 0.5), ((8, 8, 8), 2.0)])
def test_spread_matches_bruteforce(shape, h):
    g = mb.Grid(shape[2], shape[1], shape[0], h=h)
    q, F, _ = wl.random_blobs(6, shape, seed=11, h=h)
    # include blobs exactly on nodes, faces and the periodic boundary
    q[0] = [0.0, 0.0, 0.0]
    q[1] = [0.5 * h, h, 1.5 * h]
    q[2] = g.L - 1e-9
    f = mb.spread(g, q, F)
    ref = _dense_spread(g, q, F)
    assert np.max(np.abs(f - ref)) <= 1e-14 * max(1.0, np.max(np.abs(ref)))


def test_adjointness_and_self_overlap():
    g = mb.Grid(16, 12, 8, h=0.7)
    q, F, _ = wl.random_blobs(40, g.shape, seed=5, h=g.h)
    v = wl.random_field(g.shape, seed=6)
    lhs = g.h ** 3 * np.sum(mb.spread(g, q, F) * v)
    rhs = np.sum(F * mb.interp(g, q, v))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
    # J_i S_i e = e / (8 h^3) for one blob anywhere (grid-independent L2 norm)
    rng = np.random.default_rng(3)
    for _ in range(20):
        qb = rng.uniform(0, 1, size=(1, 3)) * g.L
        for comp in range(3):
            e = np.zeros((1, 3))
            e[0, comp] = 1.0
            u = mb.interp(g, qb, mb.spread(g, qb, e))
            assert abs(u[0, comp] - 1.0 / (8 * g.h ** 3)) < 1e-13 / g.h ** 3
            assert np.all(np.abs(np.delete(u[0], comp)) < 1e-15)


def test_interp_constant_and_linear_fields_exact():
    g = mb.Grid(16, 16, 16, h=1.3)
    rng = np.random.default_rng(9)
    # constant field: J[1] = 1
    v = np.ones((3,) + g.shape) * np.array([1.5, -2.0, 0.25])[:, None, None, None]
    q = rng.uniform(0, 1, size=(50, 3)) * g.L
    u = mb.interp(g, q, v)
    assert np.max(np.abs(u - [1.5, -2.0, 0.25])) < 1e-14
    # linear field (no wrap inside the 3-node window): J[r - q] = 0
    q = rng.uniform(4, 12, size=(50, 3)) * g.h
    nz, ny, nx = g.shape
    a = np.array([0.3, -0.7, 1.1])
    for comp in range(3):
        shift = np.array([0.5, 0.5, 0.5])
        shift[comp] = 0.0
        X = (np.arange(nx) + shift[0]) * g.h
        Y = (np.arange(ny) + shift[1]) * g.h
        Z = (np.arange(nz) + shift[2]) * g.h
        field = (a[0] * X[None, None, :] + a[1] * Y[None, :, None] + a[2] * Z[:, None, None])
        vv = np.zeros((3,) + g.shape)
        vv[comp] = field
        u = mb.interp(g, q, vv)
        assert np.max(np.abs(u[:, comp] - q @ a)) < 1e-12


def test_faxen_identity_multiblob():
    """Appendix, Eq. jm2a with the centre blob kept: J_m[(r - q0)^2] =
    (1/N) sum_i a_F^2(q_i) + (1/N) sum_i |s_i|^2 (for N = 13 the second term is 12 a^2/13)."""
    g = mb.Grid(24, 24, 24, h=1.0)
    rng = np.random.default_rng(2)
    a = 2.0
    s = wl.build_particles(np.array([12.3, 11.7, 12.9]), a, rng, g.L)
    q = s.pos
    q0 = q.mean(0)
    nz, ny, nx = g.shape
    for comp in range(3):
        shift = np.array([0.5, 0.5, 0.5])
        shift[comp] = 0.0
        X = (np.arange(nx) + shift[0]) * g.h - q0[0]
        Y = (np.arange(ny) + shift[1]) * g.h - q0[1]
        Z = (np.arange(nz) + shift[2]) * g.h - q0[2]
        r2 = X[None, None, :] ** 2 + Y[None, :, None] ** 2 + Z[:, None, None] ** 2
        vv = np.zeros((3,) + g.shape)
        vv[comp] = r2
        lhs = mb.interp(g, q, vv)[:, comp].mean()
        aF2 = []
        for qi in q:
            tot = 0.0
            for d in range(3):
                x = qi[d] / g.h - shift[d]
                j = np.arange(np.floor(x) - 3, np.floor(x) + 4)
                tot += (((j - x) ** 2) * _phi_vec(j - x)).sum() * g.h ** 2
            aF2.append(tot)
        rhs = np.mean(aF2) + np.mean(((q - q0) ** 2).sum(1))
        assert abs(lhs - rhs) < 1e-12 * rhs
        assert abs(np.mean(((q - q0) ** 2).sum(1)) - 12 * a * a / 13) < 1e-12
