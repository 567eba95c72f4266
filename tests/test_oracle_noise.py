"""Pins of the oracle's thermal stress (the fluctuating stress of Eq. vf, Sec. 3) against
what a library, the mathematics and the paper fix (no GPU).

- Philox4x64-10 equals numpy's Philox bit generator (same published algorithm).
- The per-cell normals are standard normal and independent across components, cells, steps,
  boxes and seeds.
- The stress divergence is the MAC divergence of a staggered tensor: it maps the MAC gradient
  of a velocity field to its 7-point Laplacian, an isotropic stress to a pure gradient (which
  the projection removes), and D D^T = -L exactly.
- Eq. (ef): the fluid velocity of the fluctuating Crank-Nicolson step has the equipartition
  variance kT/(rho h^3) per projected mode.
"""
import numpy as np
import pytest

import oracle as mb


def _numpy_philox(counter, key):
    """numpy advances its 256-bit counter before each block: start one below."""
    c = [int(x) for x in counter]
    for i in range(4):
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = (1 << 64) - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(c, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("counter,key", [
    ([1, 0, 0, 0], [0, 0]),
    ([0, 0, 0, 0], [7, 0]),
    ([123456789, 42, 3, 1], [2024, 0]),
    ([2 ** 64 - 1, 2 ** 64 - 1, 5, 0], [2 ** 63 + 11, 2 ** 62 + 3]),
    ([0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0, 0x082EFA98EC4E6C89],
     [0x452821E638D01377, 0xBE5466CF34E90C6C]),
])
def test_philox_matches_numpy(counter, key):
    got = mb.philox4x64(counter, key)
    want = _numpy_philox(counter, key)
    assert np.array_equal(got, want), ([hex(int(x)) for x in got], [hex(int(x)) for x in want])


def test_stress_normals_are_standard_normal_and_independent():
    stats = pytest.importorskip("scipy.stats")
    g = mb.Grid(32, 16, 16)
    W = mb.stress_normals(g, seed=11, step=3, box=0)
    n = W[0].size
    for c in range(9):
        x = W[c].ravel()
        assert abs(x.mean()) < 5.0 / np.sqrt(n)
        assert abs(x.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    # the nine components, and neighbouring cells, are uncorrelated
    C = np.corrcoef(W.reshape(9, -1))
    assert np.max(np.abs(C - np.eye(9))) < 5.0 / np.sqrt(n)
    for ax in (1, 2, 3):
        r = np.mean(W * np.roll(W, 1, axis=ax))
        assert abs(r) < 5.0 / np.sqrt(9 * n)
    # pairs of one Box-Muller draw (xx, xy) are jointly isotropic: the angle is uniform
    ang = np.arctan2(W[1].ravel(), W[0].ravel())
    assert stats.kstest(ang, "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-4


def test_stress_normals_depend_on_every_key():
    g = mb.Grid(8, 8, 8)
    base = mb.stress_normals(g, 5, 10, 0)
    assert np.array_equal(base, mb.stress_normals(g, 5, 10, 0))
    for other in (mb.stress_normals(g, 6, 10, 0), mb.stress_normals(g, 5, 11, 0),
                  mb.stress_normals(g, 5, 10, 1)):
        assert abs(np.corrcoef(base.ravel(), other.ravel())[0, 1]) < 0.05


def _lap(u, h):
    """7-point Laplacian of a periodic array [nz][ny][nx]."""
    return sum(np.roll(u, 1, axis=a) - 2 * u + np.roll(u, -1, axis=a) for a in range(3)) / h ** 2


def _shift(u, axis_xyz, s):
    """u at index i + s along x (0), y (1) or z (2), periodic."""
    return np.roll(u, -s, axis=2 - axis_xyz)


def test_divergence_of_mac_gradient_is_laplacian():
    """Staggered velocity gradient: G_aa = forward difference to the cell centre, G_ab =
    backward difference to the edge (b != a).  Its divergence must be L u per component."""
    g = mb.Grid(8, 16, 4, h=0.7)
    rng = np.random.default_rng(1)
    u = rng.normal(size=(3,) + g.shape)
    W = np.zeros((9,) + g.shape)
    for a in range(3):
        for b in range(3):
            if a == b:
                W[3 * a + b] = (_shift(u[a], b, 1) - u[a]) / g.h
            else:
                W[3 * a + b] = (u[a] - _shift(u[a], b, -1)) / g.h
    f = mb.stress_div(g, W)
    for a in range(3):
        want = _lap(u[a], g.h)
        assert np.max(np.abs(f[a] - want)) < 1e-12 * np.max(np.abs(want))


def test_isotropic_stress_is_a_gradient_removed_by_projection():
    g = mb.Grid(8, 8, 16, h=1.3, rho=1.0, eta=0.9, dt=0.1, mean_mode=1)
    rng = np.random.default_rng(2)
    p = rng.normal(size=g.shape)
    W = np.zeros((9,) + g.shape)
    for a in range(3):
        W[4 * a] = p
    f = mb.stress_div(g, W)
    for a in range(3):       # the MAC gradient (centres to faces, backward difference)
        assert np.allclose(f[a], (p - _shift(p, a, -1)) / g.h, rtol=0, atol=1e-13)
    v = mb.fluid_update(g, g.zeros(), f)
    assert np.max(np.abs(v)) < 1e-12 * np.max(np.abs(f))


def test_noise_covariance_is_minus_laplacian():
    """D D^T = -L (block diagonal over components): the noise force has covariance
    (2 eta kT/(h^3 dt)) (-L), the fluctuation-dissipation balance of the viscous term."""
    g = mb.Grid(4, 8, 4, h=0.8)
    N = 4 * 8 * 4
    D = np.zeros((3 * N, 9 * N))
    for j in range(9 * N):
        e = np.zeros(9 * N)
        e[j] = 1.0
        D[:, j] = mb.stress_div(g, e.reshape((9,) + g.shape)).ravel()
    L = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        L[:, j] = _lap(e.reshape(g.shape), g.h).ravel()
    want = np.kron(np.eye(3), -L)
    assert np.max(np.abs(D @ D.T - want)) < 1e-12 * np.max(np.abs(want))


def _equipartition_fraction(g):
    """(1/N) sum over k != 0 of the projector diagonal P_aa(k) = 1 - |D_a|^2 / lambda, per a."""
    n = (g.nx, g.ny, g.nz)
    s2 = [4.0 / g.h ** 2 * np.sin(np.pi * np.arange(m) / m) ** 2 for m in n]
    Sx, Sy, Sz = np.meshgrid(s2[0], s2[1], s2[2], indexing="ij")
    lam = Sx + Sy + Sz
    lam[0, 0, 0] = 1.0
    out = []
    for Sa in (Sx, Sy, Sz):
        Paa = 1.0 - Sa / lam
        Paa[0, 0, 0] = 0.0
        out.append(Paa.sum() / lam.size)
    return np.array(out)


def test_fluid_equipartition_eq_ef():
    """Fluid only, kT > 0: after relaxation the per-component variance of the staggered
    velocity is (kT / (rho h^3)) (1/N) sum_k P_aa(k), the discrete form of Eq. (ef)."""
    g = mb.Grid(8, 8, 16, h=0.7, rho=0.8, eta=1.3, dt=0.4, mean_mode=0)
    kT = 2.5e-3
    empty = dict(pid=np.zeros(0, np.int32), bonds=np.zeros((0, 2), np.int32),
                 rest=np.zeros(0), k_spring=0.0)
    q = np.zeros((0, 3))
    v = g.zeros()
    q, v = mb.step(g, 40, q, v, kT=kT, seed=3, step0=0, **empty)
    acc = np.zeros(3)
    m = 0
    stride, samples = 4, 500
    for s in range(samples):
        q, v = mb.step(g, stride, q, v, kT=kT, seed=3, step0=40 + stride * s, **empty)
        acc += (v ** 2).mean(axis=(1, 2, 3))
        m += 1
    var = acc / m
    want = kT / (g.rho * g.h ** 3) * _equipartition_fraction(g)
    assert np.all(np.abs(var / want - 1.0) < 0.04), (var, want)
    # the mean momentum stays at zero (a divergence has no k = 0 part)
    assert np.max(np.abs(v.mean(axis=(1, 2, 3)))) < 1e-14


def test_noise_steps_compose_and_kT_zero_is_deterministic():
    g = mb.Grid(8, 8, 8, dt=0.1)
    rng = np.random.default_rng(4)
    q0 = rng.uniform(0, 8, size=(5, 3))
    args = dict(pid=np.arange(5, dtype=np.int32), bonds=np.zeros((0, 2), np.int32),
                rest=np.zeros(0), k_spring=0.0, ext=rng.normal(scale=1e-2, size=(5, 3)))
    qa, va = mb.step(g, 2, q0, g.zeros(), kT=1e-3, seed=9, step0=5, **args)
    q1, v1 = mb.step(g, 1, q0, g.zeros(), kT=1e-3, seed=9, step0=5, **args)
    qb, vb = mb.step(g, 1, q1, v1, kT=1e-3, seed=9, step0=6, **args)
    assert np.array_equal(qa, qb) and np.array_equal(va, vb)
    qd, vd = mb.step(g, 2, q0, g.zeros(), **args)
    qz, vz = mb.step(g, 2, q0, g.zeros(), kT=0.0, seed=9, step0=5, **args)
    assert np.array_equal(qd, qz) and np.array_equal(vd, vz)
    assert not np.allclose(va, vd)
