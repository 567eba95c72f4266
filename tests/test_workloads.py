"""The synthetic input recipes (no GPU): particle counts, geometry and separation of the
workloads the benchmark and the full-size tests use.

- Dense suspension (Sec. 10): 128^3, a = 2.2h, phi = 0.40 -> 18,808 particles, 244,504 blobs,
  no two particle centres closer than the hard-sphere diameter 2a.
- Fluctuating suspension: 256^3, a = 3.2h, phi = 0.30 -> 36,669 particles, 476,697 blobs.
- Gap sweep (Sec. 8): surface gaps 0.05 * 80^(b / 31) h, equal and opposite forces.
- Every particle is a 13-blob icosahedron with the rest lengths of its 42 bonds.
"""
import numpy as np

from paper_1407_5600_gb300 import workloads as wl


def _centres(s):
    """Blob 0 of each particle is its centre blob (the icosahedron template's order)."""
    return s.pos[0::13].copy()


def test_dense_suspension_recipe():
    spec, s = wl.dense_suspension(n=128, seed=3)
    assert (spec.nx, spec.ny, spec.nz) == (128, 128, 128)
    assert s.n_particles == 18808 and len(s.pos) == 244504
    assert s.body == (1e-4, 0, 2, 1) and s.k_rep == 100.0 and s.r_cut == 1.0
    assert np.all((s.pos >= 0) & (s.pos < 128))
    # the hard-sphere preparation keeps the particle centres at least 2a apart (checked on a
    # sample of particles against all others)
    c = _centres(s)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(c), 200, replace=False):
        d = c - c[i]
        d -= 128.0 * np.round(d / 128.0)
        r = np.sqrt((d ** 2).sum(axis=1))
        r[i] = np.inf
        assert r.min() >= 2 * 2.2 - 1e-9


def test_fluctuating_suspension_recipe():
    spec, s = wl.fluctuating_suspension(n=256, a=3.2, phi=0.30, kT=1e-3, seed=5)
    assert s.n_particles == 36669 and len(s.pos) == 476697
    assert spec.kT == 1e-3 and s.body is None


def test_gap_sweep_recipe():
    B = 32
    for b in (0, 7, 31):
        spec, s = wl.gap_sweep_box(b, n_boxes=B, n=64, a=1.6)
        c = _centres(s)
        d = c[1] - c[0]
        d -= 64.0 * np.round(d / 64.0)
        gap_want = 0.05 * 80 ** (b / (B - 1))
        dv = s.pos[1:13] - s.pos[0]
        dv -= 64.0 * np.round(dv / 64.0)
        a_vertex = np.linalg.norm(dv, axis=1).mean()
        assert abs(np.linalg.norm(d) - 2 * 1.6 - gap_want) < 1e-9
        assert abs(a_vertex - 1.6) < 1e-9
        assert np.allclose(s.ext[:13].sum(axis=0), [1e-3, 0, 0])
        assert np.allclose(s.ext[13:].sum(axis=0), [-1e-3, 0, 0])


def test_icosahedron_topology():
    spec, s = wl.single_particle(n=32, a=1.0, seed=1)
    assert len(s.pos) == 13 and len(s.bonds) == 42
    r = np.linalg.norm(s.pos[s.bonds[:, 0]] - s.pos[s.bonds[:, 1]], axis=1)
    assert np.allclose(r, s.rest)
    d = 1.0 / (np.sqrt(10 + 2 * np.sqrt(5)) / 4)
    assert np.sum(np.isclose(s.rest, d)) == 30 and np.sum(np.isclose(s.rest, 1.0)) == 12
