"""Seeded synthetic inputs shaped like the paper's workloads (arXiv:1407.5600).

This module holds only input construction: particle geometry, placement, bond lists and
force/body-force parameters.  It contains none of the method's arithmetic (no kernel, no
spreading, no fluid solve), imports nothing else from this package and is the only code that
both the CUDA path's callers and the CPU oracle's tests share.

Particle model (Sec. 2, Fig. ico): a filled icosahedron of N = 13 blobs, 12 on the vertices at
radius a and one at the centre, tied by stiff harmonic springs along the 30 edges (rest length
d, the vertex spacing) and the 12 centre-vertex spokes (rest length a).  The vertex radius is
a = sqrt(10 + 2 sqrt 5)/4 d = 0.951057 d (Sec. 2 prints a ~ 0.950 d; the Appendix prints the
formula with the 4 under the square root, which would give 1.902 d; the vertex coordinates below
fix the first reading).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GOLDEN = (1.0 + 5.0 ** 0.5) / 2.0
BLOBS_PER_PARTICLE = 13
BONDS_PER_PARTICLE = 42


def icosahedron_template(a: float):
    """Body-frame blob offsets [13][3] (index 0 = centre), local bonds [42][2], rest lengths.

    Vertices are the cyclic permutations of (0, +-1, +-g), scaled to circumradius a.
    """
    g = GOLDEN
    verts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            verts.append((0.0, s1, s2 * g))
            verts.append((s1, s2 * g, 0.0))
            verts.append((s2 * g, 0.0, s1))
    verts = np.array(verts)
    verts *= a / np.sqrt(1.0 + g * g)
    pos = np.vstack([np.zeros((1, 3)), verts])
    d2 = ((verts[:, None, :] - verts[None, :, :]) ** 2).sum(-1)
    edge2 = d2[d2 > 1e-12].min()
    bonds, rest = [], []
    for i in range(12):
        for j in range(i + 1, 12):
            if abs(d2[i, j] - edge2) < 1e-9 * edge2:
                bonds.append((i + 1, j + 1))
                rest.append(np.sqrt(d2[i, j]))
    assert len(bonds) == 30
    for i in range(12):
        bonds.append((0, i + 1))
        rest.append(np.sqrt((verts[i] ** 2).sum()))
    return pos, np.array(bonds, dtype=np.int32), np.array(rest)


def vertex_spacing(a: float) -> float:
    """Edge length d of the icosahedron of vertex radius a."""
    return a * 4.0 / np.sqrt(10.0 + 2.0 * np.sqrt(5.0))


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix from a normalised Gaussian quaternion."""
    qv = rng.normal(size=4)
    w, x, y, z = qv / np.linalg.norm(qv)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


@dataclass
class Suspension:
    """Blobs of one periodic box: positions [n][3] in [0, L), particle ids, bonds, rest lengths."""
    pos: np.ndarray
    pid: np.ndarray
    bonds: np.ndarray
    rest: np.ndarray
    n_particles: int
    a: float
    L: np.ndarray
    ext: np.ndarray | None = None          # external blob forces [n][3] or None
    body: tuple | None = None              # (f0, axis, wave_dir, j) or None
    k_spring: float = 100.0
    k_rep: float = 0.0
    r_cut: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def n_blobs(self) -> int:
        return len(self.pos)


def build_particles(centres, a, rng, L, with_rotation=True) -> Suspension:
    """Place one 13-blob icosahedron at each centre with a seeded random orientation."""
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    L = np.asarray(L, dtype=np.float64)
    tpl, tb, tr = icosahedron_template(a)
    npart = len(centres)
    pos = np.empty((npart * 13, 3))
    for p in range(npart):
        R = random_rotation(rng) if with_rotation else np.eye(3)
        pos[13 * p:13 * p + 13] = centres[p] + tpl @ R.T
    pos = np.mod(pos, L)
    pos = np.where(pos >= L, 0.0, pos)
    pid = np.repeat(np.arange(npart, dtype=np.int32), 13)
    bonds = (tb[None, :, :] + 13 * np.arange(npart, dtype=np.int32)[:, None, None]).reshape(-1, 2)
    rest = np.tile(tr, npart)
    return Suspension(pos=pos, pid=pid, bonds=bonds.astype(np.int32), rest=rest,
                      n_particles=npart, a=a, L=L)


# ---------------------------------------------------------------------------------------------
# Placement helpers.

def _fcc_sites(L: float, n_min: int) -> np.ndarray:
    """Smallest cubic FCC lattice filling the box with at least n_min sites."""
    m = 1
    while 4 * m ** 3 < n_min:
        m += 1
    c = L / m
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    ijk = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1)
    sites = (ijk.reshape(-1, 1, 3) + base[None]).reshape(-1, 3) * c + 0.25 * c
    return sites


def hard_sphere_mc(centres, L, r_hs, rng, sweeps, max_disp):
    """Parallel hard-sphere Monte Carlo moves at zero Peclet number (Sec. 10 preparation).

    Every sweep proposes a uniform displacement for all particles at once and accepts a move
    when the new position overlaps neither any old position nor any other proposed new position,
    which keeps the configuration overlap-free (centre distance >= 2 r_hs)."""
    from scipy.spatial import cKDTree

    x = np.mod(np.asarray(centres, dtype=np.float64), L)
    dmin = 2.0 * r_hs
    for _ in range(sweeps):
        prop = np.mod(x + rng.uniform(-max_disp, max_disp, size=x.shape), L)
        prop[prop >= L] = 0.0
        ok = np.ones(len(x), dtype=bool)
        old_tree = cKDTree(x, boxsize=L)
        new_tree = cKDTree(prop, boxsize=L)
        for i, js in enumerate(old_tree.query_ball_point(prop, dmin)):
            if any(j != i for j in js):
                ok[i] = False
        for i, js in enumerate(new_tree.query_ball_point(prop, dmin)):
            if any(j != i for j in js):
                ok[i] = False
        x[ok] = prop[ok]
    return x


def random_nonoverlapping(n, L, r_hs, rng, max_tries=100000):
    """Random sequential addition of n spheres of radius r_hs (dilute cases only)."""
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("random sequential addition did not converge")
        c = rng.uniform(0.0, L, size=3)
        ok = True
        for o in out:
            d = c - o
            d -= L * np.round(d / L)
            if (d * d).sum() < (2 * r_hs) ** 2:
                ok = False
                break
        if ok:
            out.append(c)
    return np.array(out)


# ---------------------------------------------------------------------------------------------
# The workloads.

@dataclass
class GridSpec:
    nx: int
    ny: int
    nz: int
    h: float = 1.0
    rho: float = 1.0
    eta: float = 1.0
    dt: float = 0.05
    mean_mode: int = 0
    kT: float = 0.0


def single_particle(n=32, a=1.0, seed=1, force_x=1e-3, k_spring=100.0):
    """One 13-blob particle (vertex radius a) in an n^3 box pulled by a total force force_x
    along x, split equally over its blobs (Stokeslet / Hasimoto drag experiment, Sec. 5.1)."""
    rng = np.random.default_rng(seed)
    L = float(n)
    centre = rng.uniform(0.0, L, size=3)
    s = build_particles(centre, a, rng, np.array([L, L, L]))
    ext = np.zeros_like(s.pos)
    ext[:, 0] = force_x / 13.0
    s.ext = ext
    s.k_spring = k_spring
    s.meta = {"workload": f"single particle a={a}h in {n}^3", "seed": seed}
    return GridSpec(n, n, n, dt=0.05, mean_mode=1), s


def gap_sweep_box(b, n_boxes=32, n=64, a=1.6, force=1e-3, k_spring=100.0,
                  gmin=0.05, gmax=4.0):
    """Box b of the gap sweep: two particles on a line along x through the box centre, surface
    gap g_b = gmin (gmax/gmin)^(b/(B-1)) h, pulled together by equal and opposite forces
    (pair mobility and lubrication, Sec. 8)."""
    rng = np.random.default_rng(2 + b)
    L = float(n)
    gap = gmin * (gmax / gmin) ** (b / max(n_boxes - 1, 1))
    sep = 2 * a + gap
    c = np.array([L / 2, L / 2, L / 2])
    centres = np.array([c - [sep / 2, 0, 0], c + [sep / 2, 0, 0]])
    s = build_particles(centres, a, rng, np.array([L, L, L]))
    ext = np.zeros_like(s.pos)
    ext[:13, 0] = force / 13.0
    ext[13:, 0] = -force / 13.0
    s.ext = ext
    s.k_spring = k_spring
    s.meta = {"gap": gap, "box": b}
    return GridSpec(n, n, n, dt=0.05, mean_mode=0), s


def dense_suspension(n=128, a=2.2, phi=0.40, seed=3, f0=1e-4, k_spring=100.0,
                     k_rep=100.0, r_cut=1.0, mc_sweeps=6, n_particles=None):
    """Dense suspension for the viscosity protocol (Sec. 10): n_p = round(phi L^3 / (4/3 pi a^3))
    particles on an FCC start with random vacancies, randomised by hard-sphere Monte Carlo at
    R_HS = a, driven by the body force f0 sin(2 pi z / L) x_hat."""
    rng = np.random.default_rng(seed)
    L = float(n)
    if n_particles is None:
        n_particles = int(round(phi * L ** 3 / (4.0 / 3.0 * np.pi * a ** 3)))
    sites = _fcc_sites(L, n_particles)
    keep = rng.permutation(len(sites))[:n_particles]
    centres = sites[np.sort(keep)]
    spacing = (L / round((len(sites) / 4) ** (1 / 3)))
    max_disp = max(0.05, 0.5 * (spacing / np.sqrt(2) - 2 * a))
    centres = hard_sphere_mc(centres, L, a, rng, mc_sweeps, max_disp)
    s = build_particles(centres, a, rng, np.array([L, L, L]))
    s.body = (f0, 0, 2, 1)
    s.k_spring = k_spring
    s.k_rep = k_rep
    s.r_cut = r_cut
    s.meta = {"workload": f"dense suspension {n}^3 a={a}h phi={phi}", "seed": seed,
              "n_particles": n_particles}
    return GridSpec(n, n, n, dt=0.05, mean_mode=0), s


def fluctuating_suspension(n=256, a=3.2, phi=0.30, kT=1e-3, seed=5, mc_sweeps=3,
                           k_spring=100.0, k_rep=100.0, r_cut=1.0):
    """Thermal suspension (fluctuating stress, Sec. 3 and Eq. ef): the dense-suspension recipe
    at radius a and volume fraction phi, at rest (no body force), with thermal energy kT
    (spec.kT) for the equipartition and velocity-autocorrelation runs."""
    spec, s = dense_suspension(n=n, a=a, phi=phi, seed=seed, k_spring=k_spring, k_rep=k_rep,
                               r_cut=r_cut, mc_sweeps=mc_sweeps)
    s.body = None
    s.meta["workload"] = f"fluctuating suspension {n}^3 a={a}h phi={phi} kT={kT}"
    spec.kT = kT
    return spec, s


def dilute_random(n=64, n_particles=64, a=2.0, seed=4, k_spring=100.0):
    """Particles at seeded random non-overlapping positions (differentiable workload)."""
    rng = np.random.default_rng(seed)
    L = float(n)
    centres = random_nonoverlapping(n_particles, L, a + 0.5, rng)
    s = build_particles(centres, a, rng, np.array([L, L, L]))
    s.k_spring = k_spring
    s.meta = {"seed": seed}
    return GridSpec(n, n, n, dt=0.05, mean_mode=0), s


def random_blobs(nblobs, shape, seed, h=1.0, per_particle=13):
    """Unstructured blob cloud (uniform positions, Gaussian forces) for operator tests."""
    rng = np.random.default_rng(seed)
    L = np.array([shape[2], shape[1], shape[0]], dtype=np.float64) * h
    q = rng.uniform(0.0, 1.0, size=(nblobs, 3)) * L
    q[q >= L] = 0.0
    F = rng.normal(size=(nblobs, 3))
    pid = (np.arange(nblobs) // per_particle).astype(np.int32)
    return q, F, pid


def random_field(shape, seed, scale=1.0):
    """Gaussian MAC velocity field [3][nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=(3,) + tuple(shape))
