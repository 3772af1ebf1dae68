"""Seeded synthetic inputs for the FMM workloads.

This module holds input generators only (no FMM arithmetic); the tests, the
benchmark and the smoke check draw every point set and charge vector from
here, with numpy's PCG64 generator (``numpy.random.default_rng(seed)``).

The paper (Sec. III.A) benchmarks uniform points in a cube and on a sphere
surface; the workloads below follow those distributions plus a Plummer /
sphere-surface mix, Gaussian clusters and a thin-film surface-charge grid:

* ``uniform_cube``     points U[0,1)^3, charges U[-1,1]
* ``plummer_sphere``   70% Plummer sphere (scale a), 30% on the unit sphere
                       surface, charges +-1
* ``gaussian_clusters`` 8 centres U[0,1)^3, isotropic sigma, charges U[-1,1]
* ``thin_film``        surface charges of a 256x256 cell film of thickness
                       1/256 with a random unit magnetisation per cell
"""
import numpy as np


def uniform_cube(n, seed=0):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3))
    q = rng.uniform(-1.0, 1.0, n)
    return pos, q


def sample_targets(n, k, seed=1):
    """k distinct point indices (sorted) for error estimates on large N."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, k, replace=False)).astype(np.int64)


def _unit_vectors(rng, k):
    v = rng.normal(size=(k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def plummer_sphere(n, seed=0, a=0.05, plummer_fraction=0.7):
    """Plummer radii r = a / sqrt(u^(-2/3) - 1) (untruncated, isotropic, at the
    origin) for 70% of the points, the unit sphere surface for the rest."""
    rng = np.random.default_rng(seed)
    n_pl = int(round(plummer_fraction * n))
    u = rng.random(n_pl)
    u = np.where(u == 0.0, np.finfo(float).tiny, u)
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    pos_pl = _unit_vectors(rng, n_pl) * r[:, None]
    pos_sh = _unit_vectors(rng, n - n_pl)
    pos = np.concatenate([pos_pl, pos_sh], axis=0)
    q = rng.choice(np.array([-1.0, 1.0]), n)
    return pos, q


def gaussian_clusters(n, seed=0, n_clusters=8, sigma=0.02):
    rng = np.random.default_rng(seed)
    centres = rng.random((n_clusters, 3))
    which = rng.integers(0, n_clusters, n)
    pos = centres[which] + sigma * rng.normal(size=(n, 3))
    q = rng.uniform(-1.0, 1.0, n)
    return pos, q


def batched_sets(n_sets=64, seed=0, n_min=10_000, n_max=500_000):
    """Charge sets of log-uniform size, alternating uniform cube and Gaussian
    clusters.  Returns a list of (pos, q)."""
    rng = np.random.default_rng(seed)
    sizes = np.round(np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_sets))).astype(np.int64)
    out = []
    for i, m in enumerate(sizes):
        s = int(rng.integers(0, 2**31 - 1))
        out.append(uniform_cube(int(m), s) if i % 2 == 0 else gaussian_clusters(int(m), s))
    return out


def double_helix(n, seed=0, turns=4.0, radius=1.0, pitch=0.5, tube=0.05):
    """Two interleaved helical strands (phase offset pi) of the given radius,
    pitch and number of turns; points are scattered isotropically (Gaussian,
    standard deviation `tube`) around the strand centre lines; charges
    U[-1,1].  A project-made stand-in for the paper's double-helix example,
    whose parameters are not given."""
    rng = np.random.default_rng(seed)
    s = rng.random(n) * turns * 2.0 * np.pi
    strand = rng.integers(0, 2, n)
    phase = s + np.pi * strand
    pos = np.stack([radius * np.cos(phase), radius * np.sin(phase), pitch * s / (2.0 * np.pi)], axis=1)
    pos += tube * rng.normal(size=(n, 3))
    q = rng.uniform(-1.0, 1.0, n)
    return pos, q


def fibonacci_sphere(n, radius):
    """n points spread evenly over a sphere (golden-angle spiral): z_k equally
    spaced in (-1, 1), azimuth advancing by the golden angle."""
    k = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / n
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = k * np.pi * (3.0 - np.sqrt(5.0))
    return radius * np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


def active_shielding(seed=0, n_sh=128, r_sh=2.0, n_ext=256, r_ext=5.0, n_in=1024, r_in=1.5, n_out=1024,
                     r_out=2.5):
    """Geometry of the active-shielding demonstration (Sec. III.B): shield
    charge sites spread evenly on a sphere of radius r_sh, external charges
    U[-1,1] at uniformly random positions on a sphere of radius r_ext, and
    evenly spread sampling points inside (r_in) and outside (r_out)."""
    rng = np.random.default_rng(seed)
    return dict(shield=fibonacci_sphere(n_sh, r_sh), ext=_unit_vectors(rng, n_ext) * r_ext,
                q_ext=rng.uniform(-1.0, 1.0, n_ext), inside=fibonacci_sphere(n_in, r_in),
                outside=fibonacci_sphere(n_out, r_out))


def thin_film(cells=256, seed=0):
    """Film [0,1]^2 x [0,h], h = 1/cells, one random unit magnetisation m per
    cell.  Surface charges of div m sit at the top face centres (z = h,
    q = +m_z h^2) and bottom face centres (z = 0, q = -m_z h^2): 2 cells^2
    points (131072 for 256 x 256).  Lateral faces are not included."""
    rng = np.random.default_rng(seed)
    h = 1.0 / cells
    m = _unit_vectors(rng, cells * cells)
    ii, jj = np.meshgrid(np.arange(cells), np.arange(cells), indexing="ij")
    xc = ((ii.ravel() + 0.5) * h)
    yc = ((jj.ravel() + 0.5) * h)
    top = np.stack([xc, yc, np.full_like(xc, h)], axis=1)
    bot = np.stack([xc, yc, np.zeros_like(xc)], axis=1)
    pos = np.concatenate([top, bot], axis=0)
    q = np.concatenate([m[:, 2] * h * h, -m[:, 2] * h * h])
    return pos, q


# Workload parameters (expansion order p, leaf size N_max, splits s, theta).
CONFIGS = {
    "cube4k_p4": dict(n=4096, p=4, leaf_size=64, s=2, theta=0.4),
    "cube1m_p8": dict(n=1 << 20, p=8, leaf_size=128, s=2, theta=0.4),
    "plummer4m_p10": dict(n=1 << 22, p=10, leaf_size=64, s=2, theta=0.5),
    "batched64_p6": dict(p=6, s=2, theta=0.6),
    "film131k_p8": dict(n=131072, p=8, leaf_size=128, s=2, theta=0.5),
}
