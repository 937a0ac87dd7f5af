"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds no DDA arithmetic: only particle geometries (which cells of a box a
shape covers), seeded random vectors and the named workload parameters.  The
shapes follow the paper's workloads: homogeneous spheres on a cubic grid
with about 10 dipoles per wavelength in the medium (Sec. 3.1), plus the
ellipsoids and cubes used for batching.
"""
import math

import numpy as np


def _centred_sq(n):
    """(2 i + 1 - n)^2 for i in 0..n-1 as int64: squared doubled offsets of cell
    centres from the box centre."""
    i = np.arange(n, dtype=np.int64)
    return (2 * i + 1 - n) ** 2


def sphere(n, material=1):
    """uint8 (n, n, n) [z, y, x]: cells whose centres lie in the inscribed sphere."""
    q = _centred_sq(n)
    inside = (q[:, None, None] + q[None, :, None] + q[None, None, :]) <= n * n
    return (inside * material).astype(np.uint8)


def ellipsoid(nx, ny, nz, material=1):
    """uint8 (nz, ny, nx): the ellipsoid inscribed in the box."""
    qx = _centred_sq(nx) * (ny * nz) ** 2
    qy = _centred_sq(ny) * (nx * nz) ** 2
    qz = _centred_sq(nz) * (nx * ny) ** 2
    inside = (qz[:, None, None] + qy[None, :, None] + qx[None, None, :]) <= (nx * ny * nz) ** 2
    return (inside * material).astype(np.uint8)


def cube(nx, ny, nz, material=1):
    return np.full((nz, ny, nx), material, dtype=np.uint8)


def layered_sphere(n, n_mat):
    """Sphere split into n_mat slabs along z (material k in slab k): a
    multi-material test geometry."""
    occ = sphere(n)
    z = np.arange(n)
    lay = 1 + (z * n_mat) // n
    return (occ * lay[:, None, None]).astype(np.uint8)


def random_occupancy(nx, ny, nz, fill, seed, n_mat=1):
    """Random occupancy (rows may hold several runs), materials 1..n_mat."""
    rng = np.random.default_rng(seed)
    occ = (rng.random((nz, ny, nx)) < fill).astype(np.uint8)
    mats = rng.integers(1, n_mat + 1, size=occ.shape).astype(np.uint8)
    return occ * mats


def random_vectors(seed, nrhs, n_occ, dtype=np.complex128):
    """Seeded complex normal vectors [nrhs][3][n_occ]."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((nrhs, 3, n_occ)) + 1j * rng.standard_normal((nrhs, 3, n_occ))
    return v.astype(dtype)


def random_unit_vectors(seed, k):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def perpendicular_pols(prop):
    """Two real unit polarisations orthogonal to prop (and each other)."""
    a = np.asarray(prop, dtype=np.float64)
    t = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = t - a * np.dot(a, t)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    return e1, e2


# Named workloads: spheres sized by the paper's rule of ~10 dipoles per
# wavelength in the medium, i.e. about 3.18 x m dipoles across the diameter
# (Sec. 3.1).
WORKLOADS = {
    # x = 3, m = 1.5, 16^3 box, both polarisations along z, LDR, QMR to 1e-5
    "sphere16_x3_m1.5": dict(n=16, x=3.0, m=1.5 + 0.0j, pol="ldr"),
    # x = 40, m = 1.05, 134^3 box (1,260,552 dipoles), x-polarised, LDR
    "sphere134_x40_m1.05": dict(n=134, x=40.0, m=1.05 + 0.0j, pol="ldr"),
    # x = 20, m = 2.0, 128^3 box
    "sphere128_x20_m2": dict(n=128, x=20.0, m=2.0 + 0.0j, pol="ldr"),
    # x = 40, m = 2.0, 256^3 box
    "sphere256_x40_m2": dict(n=256, x=40.0, m=2.0 + 0.0j, pol="ldr"),
}


def batch_instances(count=128, seed=704037):
    """Seeded batch of particles (numpy PCG64), drawn per particle in this
    order: shape uniform over (sphere, ellipsoid, cube); size parameter
    x ~ U[2, 15] (volume-equivalent); refractive index m ~ U[1.05, 2.0] (real);
    for ellipsoids two axis ratios ~ U[1, 3]; then 8 incidence directions
    uniform on the sphere.  The lattice has n = clamp(ceil(10 x m / pi), 16, 64)
    dipoles along the major axis (about 10 per wavelength in the medium,
    Sec. 3.1's rule) and n / ratio along the minor axes.  Each direction gets
    two perpendicular polarisations: 16 right-hand sides per particle.
    Returns a list of dicts (shape, x, m, occ, prop (16, 3), pol (16, 3))."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        shape = ("sphere", "ellipsoid", "cube")[int(rng.integers(0, 3))]
        x = float(rng.uniform(2.0, 15.0))
        m = float(rng.uniform(1.05, 2.0))
        ratios = rng.uniform(1.0, 3.0, size=2) if shape == "ellipsoid" else np.ones(2)
        a = rng.standard_normal((8, 3))
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        n = int(min(64, max(16, math.ceil(10.0 * x * m / math.pi))))
        if shape == "sphere":
            occ = sphere(n)
        elif shape == "cube":
            occ = cube(n, n, n)
        else:
            ny = max(2, int(round(n / ratios[0])))
            nz = max(2, int(round(n / ratios[1])))
            occ = ellipsoid(n, ny, nz)
        prop, pol = [], []
        for ai in a:
            for e in perpendicular_pols(ai):
                prop.append(ai)
                pol.append(e)
        out.append(dict(shape=shape, x=x, m=m, occ=occ, prop=np.array(prop), pol=np.array(pol)))
    return out


def angles_deg(count=181):
    """Scattering angles 0..180 degrees in equal steps (181 -> 1 degree)."""
    return np.linspace(0.0, 180.0, count)


def size_rule_n(x, m, per_wavelength=10.0):
    """Dipoles across the diameter for a given number per wavelength in the
    medium: n = per_wavelength * x * |m| / pi (3.18 x m at 10 per wavelength)."""
    return int(math.ceil(per_wavelength * x * abs(m) / math.pi))


def sphere_cluster(n, count, seed, material=1):
    """uint8 (n, n, n): the union of `count` spheres with random diameters
    between n/3 and n/2, centres drawn so that each sphere lies inside the
    box and touches or overlaps the cluster's first sphere's neighbourhood
    (centres within one diameter of the box centre)."""
    rng = np.random.default_rng(seed)
    c = (np.arange(n) + 0.5)
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    occ = np.zeros((n, n, n), dtype=bool)
    for _ in range(count):
        d = rng.uniform(n / 3.0, n / 2.0)
        r = d / 2.0
        ctr = n / 2.0 + rng.uniform(-1.0, 1.0, size=3) * min(d, n / 2.0 - r)
        occ |= (xx - ctr[0]) ** 2 + (yy - ctr[1]) ** 2 + (zz - ctr[2]) ** 2 <= r * r
    return (occ * material).astype(np.uint8)


def training_particles(count, n=64, seed=704037):
    """(occupancy, m, kd) of the learned preconditioner's training runs:
    ellipsoids with random axis ratios in [1, 3] and clusters of 2 to 4
    spheres, in boxes of up to n cells per axis, real m uniform in [1.5, 2.0],
    10 dipoles per wavelength in the material (kd = 2 pi / (10 m))."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        m = float(rng.uniform(1.5, 2.0))
        if rng.random() < 0.5:
            r1, r2 = rng.uniform(1.0, 3.0, size=2)
            occ = ellipsoid(n, max(8, int(round(n / r1))), max(8, int(round(n / r2))))
        else:
            occ = sphere_cluster(n, int(rng.integers(2, 5)), int(rng.integers(1 << 31)))
        out.append((occ, m, 2.0 * math.pi / (10.0 * m)))
    return out
