"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This module holds none of the method's arithmetic: it only draws initial density /
velocity fields and solid masks with the shapes of the paper's workloads.  All
fields are float64 numpy arrays shaped (nz, ny, nx) (velocity (3, nz, ny, nx)),
solid masks are uint8 (1 = solid).  Every generator takes an explicit seed or is
deterministic.

Recipes (sizes and structure of the paper's cases):
* ``droplet``: a sphere of radius R with the tanh profile of Eq. e23 (width W) between
  liquid and vapour densities (static droplet, Sec. III A / III C).
* ``random_spheres``: non-overlapping spheres with radii drawn uniformly, placed with a
  periodic minimum gap, until a liquid volume fraction is reached (many droplets in
  vapour, the "plain method at scale" workload).
* ``impact``: a droplet above a flat wall moving toward it (Sec. III E / IV A).
* ``cylinder_mask``: a solid cylinder lying on the bottom wall (Sec. IV B).
* ``cylinder_impact``: a droplet falling onto such a cylinder (Sec. IV B), and
  ``serving_jobs``: a seeded mix of cylinder-impact and static-droplet jobs of uneven sizes
  with Poisson arrival times, the request stream of a job server.
* ``shear_wave`` / ``taylor_green``: single-phase decaying flows.
* ``perturbed``: a smooth random density / velocity field for one-step parity tests.
"""
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


def constants():
    """Coexistence constants written by workloads/make_constants.py (which calls only the oracle)."""
    with open(os.path.join(_HERE, "constants.json")) as fh:
        return json.load(fh)


def _grid(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def tanh_profile(r, R, rho_l, rho_v, W):
    """Liquid inside r < R, vapour outside, tanh interface of width W (form of Eq. e23)."""
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - R) / W)


def droplet(shape, R, rho_l, rho_v, W=2.0, center=None, periodic=True):
    nx, ny, nz = shape
    c = center if center is not None else (nx / 2.0, ny / 2.0, nz / 2.0)
    d = []
    for k, n in enumerate((nx, ny, nz)):
        dk = np.arange(n, dtype=np.float64) - c[k]
        if periodic:
            dk = dk - n * np.round(dk / n)
        d.append(dk)
    r = np.sqrt(d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2)
    rho = tanh_profile(r, R, rho_l, rho_v, W)
    return rho, np.zeros((3,) + rho.shape)


def cylinder_droplet(shape, R, rho_l, rho_v, W=2.0):
    """A liquid column along z (cross-section a disc of radius R): quasi-2D Laplace test."""
    nx, ny, nz = shape
    x, y, _ = _grid(shape)
    r = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2)
    rho = tanh_profile(r, R, rho_l, rho_v, W)
    return rho, np.zeros((3,) + rho.shape)


def slab(shape, width, rho_l, rho_v, W=2.0):
    """A liquid slab normal to x of the given width, centred (planar interfaces)."""
    nx, ny, nz = shape
    x, _, _ = _grid(shape)
    r = np.abs(x - nx / 2.0 + 0.5)
    rho = tanh_profile(r, width / 2.0, rho_l, rho_v, W)
    return rho, np.zeros((3,) + rho.shape)


def random_spheres(shape, rho_l, rho_v, r_min, r_max, seed=2306, target_fraction=0.10, gap=4.0,
                   max_rejections=200, W=2.0):
    """Non-overlapping spheres (periodic distance, surfaces at least `gap` apart), radii
    uniform in [r_min, r_max], added until the liquid volume fraction reaches
    `target_fraction` or `max_rejections` consecutive draws fail.  Returns (rho, u, spheres)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    spheres = []
    vol = 0.0
    total = float(nx * ny * nz)
    fails = 0
    L = np.array([nx, ny, nz], dtype=np.float64)
    while vol / total < target_fraction and fails < max_rejections:
        r = rng.uniform(r_min, r_max)
        c = rng.uniform(0.0, 1.0, 3) * L
        ok = True
        for (c2, r2) in spheres:
            d = c - c2
            d -= L * np.round(d / L)
            if np.sqrt((d * d).sum()) < r + r2 + gap:
                ok = False
                break
        if ok and 2 * r + gap > L.min():
            ok = False
        if not ok:
            fails += 1
            continue
        fails = 0
        spheres.append((c, r))
        vol += 4.0 / 3.0 * np.pi * r ** 3
    rho = np.full((nz, ny, nx), rho_v, dtype=np.float64)
    for (c, r) in spheres:
        # only the periodic bounding box of the sphere (plus the interface tail) is touched
        h = int(np.ceil(r + 4.0 * W))
        axes = []
        for k, n in enumerate((nx, ny, nz)):
            lo = int(np.floor(c[k])) - h
            idx = np.arange(lo, lo + 2 * h + 2)
            d = idx - c[k]
            if len(idx) >= n:      # box covers the whole axis: use the periodic minimum image
                idx = np.arange(n)
                d = idx - c[k]
                d = d - n * np.round(d / n)
            axes.append((idx % n, d))
        (ix, dx), (iy, dy), (iz, dz) = axes
        dist = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2)
        sub = rho[np.ix_(iz, iy, ix)]
        rho[np.ix_(iz, iy, ix)] = np.maximum(sub, tanh_profile(dist, r, rho_l, rho_v, W))
    return rho, np.zeros((3,) + rho.shape), [(tuple(float(v) for v in c), float(r)) for c, r in spheres]


def impact(shape, R, rho_l, rho_v, U, gap=3.0, W=2.0):
    """Droplet of radius R centred above the bottom wall (z = -1/2) with its surface `gap`
    cells above it, moving with velocity (0, 0, -U) inside the droplet."""
    nx, ny, nz = shape
    center = (nx / 2.0, ny / 2.0, R + gap)
    rho, u = droplet(shape, R, rho_l, rho_v, W=W, center=center, periodic=False)
    frac = np.clip((rho - rho_v) / (rho_l - rho_v), 0.0, 1.0)
    u[2] = -U * frac
    return rho, u


def cylinder_mask(shape, radius, axis="y", base=0.0):
    """uint8 mask of a solid cylinder with its axis along `axis` resting on the bottom wall
    (axis height base + radius above z = -1/2)."""
    nx, ny, nz = shape
    x, y, z = _grid(shape)
    zc = base + radius - 0.5
    if axis == "y":
        r = np.sqrt((x - nx / 2.0 + 0.5) ** 2 + (z - zc) ** 2)
    else:
        r = np.sqrt((y - ny / 2.0 + 0.5) ** 2 + (z - zc) ** 2)
    return (r <= radius).astype(np.uint8)


def random_mask(shape, fraction, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    return (rng.uniform(size=(nz, ny, nx)) < fraction).astype(np.uint8)


def shear_wave(shape, U, rho0=1.0, mode=1):
    """u_x = U sin(2 pi mode z / nz), uniform density."""
    nx, ny, nz = shape
    _, _, z = _grid(shape)
    u = np.zeros((3, nz, ny, nx))
    u[0] = U * np.sin(2.0 * np.pi * mode * z / nz)
    return np.full((nz, ny, nx), rho0), u


def taylor_green(shape, U, rho0=1.0):
    """2D Taylor-Green vortex in the x-y plane, uniform along z."""
    nx, ny, nz = shape
    x, y, _ = _grid(shape)
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    u = np.zeros((3, nz, ny, nx))
    u[0] = U * np.sin(kx * x) * np.cos(ky * y)
    u[1] = -U * (kx / ky) * np.cos(kx * x) * np.sin(ky * y)
    return np.full((nz, ny, nx), rho0), u


def perturbed(shape, seed, rho0=1.0, drho=0.05, U=0.05, modes=3):
    """Smooth random density and velocity: a few random Fourier modes per field."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    x, y, z = _grid(shape)

    def field(amp):
        out = np.zeros((nz, ny, nx))
        for _ in range(modes):
            k = rng.integers(1, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi, 3)
            a = rng.uniform(-amp, amp)
            out += a * np.sin(2 * np.pi * k[0] * x / nx + ph[0]) * np.sin(2 * np.pi * k[1] * y / ny + ph[1]) \
                * np.sin(2 * np.pi * k[2] * z / nz + ph[2])
        return out

    rho = rho0 + field(drho)
    u = np.stack([field(U), field(U), field(U)])
    return rho, u


def cylinder_impact(shape, R0, Rc, rho_l, rho_v, U, gap=3.0, W=2.0):
    """Sec. IV B: a cylinder of radius Rc lying on the bottom wall along y (axis at height
    Rc - 1/2), and above its crest a droplet of radius R0 whose surface is `gap` cells higher,
    centred over the axis and moving with (0, 0, -U).  Returns (rho, u, solid); solid cells
    carry rho = rho_v (ignored by both implementations)."""
    nx, ny, nz = shape
    solid = cylinder_mask(shape, Rc, axis="y")
    zc = 2.0 * Rc - 0.5 + gap + R0
    rho, u = droplet(shape, R0, rho_l, rho_v, W=W, center=(nx / 2.0 - 0.5, ny / 2.0, zc), periodic=False)
    frac = np.clip((rho - rho_v) / (rho_l - rho_v), 0.0, 1.0)
    u[2] = -U * frac
    rho = np.where(solid == 1, rho_v, rho)
    u[:, solid == 1] = 0.0
    return rho, u, solid


def serving_jobs(n_jobs, rate, seed=2306, edge=(64, 160), impact_fraction=0.5):
    """A request stream: `n_jobs` jobs with Poisson arrivals of `rate` per second (exponential
    gaps drawn from numpy seed `seed` + 1, so the jobs, drawn from `seed`, are the same at any
    rate).  Each job is a dict: name, kind ("impact" or "droplet"), lattice
    (19 or 27 by a fair coin), edge L ~ U{edge}, and for impacts the cylinder-to-droplet ratio
    R/R0 ~ U[0.2, 2] with R0 = L / 6 (Sec. IV B), the domain height raised to fit cylinder and
    droplet; for static droplets a radius ~ U[L/8, L/4] (a parameter sweep).  Only sizes and
    draws: the physical parameters are chosen by the caller."""
    rng = np.random.default_rng(seed)
    arrivals = np.random.default_rng(seed + 1)        # separate stream: same jobs at any rate
    t = 0.0
    jobs = []
    for k in range(n_jobs):
        t += float(arrivals.exponential(1.0 / rate)) if rate > 0 else 0.0
        L = int(rng.integers(edge[0], edge[1] + 1))
        Q = 19 if rng.random() < 0.5 else 27
        if rng.random() < impact_fraction:
            R0 = L / 6.0
            ratio = float(rng.uniform(0.2, 2.0))
            Rc = ratio * R0
            nz = max(int(round(5 * R0)), int(np.ceil(2 * Rc + 2 * R0 + 3 + R0)))
            jobs.append(dict(name=f"impact{k}", kind="impact", lattice=Q, shape=(L, L, nz), R0=R0, Rc=Rc,
                             arrival=t))
        else:
            R = float(rng.uniform(L / 8.0, L / 4.0))
            jobs.append(dict(name=f"droplet{k}", kind="droplet", lattice=Q, shape=(L, L, L), R=R, arrival=t))
    return jobs
