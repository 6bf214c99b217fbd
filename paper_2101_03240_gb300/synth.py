"""Seeded synthetic pore images and workload descriptions.

This module only *builds inputs*: voxel images (uint8, nonzero = pore,
0 = solid), request streams and parameter lists.  It holds none of the
invasion method's arithmetic (no distance transform, no invasion, no
trapping, no pressure or saturation computation), so both the CPU oracle and
the CUDA path may consume what it produces.

Image conventions: shape (nx, ny, nz), C order, linear index
idx = (x*ny + y)*nz + z.

The workloads stand in for the paper's images, which are not available:
  * blobs: uniform noise smoothed by a Gaussian and thresholded at a porosity
    quantile, the "artificially generated blobs" of the paper's 3D example
    (Fig. 4, 250^3 at 60 % porosity);
  * sphere packs: overlapping solid spheres dropped uniformly at random until
    the porosity falls to a target.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


# ----------------------------------------------------------------------------
# image recipes
# ----------------------------------------------------------------------------

def blobs(shape, sigma, porosity, rng) -> np.ndarray:
    """Gaussian-filtered uniform noise thresholded so that `porosity` of the
    voxels are pore.  `sigma` is a scalar or a per-axis tuple (voxels); the
    filter wraps at the borders."""
    from scipy.ndimage import gaussian_filter

    shape = tuple(int(s) for s in shape)
    noise = rng.random(shape, dtype=np.float32)
    f = gaussian_filter(noise, sigma=sigma, mode="wrap")
    n = f.size
    k = int(round(porosity * n))
    if k <= 0:
        return np.zeros(shape, np.uint8)
    if k >= n:
        return np.ones(shape, np.uint8)
    thr = np.partition(f.ravel(), k - 1)[k - 1]
    return (f <= thr).astype(np.uint8)


def sphere_pack(shape, radius, porosity, rng) -> np.ndarray:
    """Overlapping solid spheres of a given radius (voxels), centres uniform
    and continuous over the box; voxel v is solid iff |v - c|^2 <= radius^2.
    Spheres are added until the porosity is <= `porosity` (the sphere that
    crosses the target is kept)."""
    shape = tuple(int(s) for s in shape)
    solid = np.zeros(shape, bool)
    n = solid.size
    n_solid = 0
    r = float(radius)
    r2 = r * r
    hi = np.array(shape, float)
    while 1.0 - n_solid / n > porosity:
        c = rng.uniform(0.0, 1.0, 3) * hi
        lo_i = np.maximum(np.floor(c - r).astype(int), 0)
        hi_i = np.minimum(np.ceil(c + r).astype(int) + 1, shape)
        if np.any(hi_i <= lo_i):
            continue
        xs = np.arange(lo_i[0], hi_i[0])[:, None, None]
        ys = np.arange(lo_i[1], hi_i[1])[None, :, None]
        zs = np.arange(lo_i[2], hi_i[2])[None, None, :]
        m = (xs - c[0]) ** 2 + (ys - c[1]) ** 2 + (zs - c[2]) ** 2 <= r2
        box = solid[lo_i[0]:hi_i[0], lo_i[1]:hi_i[1], lo_i[2]:hi_i[2]]
        n_solid += int(np.count_nonzero(m & ~box))
        box |= m
    return (~solid).astype(np.uint8)


def random_image(shape, porosity, rng) -> np.ndarray:
    """Independent Bernoulli voxels: pore with probability `porosity`."""
    return (rng.random(tuple(shape)) < porosity).astype(np.uint8)


def tube(nx, radius, pad=1) -> np.ndarray:
    """Straight cylindrical tube along x: pore iff (y-cy)^2 + (z-cz)^2 < R^2
    with integer R, a cross-section of side 2R+1+2*pad centred on (cy, cz).
    With pad >= 1 solid lies on every side of the tube in y and z."""
    R = int(radius)
    n = 2 * R + 1 + 2 * int(pad)
    c = n // 2
    y = np.arange(n)[:, None]
    z = np.arange(n)[None, :]
    disk = (y - c) ** 2 + (z - c) ** 2 < R * R
    return np.broadcast_to(disk, (int(nx), n, n)).astype(np.uint8)


def throat_pore(r_throat, r_pore, l_throat, pad=2) -> np.ndarray:
    """Inlet throat (cylinder along x, radius r_throat, length l_throat), a
    spherical pore of radius r_pore, and an outlet throat of the same radius
    and length.  Pore iff inside the cylinder or the sphere (strict <)."""
    rt, rp, lt = int(r_throat), int(r_pore), int(l_throat)
    nx = 2 * lt + 2 * rp + 1
    n = 2 * rp + 1 + 2 * int(pad)
    c = n // 2
    x = np.arange(nx)[:, None, None]
    y = np.arange(n)[None, :, None]
    z = np.arange(n)[None, None, :]
    cx = lt + rp
    cyl = ((y - c) ** 2 + (z - c) ** 2 < rt * rt) & np.ones((nx, 1, 1), bool)
    sph = (x - cx) ** 2 + (y - c) ** 2 + (z - c) ** 2 < rp * rp
    return (cyl | sph).astype(np.uint8)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    image: np.ndarray
    inlet: int          # face id: 0=X0 1=X1 2=Y0 3=Y1 4=Z0 5=Z1
    outlet: int | None  # None = no trapping
    mio_levels: int = 0
    voxel_m: float = 5e-6
    sigma: float = 0.072
    theta_deg: float = 180.0


def c1_blobs48(seed=1) -> Workload:
    """48^3 blobs: noise smoothed with sigma=3 (wrap), porosity 0.65,
    inlet x=0, no trapping."""
    rng = np.random.default_rng(seed)
    return Workload("blobs48", blobs((48, 48, 48), 3.0, 0.65, rng), 0, None)


def c2_spheres200(seed=2) -> Workload:
    """200^3 overlapping solid spheres of radius 8 until porosity 0.40,
    inlet x=0, outlet x=199, trapping and Pc curve (voxel 5 um,
    sigma 0.072 N/m, theta 180 deg)."""
    rng = np.random.default_rng(seed)
    return Workload("spheres200", sphere_pack((200, 200, 200), 8, 0.40, rng), 0, 1)


def c3_blobs512(seed=3) -> Workload:
    """512^3 anisotropic blobs (sigma=(4,8,4)), porosity 0.60, inlet x=0,
    outlet x=511, trapping, and morphological-opening drainage at 40 radii."""
    rng = np.random.default_rng(seed)
    return Workload("blobs512", blobs((512, 512, 512), (4.0, 8.0, 4.0), 0.60, rng),
                    0, 1, mio_levels=40)


def c3_blobs256(seed=3) -> Workload:
    """The 512^3 blob recipe at 256^3 (sigma=(4,8,4), porosity 0.60, inlet
    x=0, outlet x=255, 40 radii): a smaller case of the same workload for
    profiler captures."""
    rng = np.random.default_rng(seed)
    return Workload("blobs256", blobs((256, 256, 256), (4.0, 8.0, 4.0), 0.60, rng), 0, 1, mio_levels=40)


def mixed_edge(i, seed_base, lo, hi):
    """Edge length of mixed_image(i, seed_base, lo, hi) without building it."""
    rng = np.random.default_rng(seed_base + i)
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def mixed_image(i, seed_base, lo, hi):
    """Image `i` of a mixed batch: edge log-uniform in [lo, hi]; even i are
    blobs (sigma U(2,6), porosity U(0.5,0.7)), odd i are sphere packs
    (radius U{4..10}, porosity U(0.35,0.5))."""
    rng = np.random.default_rng(seed_base + i)
    L = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
    if i % 2 == 0:
        s = rng.uniform(2.0, 6.0)
        p = rng.uniform(0.5, 0.7)
        return blobs((L, L, L), s, p, rng)
    r = int(rng.integers(4, 11))
    p = rng.uniform(0.35, 0.5)
    return sphere_pack((L, L, L), r, p, rng)


def c4_batch(n=256, seed=4, lo=32, hi=160):
    """Batch of `n` uneven cubes (image i seeded with 1000*seed + i)."""
    return [mixed_image(i, 1000 * seed, lo, hi) for i in range(n)]


def c5_requests(n=600, rate=20.0, seed=5, lo=64, hi=384):
    """Poisson request stream: (arrival_s, edge, kind, param seed) tuples.
    The images themselves are built lazily with `mixed_image`."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    out = []
    for j in range(n):
        r = np.random.default_rng(1000 * seed + j)
        L = int(round(math.exp(r.uniform(math.log(lo), math.log(hi)))))
        out.append((float(t[j]), L, j % 2))
    return out


def mio_levels(max_dt2: int, n_levels: int = 40) -> list[int]:
    """Squared radii of the opening levels: T_i = max(1, round(max_dt2 *
    ((n-i)/n)^2)) for i = 0..n-1 (round half up), deduplicated and strictly
    descending.  `max_dt2` is the largest squared distance in the image."""
    out = []
    for i in range(n_levels):
        t = max(1, int(math.floor(max_dt2 * ((n_levels - i) / n_levels) ** 2 + 0.5)))
        if not out or t < out[-1]:
            out.append(t)
    return out


def integer_radius_levels(max_dt2: int) -> tuple[list[int], list[int]]:
    """Opening levels with the structuring element of the paper-literal
    invasion (integer radius R, ball |d|^2 <= R^2): for R = floor(sqrt(
    max_dt2)) down to 1, erosion bound R^2 and dilation bound R^2 + 1
    (|d|^2 <= R^2 is |d|^2 < R^2 + 1 for integer d)."""
    R = math.isqrt(max(int(max_dt2), 1))
    return [r * r for r in range(R, 0, -1)], [r * r + 1 for r in range(R, 0, -1)]


FACES = {"x0": 0, "x1": 1, "y0": 2, "y1": 3, "z0": 4, "z1": 5}
