"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds geometry and random-input generators only: no lattice-Boltzmann
arithmetic lives here. Node types follow the paper's classification of nodes into
solid, fluid and boundary nodes (Sec. 3.1, the ``allNodeType`` array); the boundary
kinds are the velocity inlet and the constant-pressure outlet of Sec. 2.2.

Encoding (uint8, one byte per node, dense array indexed ``[z, y, x]`` so that x is
fastest in memory, the row order of Sec. 3.2):

    SOLID = 0, FLUID = 1, INLET = 2, OUTLET = 3

Every generator is deterministic for a given seed (numpy PCG64 stream).
"""
from __future__ import annotations

import math

import numpy as np

SOLID = 0
FLUID = 1
INLET = 2
OUTLET = 3

# Well-known seeds of the synthetic workloads.
SEED_POROUS_256 = 161102445
SEED_VESSEL = 161102446
SEED_POROUS_512 = 161102447
SEED_POROUS_128 = 161102448
SEED_FORCE_NOISE = 161102449

# The three D3Q19 weight classes (rest, axis links, diagonal links) of Sec. 2.2,
# used only to draw plausible random populations for tests.
_WEIGHT_CLASS = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def poiseuille_channel(nx: int = 32, ny: int = 32, nz: int = 32) -> np.ndarray:
    """Plane channel: the planes y = 0 and y = ny-1 are solid walls, the rest fluid."""
    nt = np.full((nz, ny, nx), FLUID, dtype=np.uint8)
    nt[:, 0, :] = SOLID
    nt[:, ny - 1, :] = SOLID
    return nt


def dense_box(nx: int, ny: int, nz: int) -> np.ndarray:
    """All-fluid box (the dense cavity3D shape of Sec. 4.3, without a lid)."""
    return np.full((nz, ny, nx), FLUID, dtype=np.uint8)


def sphere_pack(n: int, radius: float = 8.0, porosity: float = 0.35,
                seed: int = SEED_POROUS_256, ny: int | None = None,
                nz: int | None = None) -> np.ndarray:
    """Periodic pack of overlapping solid spheres (the random-spheres geometry of Sec. 4.6).

    Centres are drawn uniformly in [0, n)^3 one at a time; a node is solid when its
    periodic (minimum-image) squared distance to a centre is <= radius^2. Spheres are
    added until the porosity (non-solid nodes / all nodes) first drops to ``porosity``
    or below.
    """
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    nt = np.full((nz, ny, nx), FLUID, dtype=np.uint8)
    flat = nt.reshape(-1)
    total = nx * ny * nz
    solid = 0
    r = float(radius)
    r2 = r * r
    ext = int(math.ceil(r)) + 1
    off = np.arange(-ext, ext + 1)
    while solid / total < 1.0 - porosity:
        c = rng.random(3) * np.array([nx, ny, nz])
        bx = np.floor(c[0]) + off
        by = np.floor(c[1]) + off
        bz = np.floor(c[2]) + off
        dx2 = (bx - c[0]) ** 2
        dy2 = (by - c[1]) ** 2
        dz2 = (bz - c[2]) ** 2
        d2 = dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :]
        kz, ky, kx = np.nonzero(d2 <= r2)
        ix = (bx[kx].astype(np.int64)) % nx
        iy = (by[ky].astype(np.int64)) % ny
        iz = (bz[kz].astype(np.int64)) % nz
        idx = ix + nx * (iy + ny * iz)
        idx = np.unique(idx)
        solid += int(np.count_nonzero(flat[idx] != SOLID))
        flat[idx] = SOLID
    return nt


def _capsule_mask(shape, p0, p1, r):
    """Boolean mask of nodes within distance r of segment p0-p1, with its bounding box."""
    nz, ny, nx = shape
    lo = np.maximum(np.floor(np.minimum(p0, p1) - r - 1).astype(int), 0)
    hi = np.minimum(np.ceil(np.maximum(p0, p1) + r + 1).astype(int), [nx - 1, ny - 1, nz - 1])
    if np.any(hi < lo):
        return None
    xs = np.arange(lo[0], hi[0] + 1, dtype=np.float64)
    ys = np.arange(lo[1], hi[1] + 1, dtype=np.float64)
    zs = np.arange(lo[2], hi[2] + 1, dtype=np.float64)
    d = p1 - p0
    L2 = float(d @ d)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    px, py, pz = X - p0[0], Y - p0[1], Z - p0[2]
    t = (px * d[0] + py * d[1] + pz * d[2]) / L2
    tc = np.clip(t, 0.0, 1.0)
    qx, qy, qz = px - tc * d[0], py - tc * d[1], pz - tc * d[2]
    inside = qx * qx + qy * qy + qz * qz <= r * r
    return lo, hi, inside, t


def vessel_tree(nx: int = 1024, ny: int = 512, nz: int = 512, seed: int = SEED_VESSEL,
                root_radius: float = 24.0, ratio: float = 0.79, generations: int = 6,
                length_factor: float = 10.0, angle_deg=(25.0, 45.0)) -> np.ndarray:
    """Seeded binary tree of capsules standing in for a sparse vessel geometry.

    The root starts at the centre of the x = 0 face and runs along +x. Each segment of
    generation k has radius r_k = root_radius * ratio**k and length length_factor * r_k.
    A child's direction is its parent's rotated by theta ~ U[angle_deg] about a random
    axis perpendicular to the parent; siblings take opposite azimuths. Nodes within r of
    a segment are fluid. Fluid nodes of the x = 0 plane are INLET; fluid nodes of a leaf
    whose axial coordinate exceeds (length - 1) and fluid nodes on the other five box
    faces are OUTLET.
    """
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    nt = np.full(shape, SOLID, dtype=np.uint8)
    leaf_tips = []
    segs = []
    start = np.array([0.0, ny / 2.0, nz / 2.0])
    frontier = [(start, np.array([1.0, 0.0, 0.0]), 0)]
    while frontier:
        p0, d, k = frontier.pop(0)
        r = root_radius * ratio ** k
        L = length_factor * r
        p1 = p0 + L * d
        segs.append((p0, p1, r))
        if k + 1 < generations:
            a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
            e1 = np.cross(d, a)
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(d, e1)
            phi = rng.random() * 2.0 * math.pi
            for sgn in (1.0, -1.0):
                th = math.radians(angle_deg[0] + (angle_deg[1] - angle_deg[0]) * rng.random())
                e = sgn * (math.cos(phi) * e1 + math.sin(phi) * e2)
                cd = math.cos(th) * d + math.sin(th) * e
                cd /= np.linalg.norm(cd)
                frontier.append((p1, cd, k + 1))
        else:
            leaf_tips.append((p0, p1, r, L))
    for p0, p1, r in segs:
        m = _capsule_mask(shape, p0, p1, r)
        if m is None:
            continue
        lo, hi, inside, _ = m
        sub = nt[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        sub[inside] = FLUID
    for p0, p1, r, L in leaf_tips:
        m = _capsule_mask(shape, p0, p1, r)
        if m is None:
            continue
        lo, hi, inside, t = m
        sub = nt[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1]
        tip = inside & (t * L > L - 1.0) & (sub != SOLID)
        sub[tip] = OUTLET
    for sl in ((slice(None), slice(None), nx - 1), (slice(None), 0, slice(None)),
               (slice(None), ny - 1, slice(None)), (0, slice(None), slice(None)),
               (nz - 1, slice(None), slice(None))):
        face = nt[sl]
        face[face != SOLID] = OUTLET
    face = nt[:, :, 0]
    face[face != SOLID] = INLET
    return nt


def random_box(nx: int, ny: int, nz: int, p_solid: float = 0.25, seed: int = 0,
               boundary: bool = False) -> np.ndarray:
    """Random node types for small parity cases; optional random INLET/OUTLET nodes."""
    rng = np.random.default_rng(seed)
    u = rng.random((nz, ny, nx))
    nt = np.where(u < p_solid, SOLID, FLUID).astype(np.uint8)
    if boundary:
        v = rng.random((nz, ny, nx))
        nt[(nt == FLUID) & (v < 0.05)] = INLET
        nt[(nt == FLUID) & (v > 0.95)] = OUTLET
    return nt


def crop(nt: np.ndarray, n: int) -> np.ndarray:
    """Sub-box [0, n)^3 of a geometry, run as a problem of its own."""
    return np.ascontiguousarray(nt[:n, :n, :n])


def random_populations(nt: np.ndarray, amplitude: float = 0.05, seed: int = 1) -> np.ndarray:
    """Random positive populations near the D3Q19 weights, dense ``[19, nz, ny, nx]``
    float64; solid nodes hold NaN."""
    rng = np.random.default_rng(seed)
    f = _WEIGHT_CLASS[:, None, None, None] * (
        1.0 + amplitude * (2.0 * rng.random((19,) + nt.shape) - 1.0))
    f[:, nt == SOLID] = np.nan
    return f


def body_force_field(nt: np.ndarray, mean: float = 1e-5, std: float = 1e-7,
                     seed: int = SEED_FORCE_NOISE) -> np.ndarray:
    """Per-node x body force g(x) = mean + N(0, std^2), dense ``[nz, ny, nx]`` float64."""
    rng = np.random.default_rng(seed)
    return mean + std * rng.standard_normal(nt.shape)


def random_directions(shape, count: int, seed: int) -> np.ndarray:
    """``count`` seeded standard-normal direction fields of the given shape."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((count,) + tuple(shape))
