"""Seeded synthetic inputs for the D2Q9 solver: geometries and initial fields.

This module holds no lattice-Boltzmann arithmetic.  It only draws geometries
(solid masks) and macroscopic fields (density, velocity, force, targets) that
the CUDA library and the FP64 CPU oracle both take as input.  It imports
neither of them.

Stand-ins for the paper's workloads (the paper's own geometry files and
figure data are not available):
  * lid-driven cavity (Sec. 4.1.1): all-fluid square, walls on every side,
    north wall moving;
  * porous media (Sec. 4.2.2, "sparse geometries"): random discs, radius drawn
    uniformly, centres uniform, periodic in x;
  * channel with cylinders: seeded non-overlapping discs in a channel;
  * Taylor-Green vortex and body-force Poiseuille initial fields.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so every geometry is fixed by
its seed on every machine.
"""
from __future__ import annotations

import math

import numpy as np

GEOMETRY_SEED = 13241
TARGET_SEED = 2108
FD_SEED = 7

_M64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, golden-gamma increment)."""

    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform double in [lo, hi) from the top 53 bits."""
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def integers(self, n: int, count: int) -> np.ndarray:
        """count integers uniform in [0, n) (modulo reduction, n << 2^64)."""
        return np.array([self.next_u64() % n for _ in range(count)], dtype=np.int64)


def _stamp_disc(solid: np.ndarray, cx: float, cy: float, r: float, periodic_x: bool) -> int:
    """Mark nodes (i, j) with (i - cx)^2 + (j - cy)^2 <= r^2; x wraps if periodic,
    y is clipped.  Returns the number of nodes that turned solid."""
    ny, nx = solid.shape
    j0, j1 = max(0, math.ceil(cy - r)), min(ny - 1, math.floor(cy + r))
    i0, i1 = math.ceil(cx - r), math.floor(cx + r)
    if j0 > j1 or i1 < i0:
        return 0
    jj = np.arange(j0, j1 + 1)[:, None]
    ii = np.arange(i0, i1 + 1)[None, :]
    inside = (ii - cx) ** 2 + (jj - cy) ** 2 <= r * r
    if periodic_x:
        cols = np.mod(ii[0], nx)
    else:
        keep = (ii[0] >= 0) & (ii[0] < nx)
        inside = inside[:, keep]
        cols = ii[0][keep]
    rows = jj[:, 0]
    # a disc wider than the domain may wrap onto itself: handle column by column
    before = int(solid.sum()) if periodic_x and (i1 - i0 + 1) > nx else None
    if before is not None:
        for k, c in enumerate(cols):
            solid[rows[inside[:, k]], c] = 1
        return int(solid.sum()) - before
    sub = solid[rows[0]:rows[-1] + 1][:, cols]
    new = int(np.count_nonzero(inside & (sub == 0)))
    sub |= inside.astype(np.uint8)
    solid[rows[0]:rows[-1] + 1, cols] = sub
    return new


def porous_discs(nx: int, ny: int, porosity: float, rmin: float = 8.0, rmax: float = 32.0,
                 seed: int = GEOMETRY_SEED, periodic_x: bool = True,
                 max_rejections: int = 1_000):
    """Random-disc porous medium with porosity phi = fluid nodes / all nodes.

    Radii are uniform reals in [rmin, rmax]; centres uniform reals over the
    domain.  Phase 1 adds non-overlapping discs (centre distance >= r1 + r2,
    x distance periodic) until the solid fraction reaches 1 - phi or
    `max_rejections` candidates in a row overlap; phase 2 then adds discs that
    may overlap until the solid fraction reaches 1 - phi.  The last disc may
    overshoot the target by at most one disc area.

    Returns (solid uint8[ny, nx], achieved porosity, number of discs).
    """
    rng = SplitMix64(seed)
    solid = np.zeros((ny, nx), np.uint8)
    target = int(round((1.0 - porosity) * nx * ny))
    nsolid = 0
    cell = 2.0 * rmax
    gx, gy = max(1, int(nx // cell)), max(1, int(ny // cell))
    grid: dict = {}
    discs = []

    def cell_of(x, y):
        return int(x * gx / nx) % gx, min(gy - 1, int(y * gy / ny))

    def overlaps(x, y, r):
        ci, cj = cell_of(x, y)
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                cj2 = cj + dj
                if cj2 < 0 or cj2 >= gy:
                    continue
                ci2 = (ci + di) % gx if periodic_x else ci + di
                if ci2 < 0 or ci2 >= gx:
                    continue
                for (x2, y2, r2) in grid.get((ci2, cj2), ()):
                    dx = abs(x - x2)
                    if periodic_x:
                        dx = min(dx, nx - dx)
                    if dx * dx + (y - y2) ** 2 < (r + r2) ** 2:
                        return True
        return False

    rejections = 0
    while nsolid < target and rejections < max_rejections:
        r = rng.uniform(rmin, rmax)
        x = rng.uniform(0.0, nx)
        y = rng.uniform(0.0, ny)
        if overlaps(x, y, r):
            rejections += 1
            continue
        rejections = 0
        grid.setdefault(cell_of(x, y), []).append((x, y, r))
        discs.append((x, y, r))
        nsolid += _stamp_disc(solid, x, y, r, periodic_x)
    while nsolid < target:
        r = rng.uniform(rmin, rmax)
        x = rng.uniform(0.0, nx)
        y = rng.uniform(0.0, ny)
        discs.append((x, y, r))
        nsolid += _stamp_disc(solid, x, y, r, periodic_x)
    return solid, 1.0 - nsolid / float(nx * ny), len(discs)


def circle_array(nx: int, ny: int, porosity: float, m: int = 8):
    """Regular m x m array of equal solid discs (Sec. 4.2.2's regular
    arrangement): centres at ((k + 1/2) nx/m, (l + 1/2) ny/m), membership
    (i - cx)^2 + (j - cy)^2 <= r^2 on the integer grid, r the smallest radius
    (found by bisection on the node count) whose solid fraction reaches
    1 - porosity.  Discs do not touch for porosity > 1 - pi/4 on a square
    grid; lower porosities are rejected, as the paper leaves them out.

    Returns (solid uint8[ny, nx], achieved porosity, r)."""
    sx, sy = nx / m, ny / m
    if porosity <= 1.0 - math.pi / 4.0 * min(sx, sy) ** 2 / (sx * sy) or porosity >= 1.0:
        raise ValueError("porosity out of range for a non-touching %dx%d array" % (m, m))
    target = int(round((1.0 - porosity) * nx * ny))
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    # distance^2 of every node to the centre of its own cell
    dx = x - (np.floor(x / sx) + 0.5) * sx
    dy = y - (np.floor(y / sy) + 0.5) * sy
    d2 = dx * dx + dy * dy
    vals = np.sort(d2.ravel())
    r2 = vals[target - 1] if target > 0 else -1.0
    solid = (d2 <= r2).astype(np.uint8)
    return solid, 1.0 - int(solid.sum()) / float(nx * ny), math.sqrt(max(r2, 0.0))


def channel_cylinders(nx: int, ny: int, count: int = 12, rmin: float = 6.0, rmax: float = 12.0,
                      clearance: float = 2.0, seed: int = GEOMETRY_SEED):
    """`count` non-overlapping discs in a channel periodic in x, walls in y.

    Each disc keeps `clearance` free nodes to the y walls and to every other
    disc.  Returns (solid uint8[ny, nx], list of (cx, cy, r)).
    """
    rng = SplitMix64(seed)
    solid = np.zeros((ny, nx), np.uint8)
    discs = []
    tries = 0
    while len(discs) < count:
        tries += 1
        if tries > 1_000_000:
            raise RuntimeError("cannot place the cylinders")
        r = rng.uniform(rmin, rmax)
        x = rng.uniform(0.0, nx)
        y = rng.uniform(r + clearance, ny - 1 - r - clearance)
        ok = True
        for (x2, y2, r2) in discs:
            dx = abs(x - x2)
            dx = min(dx, nx - dx)
            if dx * dx + (y - y2) ** 2 < (r + r2 + clearance) ** 2:
                ok = False
                break
        if ok:
            discs.append((x, y, r))
            _stamp_disc(solid, x, y, r, True)
    return solid, discs


def random_solid(nx: int, ny: int, fraction: float, seed: int) -> np.ndarray:
    """Independent random solid nodes (for tables and edge cases on tiny grids)."""
    rng = SplitMix64(seed)
    vals = np.array([rng.next_u64() >> 11 for _ in range(nx * ny)], dtype=np.float64)
    return (vals * (1.0 / (1 << 53)) < fraction).astype(np.uint8).reshape(ny, nx)


def taylor_green(nx: int, ny: int, U: float):
    """Taylor-Green vortex at t = 0 on node coordinates x = i, y = j:
    u_x = -U cos(kx x) sin(ky y), u_y = U (kx/ky) sin(kx x) cos(ky y) (kx = ky
    for a square box), rho = 1 - (3 U^2 / 4) (cos 2 kx x + cos 2 ky y).
    Returns (rho [ny, nx], u [2, ny, nx])."""
    kx, ky = 2 * math.pi / nx, 2 * math.pi / ny
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    ux = -U * np.cos(kx * x) * np.sin(ky * y)
    uy = U * (kx / ky) * np.sin(kx * x) * np.cos(ky * y)
    rho = 1.0 - 0.75 * U * U * (np.cos(2 * kx * x) + np.cos(2 * ky * y) * (kx / ky) ** 2)
    return rho, np.stack([ux, uy])


def poiseuille(nx: int, ny: int, tau: float, u_max: float):
    """Body-force Poiseuille channel (periodic x, half-way walls at y = -1/2 and
    ny - 1/2): force density F_x = 8 nu u_max / ny^2 and the parabola
    u_x(y) = F_x/(2 nu) (y + 1/2)(ny - 1/2 - y), rho = 1.
    Returns (F_x, rho [ny, nx], u [2, ny, nx])."""
    nu = (tau - 0.5) / 3.0
    fx = 8.0 * nu * u_max / (ny * ny)
    y = np.arange(ny, dtype=np.float64)
    prof = fx / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    u = np.zeros((2, ny, nx))
    u[0] = prof[:, None]
    return fx, np.ones((ny, nx)), u


def target_velocity(nx: int, ny: int, solid: np.ndarray, amp: float = 0.02, modes: int = 4,
                    seed: int = TARGET_SEED) -> np.ndarray:
    """Smooth seeded target field u*: amp x a sum of `modes` random Fourier modes,
    zero at solid nodes.  Returns float64 [2, ny, nx]."""
    rng = SplitMix64(seed)
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    u = np.zeros((2, ny, nx))
    for c in range(2):
        for _ in range(modes):
            kx = 1 + int(rng.uniform(0, 4))
            ky = 1 + int(rng.uniform(0, 4))
            ph1, ph2 = rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi)
            u[c] += np.cos(2 * math.pi * kx * x / nx + ph1) * np.sin(math.pi * ky * (y + 0.5) / ny + ph2)
    u *= amp / modes
    u[:, solid.astype(bool)] = 0.0
    return u


def random_field(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform(-scale, scale) float64 field of the given shape (SplitMix64)."""
    rng = SplitMix64(seed)
    n = int(np.prod(shape))
    v = np.array([rng.next_u64() >> 11 for _ in range(n)], dtype=np.float64) * (1.0 / (1 << 53))
    return (2.0 * v - 1.0).reshape(shape) * scale


def random_solid_3d(nx: int, ny: int, nz: int, fraction: float, seed: int) -> np.ndarray:
    """Independent random solid nodes of a three-dimensional box, uint8
    [nz, ny, nx] (SplitMix64; for small parity cases)."""
    rng = SplitMix64(seed)
    vals = np.array([rng.next_u64() >> 11 for _ in range(nx * ny * nz)], dtype=np.float64)
    return (vals * (1.0 / (1 << 53)) < fraction).astype(np.uint8).reshape(nz, ny, nx)


def taylor_green_3d(nx: int, ny: int, nz: int, U: float):
    """Three-dimensional Taylor-Green vortex at t = 0 on node coordinates
    (k = 2 pi / n per axis): u_x = U sin(kx x) cos(ky y) cos(kz z),
    u_y = -U (kx/ky) cos(kx x) sin(ky y) cos(kz z), u_z = 0, and the
    pressure-consistent density rho = 1 + 3 p with
    p = (U^2 / 16) (cos 2 kx x + cos 2 ky y)(cos 2 kz z + 2) (c_s^2 = 1/3).
    Returns (rho [nz, ny, nx], u [3, nz, ny, nx])."""
    kx, ky, kz = 2 * math.pi / nx, 2 * math.pi / ny, 2 * math.pi / nz
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    shape = (nz, ny, nx)
    ux = np.broadcast_to(U * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z), shape)
    uy = np.broadcast_to(-U * (kx / ky) * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z), shape)
    uz = np.zeros(shape)
    p = (U * U / 16.0) * (np.cos(2 * kx * x) + np.cos(2 * ky * y)) * (np.cos(2 * kz * z) + 2.0)
    rho = np.broadcast_to(1.0 + 3.0 * p, shape).copy()
    return rho, np.stack([ux, uy, uz])


def porous_spheres_3d(n: int, porosity: float, rmin: float = 8.0, rmax: float = 16.0,
                      seed: int = GEOMETRY_SEED):
    """Three-dimensional porous medium on a periodic n^3 box: spheres with
    uniform random centres and radii in [rmin, rmax], overlapping, added
    until the solid fraction reaches 1 - porosity; integer-grid membership
    |node - centre|^2 <= r^2 with periodic wrap.  Returns (solid uint8
    [n, n, n] (z, y, x), achieved porosity)."""
    rng = SplitMix64(seed)
    solid = np.zeros((n, n, n), np.uint8)
    target = (1.0 - porosity) * n ** 3
    count = 0
    while count < target:
        c = [rng.uniform(0, n) for _ in range(3)]
        r = rng.uniform(rmin, rmax)
        lo = [int(math.floor(ci - r)) for ci in c]
        hi = [int(math.ceil(ci + r)) + 1 for ci in c]
        zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]),
                                 indexing="ij")
        inside = (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
        idx = (zz[inside] % n, yy[inside] % n, xx[inside] % n)
        before = int(solid[idx].sum())
        solid[idx] = 1
        count += int(solid[idx].sum()) - before
    return solid, 1.0 - count / n ** 3
