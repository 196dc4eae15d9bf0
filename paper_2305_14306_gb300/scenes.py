"""Seeded synthetic point clouds shaped like the paper's workloads.

The paper measures on KITTI, nuScenes, SUN RGB-D, SemanticKITTI and S3DIS
(Section 4.1); none of them is available here, so these generators stand in
for them with the same sizes and structure:

* ``uniform_box``   -- i.i.d. uniform points in the KITTI detection range
  (x in [0, 70.4], y in [-40, 40], z in [-3, 1] m), the 16,384-point input of
  point-based detectors (Section 4.3).
* ``lidar_scene``   -- a spinning LiDAR: rings of rays cast against a ground
  plane and axis-aligned boxes, range noise, per-ray dropout, scan order.
* ``room_scene``    -- an indoor room (floor, ceiling, walls, boxes, panels),
  area-uniform surface points with Gaussian noise, shuffled (S3DIS-like).
* ``lidar_batch``   -- many LiDAR clouds of log-uniform size, each an exact
  seeded subset of a dense scan kept in scan order.
* ``request_stream`` -- Poisson arrivals of scenes of log-uniform size for the
  serving loop.

Nothing here computes any part of the sampler; the module only draws inputs.
Every function is deterministic in its seed (numpy PCG64).
"""
from __future__ import annotations

import math

import numpy as np

KITTI_LO = (0.0, -40.0, -3.0)
KITTI_HI = (70.4, 40.0, 1.0)


def uniform_box(n: int = 16384, seed: int = 0, lo=KITTI_LO, hi=KITTI_HI) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    p = lo + (hi - lo) * rng.random((n, 3))
    return np.ascontiguousarray(p.astype(np.float32))


def _ray_box_hits(o_dirs: np.ndarray, boxes: np.ndarray, az: np.ndarray | None = None) -> np.ndarray:
    """Nearest positive ray parameter against axis-aligned boxes (slab test).

    o_dirs: (R, 3) unit directions from the origin; boxes: (B, 6) min/max.
    Returns (R,) distances, inf where no box is hit.

    az (optional): the rays form a ring-major grid (R = rings x len(az)) whose
    k-th column has azimuth az[k], ascending.  A box whose footprint does not
    hold the origin spans the azimuths of its footprint corners, so only the
    columns inside that range (widened by 1e-6 rad) can hit it; the others are
    skipped.  The test of every ray that is evaluated is the same arithmetic,
    so the result does not depend on the culling.
    """
    R = o_dirs.shape[0]
    best = np.full(R, np.inf)
    cols = None if az is None else az.shape[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / o_dirs
        for b in boxes:
            sel = slice(None)
            if cols is not None and not (b[0] <= 0.0 <= b[3] and b[1] <= 0.0 <= b[4]):
                cx = np.array([b[0], b[3], b[0], b[3]])
                cy = np.array([b[1], b[1], b[4], b[4]])
                ang = np.arctan2(cy, cx)
                if ang.max() - ang.min() < np.pi:  # no wrap through +-pi
                    k0 = int(np.searchsorted(az, ang.min() - 1e-6, side="left"))
                    k1 = int(np.searchsorted(az, ang.max() + 1e-6, side="right"))
                    if k0 >= k1:
                        continue
                    rows = R // cols
                    sel = (np.arange(rows)[:, None] * cols + np.arange(k0, k1)[None, :]).reshape(-1)
            iv = inv[sel]
            t1 = b[:3][None, :] * iv
            t2 = b[3:][None, :] * iv
            tmin = np.nanmax(np.minimum(t1, t2), axis=1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=1)
            hit = (tmax >= 0) & (tmin <= tmax) & (tmin > 0)
            cur = best[sel]
            best[sel] = np.where(hit & (tmin < cur), tmin, cur)
    return best


def lidar_scene(seed: int = 0, rings: int = 64, az_steps: int = 512, fov_deg: float = 90.0,
                elev_deg=(-24.9, 2.0), keep: float = 0.65, n_boxes=(20, 40),
                max_range: float = 80.0, noise: float = 0.01, ground_z: float = -1.73,
                shuffle: bool = False) -> np.ndarray:
    """Spinning-LiDAR scene, sensor at the origin, points in ring-major scan order.

    Defaults give the "kitti-fov" reading: 2,048 steps per revolution over the
    front 90 degrees (512 azimuth steps) x 64 rings, keep-probability 0.65,
    which lands near 16-20k returns.
    """
    rng = np.random.default_rng(seed)
    elev = np.deg2rad(np.linspace(elev_deg[0], elev_deg[1], rings))
    az = np.deg2rad(-fov_deg / 2 + (np.arange(az_steps) + 0.5) * fov_deg / az_steps)
    E, A = np.meshgrid(elev, az, indexing="ij")  # ring-major
    d = np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1).reshape(-1, 3)

    nb = int(rng.integers(n_boxes[0], n_boxes[1] + 1))
    sides = rng.uniform(0.5, 4.0, size=(nb, 3))
    rng_c = rng.uniform(5.0, 60.0, size=nb)
    az_c = np.deg2rad(rng.uniform(-fov_deg / 2, fov_deg / 2, size=nb))
    cx, cy = rng_c * np.cos(az_c), rng_c * np.sin(az_c)
    boxes = np.stack([cx - sides[:, 0] / 2, cy - sides[:, 1] / 2, np.full(nb, ground_z),
                      cx + sides[:, 0] / 2, cy + sides[:, 1] / 2, ground_z + sides[:, 2]], axis=1)

    t = np.full(d.shape[0], np.inf)
    down = d[:, 2] < 0
    t[down] = ground_z / d[down, 2]
    tb = _ray_box_hits(d, boxes, az)
    t = np.minimum(t, tb)
    t = t + rng.normal(0.0, noise, size=t.shape)
    ok = np.isfinite(t) & (t > 0) & (t <= max_range)
    ok &= rng.random(t.shape) < keep
    p = d[ok] * t[ok, None]
    if shuffle:
        p = p[rng.permutation(p.shape[0])]
    return np.ascontiguousarray(p.astype(np.float32))


def lidar_min(n_min: int = 16384, seed: int = 0, **kw):
    """LiDAR scene with at least n_min returns: advance the seed until it holds."""
    s = seed
    while True:
        p = lidar_scene(seed=s, **kw)
        if p.shape[0] >= n_min:
            return p, s
        s += 1


def room_scene(n: int = 1 << 20, seed: int = 0, size=(10.0, 10.0, 3.0), n_objects=(30, 60),
               noise: float = 0.005, shuffle: bool = True) -> np.ndarray:
    """Indoor room: area-uniform points on floor, ceiling, 4 walls and 30-60 objects.

    Half of the objects are boxes (sides U[0.2, 2] m) resting on the floor and
    contributing their 5 visible faces, half are axis-aligned panels with sides
    U[0.5, 3] m.  Gaussian noise per coordinate, seeded shuffle.
    """
    rng = np.random.default_rng(seed)
    X, Y, Z = size
    rects = []  # (origin, edge u, edge v)

    def rect(o, u, v):
        rects.append((np.asarray(o, float), np.asarray(u, float), np.asarray(v, float)))

    rect((0, 0, 0), (X, 0, 0), (0, Y, 0))       # floor
    rect((0, 0, Z), (X, 0, 0), (0, Y, 0))       # ceiling
    rect((0, 0, 0), (X, 0, 0), (0, 0, Z))       # walls
    rect((0, Y, 0), (X, 0, 0), (0, 0, Z))
    rect((0, 0, 0), (0, Y, 0), (0, 0, Z))
    rect((X, 0, 0), (0, Y, 0), (0, 0, Z))
    n_obj = int(rng.integers(n_objects[0], n_objects[1] + 1))
    for k in range(n_obj):
        if k % 2 == 0:
            sx, sy, sz = rng.uniform(0.2, 2.0, size=3)
            x0 = rng.uniform(0, X - sx)
            y0 = rng.uniform(0, Y - sy)
            rect((x0, y0, sz), (sx, 0, 0), (0, sy, 0))          # top
            rect((x0, y0, 0), (sx, 0, 0), (0, 0, sz))           # 4 sides
            rect((x0, y0 + sy, 0), (sx, 0, 0), (0, 0, sz))
            rect((x0, y0, 0), (0, sy, 0), (0, 0, sz))
            rect((x0 + sx, y0, 0), (0, sy, 0), (0, 0, sz))
        else:
            a, b = rng.uniform(0.5, 3.0, size=2)
            axis = int(rng.integers(0, 3))
            if axis == 2:  # horizontal panel
                x0, y0 = rng.uniform(0, X - a), rng.uniform(0, Y - b)
                rect((x0, y0, rng.uniform(0, Z)), (a, 0, 0), (0, b, 0))
            elif axis == 0:  # panel normal to x
                h = min(a, Z)
                y0, z0 = rng.uniform(0, Y - b), rng.uniform(0, Z - h)
                rect((rng.uniform(0, X), y0, z0), (0, b, 0), (0, 0, h))
            else:  # panel normal to y
                h = min(a, Z)
                x0, z0 = rng.uniform(0, X - b), rng.uniform(0, Z - h)
                rect((x0, rng.uniform(0, Y), z0), (b, 0, 0), (0, 0, h))
    O = np.stack([r[0] for r in rects])
    U = np.stack([r[1] for r in rects])
    V = np.stack([r[2] for r in rects])
    area = np.linalg.norm(np.cross(U, V), axis=1)
    cdf = np.cumsum(area) / area.sum()
    which = np.minimum(np.searchsorted(cdf, rng.random(n), side="right"), len(rects) - 1)
    uv = rng.random((n, 2))
    p = O[which] + uv[:, :1] * U[which] + uv[:, 1:] * V[which]
    p = p + rng.normal(0.0, noise, size=p.shape)
    if shuffle:
        p = p[rng.permutation(n)]
    return np.ascontiguousarray(p.astype(np.float32))


def lidar_exact(n: int, seed: int) -> np.ndarray:
    """A LiDAR cloud of exactly n returns: a dense scan (more rings if needed),
    then a seeded subset of n returns kept in scan order."""
    rng = np.random.default_rng(seed + 7_777_777)
    rings = 64
    while True:
        p = lidar_scene(seed=seed, rings=rings, az_steps=2048, keep=1.0)
        if p.shape[0] >= n:
            break
        rings *= 2
    keep = np.sort(rng.choice(p.shape[0], size=n, replace=False))
    return np.ascontiguousarray(p[keep])


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def lidar_batch(count: int = 64, lo: int = 20000, hi: int = 200000, seed: int = 0):
    """`count` LiDAR clouds with N log-uniform in [lo, hi]; returns a list of arrays."""
    sizes = log_uniform_sizes(count, lo, hi, seed)
    return [lidar_exact(int(n), seed * 1000 + i) for i, n in enumerate(sizes)]


def concat(clouds):
    """Concatenate clouds into one (N, 3) array plus int64 segment offsets (S + 1)."""
    offs = np.zeros(len(clouds) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([c.shape[0] for c in clouds])
    pts = np.concatenate(clouds, axis=0) if clouds else np.zeros((0, 3), np.float32)
    return np.ascontiguousarray(pts, dtype=np.float32), offs


def request_stream(count: int, rate_hz: float, seed: int = 0, lo: int = 10000, hi: int = 1_000_000):
    """Poisson arrivals: (arrival_s, n, m) per request, m drawn from {n/4, n/16, 4096}."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps) - gaps[0]
    n = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    choice = rng.integers(0, 3, size=count)
    m = np.where(choice == 0, n // 4, np.where(choice == 1, n // 16, np.minimum(4096, n)))
    return t, n, m.astype(np.int64)


def scene_for(n: int, seed: int) -> np.ndarray:
    """Serving scenes: LiDAR up to 200k points, an indoor room above."""
    if n <= 200_000:
        return lidar_exact(int(n), seed)
    return room_scene(int(n), seed=seed)
