"""Seeded synthetic scan pairs and pose batches (inputs only).

This module makes the inputs that both the CUDA library and the CPU oracle are
fed: point clouds (fp32 xyz, metres), the known transform between two scans
(eta = [tx, ty, tz, thx, thy, thz], FP64, metres / radians, mapping B's frame
into A's frame as p_A = R p_B + t with R = Rz Ry Rx) and batches of candidate
poses.  It holds none of the method's arithmetic (no voxelization, no features,
no histograms, no MI) and imports neither the library nor the oracle.

The paper evaluates on the Ford Campus and KITTI LiDAR datasets (Sec. IV), which
are not available here; these generators stand in for their shape: a vehicle-
mounted multi-beam scanner over an urban scene with a ground plane, buildings,
cars and poles, and a second scan taken from a nearby pose.

Frames: each scan's frame has its origin on the ground below the sensor (z = 0
is the ground), x forward, z up; the sensor sits 1.8 m above that origin.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SENSOR_HEIGHT = 1.8
SEED_BASE = 1709060


@dataclasses.dataclass
class Scene:
    boxes: np.ndarray   # (nb, 6) float64: xmin, ymin, zmin, xmax, ymax, zmax (world)
    poles: np.ndarray   # (np, 4) float64: cx, cy, radius, height
    ground_sigma: float = 0.02


@dataclasses.dataclass
class GridSpec:
    origin: tuple
    res_m: float
    dims: tuple
    feature: int          # 0 count, 1 z-variance, 2 joint
    count_levels: int = 7
    var_levels: int = 15


@dataclasses.dataclass
class Pair:
    xyzA: np.ndarray      # (nA, 3) float32, A's frame
    xyzB: np.ndarray      # (nB, 3) float32, B's frame
    T: np.ndarray         # (6,) float64 eta mapping B -> A
    grid: GridSpec


def rot_zyx(eta) -> np.ndarray:
    """R = Rz(thz) @ Ry(thy) @ Rx(thx) in FP64 (for generating data only)."""
    ax, ay, az = float(eta[3]), float(eta[4]), float(eta[5])
    cx, sx, cy, sy, cz, sz = math.cos(ax), math.sin(ax), math.cos(ay), math.sin(ay), math.cos(az), math.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def to_frame(world_pts: np.ndarray, T) -> np.ndarray:
    """World (A-frame) points expressed in the frame whose pose is T: p_B = R^T (p_A - t)."""
    R = rot_zyx(T)
    t = np.asarray(T[:3], dtype=np.float64)
    return (world_pts - t) @ R


# ----------------------------------------------------------------------------------
# Tiny scene: area-weighted surface sampling (no occlusion)
# ----------------------------------------------------------------------------------
def tiny_scene(rng: np.random.Generator) -> Scene:
    boxes = []
    while len(boxes) < 6:
        sx, sy, sz = rng.uniform(2.0, 8.0, size=3)
        r = rng.uniform(5.0, 15.0)
        a = rng.uniform(-math.pi, math.pi)
        cx, cy = r * math.cos(a), r * math.sin(a)
        b = np.array([cx - sx / 2, cy - sy / 2, 0.0, cx + sx / 2, cy + sy / 2, sz])
        if any(not (b[3] < o[0] or o[3] < b[0] or b[4] < o[1] or o[4] < b[1]) for o in boxes):
            continue
        if b[0] < 2.0 and b[3] > -2.0 and b[1] < 2.0 and b[4] > -2.0:
            continue
        boxes.append(b)
    poles = []
    while len(poles) < 10:
        r = rng.uniform(3.0, 18.0)
        a = rng.uniform(-math.pi, math.pi)
        cx, cy = r * math.cos(a), r * math.sin(a)
        if any(o[0] - 0.2 < cx < o[3] + 0.2 and o[1] - 0.2 < cy < o[4] + 0.2 for o in boxes):
            continue
        poles.append([cx, cy, 0.15, rng.uniform(3.0, 7.0)])
    return Scene(np.array(boxes), np.array(poles))


def _sample_surfaces(scene: Scene, n: int, center_xy, radius: float, rng: np.random.Generator) -> np.ndarray:
    """n points on the scene's surfaces within `radius` (horizontal) of center_xy."""
    cx0, cy0 = center_xy
    surfaces = []  # (area, sampler)
    R = radius + 0.5

    def ground(m):
        rr = R * np.sqrt(rng.uniform(0, 1, m))
        aa = rng.uniform(-math.pi, math.pi, m)
        return np.stack([cx0 + rr * np.cos(aa), cy0 + rr * np.sin(aa), rng.normal(0.0, scene.ground_sigma, m)], 1)

    surfaces.append((math.pi * R * R, ground))
    for b in scene.boxes:
        x0, y0, z0, x1, y1, z1 = b
        dx, dy, dz = x1 - x0, y1 - y0, z1 - z0

        def top(m, x0=x0, y0=y0, x1=x1, y1=y1, z1=z1):
            return np.stack([rng.uniform(x0, x1, m), rng.uniform(y0, y1, m), np.full(m, z1)], 1)

        def sidex(m, xv, y0=y0, y1=y1, z0=z0, z1=z1):
            return np.stack([np.full(m, xv), rng.uniform(y0, y1, m), rng.uniform(z0, z1, m)], 1)

        def sidey(m, yv, x0=x0, x1=x1, z0=z0, z1=z1):
            return np.stack([rng.uniform(x0, x1, m), np.full(m, yv), rng.uniform(z0, z1, m)], 1)

        surfaces.append((dx * dy, top))
        surfaces.append((dy * dz, lambda m, xv=x0, f=sidex: f(m, xv)))
        surfaces.append((dy * dz, lambda m, xv=x1, f=sidex: f(m, xv)))
        surfaces.append((dx * dz, lambda m, yv=y0, f=sidey: f(m, yv)))
        surfaces.append((dx * dz, lambda m, yv=y1, f=sidey: f(m, yv)))
    for p in scene.poles:
        pcx, pcy, pr, ph = p

        def pole(m, pcx=pcx, pcy=pcy, pr=pr, ph=ph):
            aa = rng.uniform(-math.pi, math.pi, m)
            return np.stack([pcx + pr * np.cos(aa), pcy + pr * np.sin(aa), rng.uniform(0.0, ph, m)], 1)

        surfaces.append((2 * math.pi * pr * ph, pole))

    areas = np.array([a for a, _ in surfaces])
    out = []
    have = 0
    # oversample, then keep points inside the radius; repeat until n are collected
    while have < n:
        counts = rng.multinomial(int((n - have) * 1.6) + 64, areas / areas.sum())
        chunk = np.concatenate([f(int(c)) for (a, f), c in zip(surfaces, counts) if c > 0], 0)
        d = np.hypot(chunk[:, 0] - cx0, chunk[:, 1] - cy0)
        chunk = chunk[d <= radius]
        rng.shuffle(chunk, axis=0)
        out.append(chunk)
        have += chunk.shape[0]
    return np.concatenate(out, 0)[:n]


def tiny_grid() -> GridSpec:
    return GridSpec(origin=(-20.0, -20.0, -1.0), res_m=1.0, dims=(40, 40, 8), feature=0, count_levels=7)


def tiny_pair(seed: int = SEED_BASE + 1, T=None, n: int = 8000) -> Pair:
    """Ground plane z=0 with N(0, 0.02 m) noise, 6 axis-aligned boxes of 2-8 m, 10 poles
    r = 0.15 m, n points per scan within 20 m of each scan's origin.  B samples the same
    scene with fresh draws and is expressed in its own frame (pose T)."""
    rng = np.random.default_rng(seed)
    scene = tiny_scene(rng)
    if T is None:
        T = np.array([rng.uniform(-1, 1) / math.sqrt(3), rng.uniform(-1, 1) / math.sqrt(3),
                      rng.uniform(-0.5, 0.5) / math.sqrt(3),
                      *np.deg2rad(rng.uniform(-5, 5, 3) / math.sqrt(3))])
    T = np.asarray(T, dtype=np.float64)
    A = _sample_surfaces(scene, n, (0.0, 0.0), 20.0, rng)
    Bw = _sample_surfaces(scene, n, (T[0], T[1]), 20.0, rng)
    B = to_frame(Bw, T)
    return Pair(A.astype(np.float32), B.astype(np.float32), T, tiny_grid())


# ----------------------------------------------------------------------------------
# LiDAR-shaped scans: multi-beam ray casting of an urban scene
# ----------------------------------------------------------------------------------
def urban_scene(rng: np.random.Generator, extent: float = 110.0, n_buildings: int = 32, n_cars: int = 30,
                n_poles: int = 40) -> Scene:
    """Two crossing streets (along x and y through the origin, half-width 5-7 m) lined by
    building boxes 8-25 m tall set back 8-15 m from the street axis; car boxes
    4.5 x 1.8 x 1.5 m in the lanes; poles r = 0.15 m, 6-8 m tall on the kerbs."""
    boxes = []
    half = rng.uniform(5.0, 7.0)
    tries = 0
    while len(boxes) < n_buildings and tries < 10000:
        tries += 1
        along = rng.uniform(-extent, extent)
        side = rng.choice([-1.0, 1.0])
        setback = rng.uniform(8.0, 15.0)
        depth = rng.uniform(8.0, 20.0)
        length = rng.uniform(10.0, 30.0)
        height = rng.uniform(8.0, 25.0)
        if rng.uniform() < 0.5:  # along the x street
            x0, x1 = along - length / 2, along + length / 2
            y0 = side * setback if side > 0 else -setback - depth
            y1 = y0 + depth
        else:                    # along the y street
            y0, y1 = along - length / 2, along + length / 2
            x0 = side * setback if side > 0 else -setback - depth
            x1 = x0 + depth
        b = np.array([x0, y0, 0.0, x1, y1, height])
        # keep the crossing streets clear
        if (b[1] < half and b[4] > -half) or (b[0] < half and b[3] > -half):
            continue
        if any(not (b[3] + 1 < o[0] or o[3] + 1 < b[0] or b[4] + 1 < o[1] or o[4] + 1 < b[1]) for o in boxes):
            continue
        boxes.append(b)
    cars = []
    tries = 0
    while len(cars) < n_cars and tries < 10000:
        tries += 1
        along = rng.uniform(-60.0, 60.0)
        lane = rng.uniform(-half + 1.0, half - 1.0)
        if abs(along) < 6.0:
            continue
        if rng.uniform() < 0.5:
            b = np.array([along - 2.25, lane - 0.9, 0.0, along + 2.25, lane + 0.9, 1.5])
        else:
            b = np.array([lane - 0.9, along - 2.25, 0.0, lane + 0.9, along + 2.25, 1.5])
        if any(not (b[3] + 0.5 < o[0] or o[3] + 0.5 < b[0] or b[4] + 0.5 < o[1] or o[4] + 0.5 < b[1]) for o in cars):
            continue
        cars.append(b)
    poles = []
    while len(poles) < n_poles:
        along = rng.uniform(-80.0, 80.0)
        side = rng.choice([-1.0, 1.0]) * (half + 0.5)
        if rng.uniform() < 0.5:
            poles.append([along, side, 0.15, rng.uniform(6.0, 8.0)])
        else:
            poles.append([side, along, 0.15, rng.uniform(6.0, 8.0)])
    allb = np.array(boxes + cars) if (boxes or cars) else np.zeros((0, 6))
    return Scene(allb, np.array(poles))


def raycast(scene: Scene, T, n_beams=64, elev_deg=(-24.8, 2.0), az_step_deg=0.17, max_range=100.0,
            range_sigma=0.02, dropout=0.1, rng: np.random.Generator | None = None) -> np.ndarray:
    """Points of a spinning multi-beam scanner at pose T (sensor 1.8 m above the frame origin),
    in the scanner's own frame, ring-major (beam, then azimuth) order.  A fraction `dropout`
    of the returns is lost at random (dark or specular surfaces return nothing)."""
    T = np.asarray(T, dtype=np.float64)
    R = rot_zyx(T)
    origin = R @ np.array([0.0, 0.0, SENSOR_HEIGHT]) + T[:3]
    n_az = int(round(360.0 / az_step_deg))
    el = np.deg2rad(np.linspace(elev_deg[0], elev_deg[1], n_beams))
    az = np.deg2rad(np.arange(n_az) * (360.0 / n_az))
    ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
    dl = np.stack([np.broadcast_to(ce * np.cos(az)[None, :], (n_beams, n_az)),
                   np.broadcast_to(ce * np.sin(az)[None, :], (n_beams, n_az)),
                   np.broadcast_to(se, (n_beams, n_az))], -1).reshape(-1, 3)
    d = dl @ R.T  # world directions
    tbest = np.full(d.shape[0], np.inf)
    # ground plane z = 0
    with np.errstate(divide="ignore", invalid="ignore"):
        tg = np.where(d[:, 2] < 0, -origin[2] / d[:, 2], np.inf)
    tbest = np.minimum(tbest, tg)
    inv = np.where(np.abs(d) > 1e-12, 1.0 / np.where(np.abs(d) > 1e-12, d, 1.0), np.inf)
    for b in scene.boxes:
        t1 = (b[:3] - origin) * inv
        t2 = (b[3:] - origin) * inv
        # rays parallel to a slab: inside -> (-inf, inf), outside -> empty
        par = ~np.isfinite(inv)
        lo = np.where(par, np.where((origin >= b[:3]) & (origin <= b[3:]), -np.inf, np.inf), np.minimum(t1, t2))
        hi = np.where(par, np.where((origin >= b[:3]) & (origin <= b[3:]), np.inf, -np.inf), np.maximum(t1, t2))
        tn = lo.max(1)
        tf = hi.min(1)
        hit = (tn <= tf) & (tf > 0) & (tn > 1e-6)
        tbest = np.where(hit & (tn < tbest), tn, tbest)
    for p in scene.poles:
        cx, cy, r, h = p
        ox, oy = origin[0] - cx, origin[1] - cy
        a = d[:, 0] ** 2 + d[:, 1] ** 2
        bq = 2 * (ox * d[:, 0] + oy * d[:, 1])
        c = ox * ox + oy * oy - r * r
        disc = bq * bq - 4 * a * c
        ok = (disc >= 0) & (a > 1e-12)
        sq = np.sqrt(np.where(ok, disc, 0))
        t = np.where(ok, (-bq - sq) / (2 * np.where(a > 1e-12, a, 1)), np.inf)
        z = origin[2] + t * d[:, 2]
        hit = ok & (t > 1e-6) & (z >= 0) & (z <= h)
        tbest = np.where(hit & (t < tbest), t, tbest)
    keep = tbest <= max_range
    if rng is not None and range_sigma > 0:
        tbest = tbest + rng.normal(0.0, range_sigma, tbest.shape[0])
    if rng is not None and dropout > 0:
        keep &= rng.uniform(0.0, 1.0, tbest.shape[0]) >= dropout
    pts_world = origin + tbest[keep, None] * d[keep]
    return to_frame(pts_world, T)


def lidar_grid(res_m: float = 0.5, extent_xy: float = 80.0, extent_z: float = 8.0) -> GridSpec:
    X = int(round(extent_xy / res_m))
    Z = int(round(extent_z / res_m))
    return GridSpec(origin=(-extent_xy / 2, -extent_xy / 2, -1.0), res_m=res_m, dims=(X, X, Z), feature=1,
                    var_levels=15)


def random_offset(rng: np.random.Generator, max_t=2.0, max_yaw_deg=5.0, max_rp_deg=1.0, max_tz=0.1):
    r = max_t * math.sqrt(rng.uniform())
    a = rng.uniform(-math.pi, math.pi)
    return np.array([r * math.cos(a), r * math.sin(a), rng.uniform(-max_tz, max_tz),
                     math.radians(rng.uniform(-max_rp_deg, max_rp_deg)),
                     math.radians(rng.uniform(-max_rp_deg, max_rp_deg)),
                     math.radians(rng.uniform(-max_yaw_deg, max_yaw_deg))])


def lidar_pair(seed: int = SEED_BASE + 2, T=None, n_beams=64, az_step_deg=0.17, max_range=100.0,
               res_m=0.5, grid: GridSpec | None = None) -> Pair:
    """64-beam scanner (-24.8 .. +2 deg, 0.17 deg azimuth, hits <= 100 m, range noise
    N(0, 0.02 m)) over an urban scene; B from a pose offset |t| <= 2 m, |yaw| <= 5 deg."""
    rng = np.random.default_rng(seed)
    scene = urban_scene(rng)
    if T is None:
        T = random_offset(rng)
    T = np.asarray(T, dtype=np.float64)
    A = raycast(scene, np.zeros(6), n_beams=n_beams, az_step_deg=az_step_deg, max_range=max_range, rng=rng)
    B = raycast(scene, T, n_beams=n_beams, az_step_deg=az_step_deg, max_range=max_range, rng=rng)
    return Pair(A.astype(np.float32), B.astype(np.float32), T, grid or lidar_grid(res_m))


def subsample(xyz: np.ndarray, n: int, rng: np.random.Generator) -> np.ndarray:
    """Keep n points, preserving their order."""
    if n >= xyz.shape[0]:
        return xyz
    idx = np.sort(rng.choice(xyz.shape[0], size=n, replace=False))
    return xyz[idx]


# ----------------------------------------------------------------------------------
# Pose batches
# ----------------------------------------------------------------------------------
def pose_grid(center, half_width, counts) -> np.ndarray:
    """Candidate poses on a regular grid: counts[a] values per axis spread evenly over
    center[a] +- half_width[a]; the last axis varies fastest.  (FP64 eta rows.)"""
    axes = []
    for c, h, m in zip(center, half_width, counts):
        axes.append(np.array([c]) if m <= 1 else c + np.linspace(-h, h, m))
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], 1)


def tiny_poses(center=(0, 0, 0, 0, 0, 0)) -> np.ndarray:
    """3^6 = 729 poses {-s, 0, +s} per axis with s = (1 m, 1 m, 0.5 m, 2.5, 2.5, 5 deg)."""
    s = np.array([1.0, 1.0, 0.5, math.radians(2.5), math.radians(2.5), math.radians(5.0)])
    return pose_grid(center, s, (3, 3, 3, 3, 3, 3))


def lidar_poses(center=(0, 0, 0, 0, 0, 0), half_width=(2.0, 2.0, 0.25, math.radians(1.0), math.radians(1.0),
                                                       math.radians(5.0)),
                counts=(8, 8, 2, 2, 2, 8)) -> np.ndarray:
    """4,096 poses: 8 tx x 8 ty x 2 tz x 2 roll x 2 pitch x 8 yaw around center."""
    return pose_grid(center, half_width, counts)


# ----------------------------------------------------------------------------------
# Batched and served workloads: many pairs of uneven sizes and grid resolutions
# ----------------------------------------------------------------------------------
BATCH_RESOLUTIONS = (0.25, 0.5, 1.0)


def batched_pairs(n_pairs: int = 64, seed: int = SEED_BASE + 3, n_scenes: int = 4, n_min: int = 20000,
                  n_max: int = 130000, n_beams: int = 64, az_step_deg: float = 0.15) -> list:
    """n_pairs independent pairs: point counts log-uniform in [n_min, n_max] (subsampled,
    scan order kept, from n_scenes ray-cast pairs), grid resolution cycling over 0.25 /
    0.5 / 1 m with dims covering 80 x 80 x 8 m.  Both scans of a pair get the same count."""
    rng = np.random.default_rng(seed)
    bases = [lidar_pair(seed=seed + 100 + k, n_beams=n_beams, az_step_deg=az_step_deg) for k in range(n_scenes)]
    out = []
    for i in range(n_pairs):
        base = bases[i % n_scenes]
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        A = subsample(base.xyzA, n, rng)
        B = subsample(base.xyzB, n, rng)
        res = BATCH_RESOLUTIONS[i % len(BATCH_RESOLUTIONS)]
        out.append(Pair(A, B, base.T.copy(), lidar_grid(res)))
    return out


def poisson_arrivals(rate_hz: float, n: int, seed: int = SEED_BASE + 4) -> np.ndarray:
    """Arrival times (s) of n requests of a Poisson process with the given mean rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


# ----------------------------------------------------------------------------------
# Large workload: 128-beam scanner, 0.2 m grid, joint count x z-variance feature
# ----------------------------------------------------------------------------------
def large_grid() -> GridSpec:
    """400 x 400 x 40 voxels at 0.2 m (6.4M voxels); joint count (7 levels) x z-variance
    (8 levels) feature: 1 + 7 * 8 = 57 symbols."""
    return GridSpec(origin=(-40.0, -40.0, -1.0), res_m=0.2, dims=(400, 400, 40), feature=2, count_levels=7,
                    var_levels=8)


def large_pair(seed: int = SEED_BASE + 5, T=None) -> Pair:
    """128 beams over -25 .. +15 deg, 0.15 deg azimuth (2,400 steps), hits <= 120 m, range
    noise N(0, 0.02 m); B from a pose offset up to 10 m / 30 deg yaw."""
    rng = np.random.default_rng(seed)
    scene = urban_scene(rng)
    if T is None:
        r = 10.0 * math.sqrt(rng.uniform())
        a = rng.uniform(-math.pi, math.pi)
        T = np.array([r * math.cos(a), r * math.sin(a), rng.uniform(-0.1, 0.1), math.radians(rng.uniform(-1, 1)),
                      math.radians(rng.uniform(-1, 1)), math.radians(rng.uniform(-30, 30))])
    T = np.asarray(T, dtype=np.float64)
    kw = dict(n_beams=128, elev_deg=(-25.0, 15.0), az_step_deg=0.15, max_range=120.0, rng=rng)
    A = raycast(scene, np.zeros(6), **kw)
    B = raycast(scene, T, **kw)
    return Pair(A.astype(np.float32), B.astype(np.float32), T, large_grid())


def large_poses(center=(0, 0, 0, 0, 0, 0)) -> np.ndarray:
    """32,768 poses: 16 tx x 16 ty x 2 tz x 2 roll x 2 pitch x 16 yaw over +-10 m, +-0.25 m,
    +-1 deg, +-30 deg around center."""
    return pose_grid(center, (10.0, 10.0, 0.25, math.radians(1.0), math.radians(1.0), math.radians(30.0)),
                     (16, 16, 2, 2, 2, 16))
