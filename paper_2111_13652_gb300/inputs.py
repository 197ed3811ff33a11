"""Seeded synthetic inputs: analytic scenes, an FP64 ray-caster, camera trajectories, depth noise.

This module produces *inputs only*: depth images, camera poses and (for the dense sphere case)
the analytic grid values that the method is then run on.  It holds none of the method's
arithmetic (no back-projection into the map, no fusion, no tracking), so the CUDA path and the
CPU oracle can both consume it without sharing method code.

Conventions (stated once, used everywhere):
  * camera frame: x right, y down, z forward; pixel (u, v) looks along (u - cx)/fx, (v - cy)/fy, 1;
  * a pose T_wc is a 4x4 row-major FP64 matrix mapping camera points to world points, P = R p + t;
  * depth is z-depth in metres (FP32), 0 marks "no measurement";
  * signed distances are inside-positive (negative in free space), matching Sec. 3.1 of the paper.

The synthetic workloads take the shapes of the paper's RGB-D data (Sec. 5.3: 640x480 frames,
3.5 m depth cutoff, 1-2 cm voxels, truncation 5 voxels); the TUM/Redwood sequences themselves
are not used.
"""
from __future__ import annotations

import dataclasses
import math
import os

import numpy as np

# --------------------------------------------------------------------------------------------
# small pose helpers (input construction only)
# --------------------------------------------------------------------------------------------


def look_at(position, target, up=(0.0, 0.0, 1.0), roll=0.0) -> np.ndarray:
    """Camera-to-world pose at `position` whose optical axis (+z) points at `target`."""
    c = np.asarray(position, np.float64)
    z = np.asarray(target, np.float64) - c
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    if np.linalg.norm(x) < 1e-9:  # looking straight up/down: pick any horizontal x
        x = np.cross(z, np.array([1.0, 0.0, 0.0]))
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=1)
    if roll != 0.0:
        R = R @ axis_angle(np.array([0.0, 0.0, 1.0]), roll)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = c
    return T


def axis_angle(axis, angle) -> np.ndarray:
    """Rotation matrix about a unit axis (input construction; Rodrigues' formula)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def perturb_pose(T: np.ndarray, rng: np.random.Generator, angle_deg=5.0, trans_m=0.05) -> np.ndarray:
    """Left-multiply T by a rotation of `angle_deg` about a random axis and a random translation."""
    axis = rng.normal(size=3)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    dT = np.eye(4)
    dT[:3, :3] = axis_angle(axis, math.radians(angle_deg))
    dT[:3, 3] = trans_m * d
    return dT @ T


# --------------------------------------------------------------------------------------------
# camera
# --------------------------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    depth_max: float = 3.5

    def ray_dirs_cam(self) -> np.ndarray:
        """(H*W, 3) FP64 camera-frame ray directions with unit z (so ray parameter = z-depth)."""
        u = np.arange(self.width, dtype=np.float64)
        v = np.arange(self.height, dtype=np.float64)
        uu, vv = np.meshgrid(u, v)
        d = np.stack([(uu - self.cx) / self.fx, (vv - self.cy) / self.fy, np.ones_like(uu)], axis=-1)
        return d.reshape(-1, 3)


KINECT_640 = Camera(525.0, 525.0, 319.5, 239.5, 640, 480, 3.5)
TINY_160 = Camera(140.0, 140.0, 80.0, 60.0, 160, 120, 3.5)


# --------------------------------------------------------------------------------------------
# analytic scenes and ray casting (FP64)
# --------------------------------------------------------------------------------------------


def _ray_sphere(o, d, c, r):
    """Smallest positive ray parameter hitting sphere (c, r) from outside; inf if none."""
    oc = o - c
    a = np.einsum("ij,ij->i", d, d)
    b = 2.0 * (d @ oc)
    cc = float(oc @ oc) - r * r
    disc = b * b - 4 * a * cc
    t = np.full(d.shape[0], np.inf)
    ok = np.nonzero(disc >= 0)[0]
    if ok.size == 0:
        return t
    sq = np.sqrt(disc[ok])
    t0 = (-b[ok] - sq) / (2 * a[ok])
    t1 = (-b[ok] + sq) / (2 * a[ok])
    t[ok] = np.where(t0 > 1e-9, t0, np.where(t1 > 1e-9, t1, np.inf))
    return t


def _ray_box(o, d, lo, hi):
    """Entry parameter into the solid axis-aligned box [lo, hi] (camera outside); inf if missed."""
    t = np.full(d.shape[0], np.inf)
    c = 0.5 * (lo + hi)
    cand = np.isfinite(_ray_sphere(o, d, c, float(np.linalg.norm(hi - c)) + 1e-6))
    if not np.any(cand):
        return t
    dc = d[cand]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / dc
        t1 = (lo - o) * inv
        t2 = (hi - o) * inv
    t1 = np.where(np.isnan(t1), -np.inf, t1)
    t2 = np.where(np.isnan(t2), np.inf, t2)
    tmin = np.max(np.minimum(t1, t2), axis=1)
    tmax = np.min(np.maximum(t1, t2), axis=1)
    hit = (tmax >= tmin) & (tmax > 1e-9)
    t[cand] = np.where(hit, np.where(tmin > 1e-9, tmin, tmax), np.inf)
    return t


def _ray_room_exit(o, d, lo, hi):
    """Ray parameter where a ray starting inside the box [lo, hi] leaves it (hits a wall)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t_hi = (hi - o) * inv
        t_lo = (lo - o) * inv
    t_exit = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
    return np.min(t_exit, axis=1)


@dataclasses.dataclass
class SphereScene:
    center: np.ndarray
    radius: float

    def raycast(self, o, d):
        return _ray_sphere(o, d, self.center, self.radius)

    def sdf(self, x):
        """Inside-positive signed distance r - |x - c| and its gradient -(x - c)/|x - c|."""
        rel = x - self.center
        n = np.linalg.norm(rel, axis=-1)
        psi = self.radius - n
        with np.errstate(invalid="ignore", divide="ignore"):
            g = -rel / n[..., None]
        return psi, g


@dataclasses.dataclass
class RoomScene:
    lo: np.ndarray  # room interior bounds (walls face inward)
    hi: np.ndarray
    spheres: list  # [(center(3,), r)]
    boxes: list  # [(lo(3,), hi(3,))]

    def raycast(self, o, d):
        return self.raycast_id(o, d)[0]

    def raycast_id(self, o, d):
        """Ray parameter and surface id: 0..5 the walls (-x, +x, -y, +y, -z, +z), 6.. spheres, then boxes."""
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            t_hi = (self.hi - o) * inv
            t_lo = (self.lo - o) * inv
        t_exit = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
        axis = np.argmin(t_exit, axis=1)
        t = t_exit[np.arange(len(d)), axis]
        sid = 2 * axis + (d[np.arange(len(d)), axis] > 0)
        for k, (c, r) in enumerate(self.spheres):
            ts = _ray_sphere(o, d, c, r)
            closer = ts < t
            t = np.where(closer, ts, t)
            sid = np.where(closer, 6 + k, sid)
        for k, (blo, bhi) in enumerate(self.boxes):
            tb = _ray_box(o, d, blo, bhi)
            closer = tb < t
            t = np.where(closer, tb, t)
            sid = np.where(closer, 6 + len(self.spheres) + k, sid)
        return t, sid

    def normals(self, p, sid):
        """Unit surface normals (sign irrelevant) at hit points p with surface ids sid."""
        n = np.zeros_like(p)
        wall = sid < 6
        n[wall, sid[wall] // 2] = 1.0
        ns = len(self.spheres)
        for k, (c, r) in enumerate(self.spheres):
            m = sid == 6 + k
            n[m] = (p[m] - c) / r
        for k, (blo, bhi) in enumerate(self.boxes):
            m = np.where(sid == 6 + ns + k)[0]
            q = p[m]
            ax = np.argmin(np.minimum(np.abs(q - blo), np.abs(q - bhi)), axis=1)
            n[m, ax] = 1.0
        return n

    def free_clearance(self, x):
        """Distance from point x to the nearest obstacle surface (positive in free space)."""
        x = np.asarray(x, np.float64)
        dist = min(np.min(x - self.lo), np.min(self.hi - x))
        for c, r in self.spheres:
            dist = min(dist, np.linalg.norm(x - c) - r)
        for blo, bhi in self.boxes:
            q = np.maximum(np.maximum(blo - x, x - bhi), 0.0)
            dist = min(dist, np.linalg.norm(q) if np.any(q > 0) else -1.0)
        return dist


@dataclasses.dataclass
class PlanesScene:
    """Union of half-spaces' boundary planes seen from inside: n.x = off (n points into the wall)."""
    normals: np.ndarray  # (k, 3) unit
    offsets: np.ndarray  # (k,)

    def raycast(self, o, d):
        t = np.full(d.shape[0], np.inf)
        for n, off in zip(self.normals, self.offsets):
            dn = d @ n
            with np.errstate(divide="ignore", invalid="ignore"):
                tt = (off - o @ n) / dn
            t = np.minimum(t, np.where((dn > 1e-12) & (tt > 1e-9), tt, np.inf))
        return t

    def sdf(self, x):
        """Inside-positive distance of the 'outside the room' region: max_k (n_k.x - off_k)."""
        vals = np.stack([x @ n - off for n, off in zip(self.normals, self.offsets)], axis=-1)
        k = np.argmax(vals, axis=-1)
        psi = np.take_along_axis(vals, k[..., None], axis=-1)[..., 0]
        g = self.normals[k]
        return psi, g


def render_depth(scene, cam: Camera, T_wc: np.ndarray) -> np.ndarray:
    """FP64 ray cast of `scene` from pose T_wc; returns an (H, W) FP32 z-depth image, 0 = miss."""
    dc = cam.ray_dirs_cam()
    d = dc @ T_wc[:3, :3].T
    o = T_wc[:3, 3]
    t = scene.raycast(o, d)  # ray parameter == z-depth since dc has unit z
    depth = np.where(np.isfinite(t), t, 0.0)
    return depth.reshape(cam.height, cam.width).astype(np.float32)


def add_depth_noise(depth: np.ndarray, rng: np.random.Generator, k=0.0012) -> np.ndarray:
    """Axial noise with standard deviation k z^2 (Kinect-like), zeros kept as misses."""
    z = depth.astype(np.float64)
    noisy = z + rng.normal(size=z.shape) * (k * z * z)
    noisy = np.where(z > 0, np.maximum(noisy, 0.0), 0.0)
    return noisy.astype(np.float32)


# --------------------------------------------------------------------------------------------
# the dense-sphere workload (64^3 grid, 2 cm voxels, sphere r = 0.4 m at the grid centre)
# --------------------------------------------------------------------------------------------


@dataclasses.dataclass
class DenseSphereCase:
    cam: Camera
    voxel_size: float
    truncation: float
    dims: tuple
    origin: tuple  # integer coordinate of voxel (0, 0, 0)
    psi: np.ndarray  # (dz, dy, dx) FP32, x fastest
    grad: np.ndarray  # (dz, dy, dx, 3) FP32
    weight: np.ndarray  # (dz, dy, dx) FP32
    depth: np.ndarray  # (H, W) FP32
    T_gt: np.ndarray
    T_init: np.ndarray
    scene: SphereScene
    n_iters: int = 20


def dense_sphere_case(seed: int = 1, dims=64, voxel_size=0.02, radius=0.4, distance=1.2,
                      cam: Camera = TINY_160, n_iters: int = 20) -> DenseSphereCase:
    """Analytic sphere SDF on a dense grid plus one depth image from a seed-random viewpoint."""
    rng = np.random.default_rng(seed)
    T = 5 * voxel_size
    half = dims // 2
    origin = (-half, -half, -half)
    m = np.arange(dims) - half
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    vox = np.stack([mx, my, mz], axis=-1).astype(np.float64) * np.float64(np.float32(voxel_size))
    scene = SphereScene(np.zeros(3), radius)
    psi, g = scene.sdf(vox)
    w = (np.abs(psi) <= T).astype(np.float32)
    g = np.nan_to_num(g)
    direction = rng.normal(size=3)
    direction /= np.linalg.norm(direction)
    T_gt = look_at(distance * direction, np.zeros(3), roll=rng.uniform(-math.pi, math.pi))
    depth = render_depth(scene, cam, T_gt)
    T_init = perturb_pose(T_gt, rng, 5.0, 0.05)
    return DenseSphereCase(cam, voxel_size, T, (dims, dims, dims), origin,
                           psi.astype(np.float32), g.astype(np.float32), w, depth, T_gt, T_init,
                           scene, n_iters)


# --------------------------------------------------------------------------------------------
# the hashed room workload (4x4x3 m room, 10 spheres, 6 boxes, smooth trajectory)
# --------------------------------------------------------------------------------------------


def make_room(seed: int, size=(4.0, 4.0, 3.0), n_spheres=10, n_boxes=6) -> RoomScene:
    """Room with inward-facing walls and seed-placed, non-overlapping spheres and boxes."""
    rng = np.random.default_rng(seed)
    lo = np.zeros(3)
    hi = np.asarray(size, np.float64)
    placed = []  # bounding spheres (c, r) for overlap rejection
    spheres, boxes = [], []
    margin = 0.05

    def free(c, r):
        return all(np.linalg.norm(c - pc) > r + pr + margin for pc, pr in placed)

    while len(boxes) < n_boxes:
        half = rng.uniform(0.1, 0.4, size=3)
        c = np.array([rng.uniform(0.3 + half[0], hi[0] - 0.3 - half[0]),
                      rng.uniform(0.3 + half[1], hi[1] - 0.3 - half[1]),
                      half[2]])  # resting on the floor
        r = float(np.linalg.norm(half))
        if free(c, r):
            placed.append((c, r))
            boxes.append((c - half, c + half))
    while len(spheres) < n_spheres:
        r = rng.uniform(0.1, 0.4)
        c = np.array([rng.uniform(r + 0.2, hi[0] - r - 0.2), rng.uniform(r + 0.2, hi[1] - r - 0.2),
                      rng.uniform(r + 0.1, hi[2] - r - 0.2)])
        if free(c, r):
            placed.append((c, r))
            spheres.append((c, float(r)))
    return RoomScene(lo, hi, spheres, boxes)


def _bspline(ctrl: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Uniform cubic B-spline through control rows `ctrl`, evaluated at s in [0, len(ctrl) - 3)."""
    i = np.clip(np.floor(s).astype(int), 0, len(ctrl) - 4)
    u = (s - i)[:, None]
    b0 = (1 - u) ** 3 / 6
    b1 = (3 * u**3 - 6 * u**2 + 4) / 6
    b2 = (-3 * u**3 + 3 * u**2 + 3 * u + 1) / 6
    b3 = u**3 / 6
    return b0 * ctrl[i] + b1 * ctrl[i + 1] + b2 * ctrl[i + 2] + b3 * ctrl[i + 3]


def room_trajectory(scene: RoomScene, n_frames: int, seed: int, frames_per_segment=25,
                    step=0.5) -> list:
    """Smooth camera path: B-spline over a seeded random walk of positions and look-at targets.

    Positions stay >= 0.35 m from every surface and >= 0.7 m from the walls; about step /
    frames_per_segment metres of motion per frame (2 cm at the defaults)."""
    # separate streams for positions and targets: the first frames do not depend on n_frames
    rng = np.random.default_rng(seed + 7919)
    rng_t = np.random.default_rng(seed + 7920)
    n_ctrl = n_frames // frames_per_segment + 4
    center = 0.5 * (scene.lo + scene.hi)
    pos = [center.copy()]
    while scene.free_clearance(pos[0]) < 0.35:
        pos[0] = center + rng.uniform(-0.8, 0.8, size=3) * np.array([1, 1, 0.3])
    tries = 0
    while len(pos) < n_ctrl:
        cand = pos[-1] + step * _unit(rng.normal(size=3) * np.array([1, 1, 0.4]))
        ok = np.all(cand > scene.lo + 0.7) and np.all(cand < scene.hi - 0.7)
        if ok and scene.free_clearance(cand) > 0.35:
            pos.append(cand)
            tries = 0
        else:
            tries += 1
            if tries > 200:  # back off toward the centre
                pos.append(0.5 * (pos[-1] + center))
    pos = np.array(pos)
    tgt = [center + rng_t.uniform(-1, 1, size=3) * np.array([1.2, 1.2, 0.6])]
    while len(tgt) < n_ctrl:
        tgt.append(np.clip(tgt[-1] + 0.6 * _unit(rng_t.normal(size=3)), scene.lo + 0.2, scene.hi - 0.2))
    tgt = np.array(tgt)
    s = np.arange(n_frames, dtype=np.float64) / frames_per_segment
    P = _bspline(pos, s)
    Q = _bspline(tgt, s)
    poses = []
    for p, q in zip(P, Q):
        if np.linalg.norm(q - p) < 0.5:  # keep the target away from the camera
            q = p + 0.5 * _unit(q - p + 1e-3)
        poses.append(look_at(p, q))
    return poses


def _unit(x):
    return x / np.linalg.norm(x)


@dataclasses.dataclass
class RoomSequence:
    cam: Camera
    scene: RoomScene
    poses: list  # ground-truth T_wc per frame
    depths: np.ndarray  # (F, H, W) FP32, noisy
    voxel_size: float
    truncation: float


class _SingleThreadedChildren:
    """Within the block, processes started inherit single-threaded BLAS / OpenMP settings, so that
    a pool of one process per core does not start one thread per core in each of them."""

    VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")

    def __enter__(self):
        self.saved = {k: os.environ.get(k) for k in self.VARS}
        for k in self.VARS:
            os.environ[k] = "1"

    def __exit__(self, *a):
        for k, v in self.saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def room_sequence(seed: int = 2, n_frames: int = 100, cam: Camera = KINECT_640, voxel_size=0.01,
                  noise=True, frames_per_segment=25, processes: int = 1,
                  conditioned_horizon: int | None = None) -> RoomSequence:
    """Room scene, smooth trajectory and noisy depth frames (sigma = 0.0012 z^2).  `processes` > 1
    ray-casts the frames in a spawned pool; the noise is drawn afterwards in frame order, so the
    frames do not depend on it.  With conditioned_horizon the trajectory is re-drawn until every
    view over that many frames is well-conditioned (conditioned_trajectory)."""
    scene = make_room(seed)
    if conditioned_horizon is None:
        poses = room_trajectory(scene, n_frames, seed, frames_per_segment)
    else:
        poses = conditioned_trajectory(scene, cam, n_frames, seed, frames_per_segment, conditioned_horizon)
    rng = np.random.default_rng(seed + 104729)
    if processes > 1:
        import concurrent.futures as cf
        import functools
        import multiprocessing as mp

        with _SingleThreadedChildren(), cf.ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
            clean = list(ex.map(functools.partial(render_depth, scene, cam), poses, chunksize=4))
    else:
        clean = [render_depth(scene, cam, T) for T in poses]
    depths = np.empty((n_frames, cam.height, cam.width), np.float32)
    for f, d in enumerate(clean):
        depths[f] = add_depth_noise(d, rng) if noise else d
    return RoomSequence(cam, scene, poses, depths, voxel_size, 5 * voxel_size)


# --------------------------------------------------------------------------------------------
# the batch workload: many independent scenes of uneven sizes
# --------------------------------------------------------------------------------------------

RESOLUTIONS = [(160, 120), (320, 240), (480, 360), (640, 480)]


def scaled_camera(width, height) -> Camera:
    """Kinect-like intrinsics scaled to the resolution (f = 525 at 640 px)."""
    f = 525.0 * width / 640.0
    return Camera(f, f, width / 2.0 - 0.5, height / 2.0 - 0.5, width, height, 3.5)


@dataclasses.dataclass
class BatchScene:
    index: int
    cam: Camera
    voxel_size: float
    dense_dims: tuple | None  # None: hashed map
    dense_origin: tuple | None
    hash_slots: int
    damping: float
    poses: list
    depths: np.ndarray  # (F, H, W) FP32


def sphere_orbit_poses(n_frames: int, seed: int, radius=0.5, deg_per_frame=1.5) -> list:
    """Camera on a tilted circle around the origin, looking at it."""
    rng = np.random.default_rng(seed)
    tilt = rng.uniform(-0.5, 0.5)
    phase = rng.uniform(0, 2 * math.pi)
    poses = []
    for f in range(n_frames):
        a = phase + math.radians(deg_per_frame) * f
        c = radius * np.array([math.cos(a) * math.cos(tilt), math.sin(a) * math.cos(tilt), math.sin(tilt)])
        poses.append(look_at(c, np.zeros(3), roll=0.3 * math.sin(a)))
    return poses


def view_observability(scene: RoomScene, cam: Camera, T_wc: np.ndarray, stride: int = 8) -> float:
    """Smallest eigenvalue of the mean of n n^T over the surface normals a view sees within the
    depth range (every stride-th pixel).  A camera position is recoverable from depth along every
    direction only if the visible normals span 3D; a view of one wall (or of two walls and
    nothing else) has a value near 0."""
    dc = cam.ray_dirs_cam().reshape(cam.height, cam.width, 3)[::stride, ::stride].reshape(-1, 3)
    d = dc @ T_wc[:3, :3].T
    o = T_wc[:3, 3]
    t, sid = scene.raycast_id(o, d)
    ok = np.isfinite(t) & (t > 0) & (t <= cam.depth_max)
    if not np.any(ok):
        return 0.0
    n = scene.normals(o + d[ok] * t[ok, None], sid[ok])
    return float(np.linalg.eigvalsh(n.T @ n / len(n))[0])


def max_turn_deg(poses) -> float:
    """Largest rotation angle between consecutive camera orientations, in degrees."""
    worst = 0.0
    for a, b in zip(poses[:-1], poses[1:]):
        c = (np.trace(a[:3, :3].T @ b[:3, :3]) - 1.0) / 2.0
        worst = max(worst, math.degrees(math.acos(min(1.0, max(-1.0, c)))))
    return worst


BATCH_HORIZON = 64  # batch-room trajectories are checked over this many frames
MIN_OBSERVABILITY = 0.03
MAX_TURN_DEG = 1.5


def conditioned_trajectory(scene: RoomScene, cam: Camera, n_frames: int, seed: int, frames_per_segment=25,
                           horizon: int = BATCH_HORIZON) -> list:
    """A room trajectory drawn as room_trajectory does, and re-drawn with the next seed until, over
    the first max(n_frames, horizon) frames, the camera turns at most MAX_TURN_DEG per frame and
    every view has view_observability >= MIN_OBSERVABILITY.  The check covers a fixed horizon, so a
    sequence's first frames do not depend on its length."""
    h = max(n_frames, horizon)
    poses = None
    for attempt in range(256):
        poses = room_trajectory(scene, h, seed + 1_000_003 * attempt, frames_per_segment)
        if max_turn_deg(poses) <= MAX_TURN_DEG and all(
                view_observability(scene, cam, T) >= MIN_OBSERVABILITY for T in poses):
            break
    else:
        raise RuntimeError(f"no well-conditioned trajectory found for seed {seed}")
    return poses[:n_frames]


def batch_room_trajectory(scene: RoomScene, cam: Camera, n_frames: int, seed: int) -> list:
    """A room trajectory of the batch workload: conditioned_trajectory over BATCH_HORIZON frames."""
    return conditioned_trajectory(scene, cam, n_frames, seed)


def batch_scene(index: int, n_frames: int, seed: int = 5) -> BatchScene:
    """Scene `index` of the batch workload: resolution and voxel size cycle with index mod 4;
    index mod 4 == 0 is a dense 64^3 grid around a sphere, the others hashed rooms."""
    kind = index % 4
    w, h = RESOLUTIONS[kind]
    cam = scaled_camera(w, h)
    vs = 0.01 * (1 + kind)
    rng = np.random.default_rng(seed * 1000 + index)
    if kind == 0:
        scene = SphereScene(np.zeros(3), float(rng.uniform(0.18, 0.24)))
        poses = sphere_orbit_poses(n_frames, seed * 1000 + index, radius=float(rng.uniform(0.45, 0.6)))
        dims, origin, slots, damping = (64, 64, 64), (-32, -32, -32), 1, 1e-4
    else:
        scene = make_room(seed * 1000 + index)
        poses = batch_room_trajectory(scene, cam, n_frames, seed * 1000 + index)
        dims, origin, damping = None, None, 0.0
        slots = 1 << 13  # 2e6 voxels of capacity at a load factor below 1/2
    depths = np.empty((n_frames, h, w), np.float32)
    for f, T in enumerate(poses):
        depths[f] = add_depth_noise(render_depth(scene, cam, T), rng)
    return BatchScene(index, cam, vs, dims, origin, slots, damping, poses, depths)


def batch_scenes(n_scenes: int, n_frames: int, seed: int = 5, processes: int = 1) -> list:
    """All scenes of the batch workload; `processes` > 1 ray-casts them in a spawned pool."""
    if processes > 1:
        import concurrent.futures as cf
        import functools
        import multiprocessing as mp

        with _SingleThreadedChildren(), cf.ProcessPoolExecutor(processes, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(functools.partial(batch_scene, n_frames=n_frames, seed=seed), range(n_scenes)))
    return [batch_scene(i, n_frames, seed) for i in range(n_scenes)]


# --------------------------------------------------------------------------------------------
# colour: per-surface albedo times 3-octave value noise (Lambertian-free: intensity = albedo)
# --------------------------------------------------------------------------------------------


def _value_noise(p: np.ndarray, seed: int, spacing: float) -> np.ndarray:
    """Trilinearly interpolated random lattice values in [0, 1) at points p (n, 3)."""
    q = p / spacing
    base = np.floor(q).astype(np.int64)
    f = q - base
    out = np.zeros(len(p))
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                c = base + np.array([dx, dy, dz])
                h = (c[:, 0] * 73856093) ^ (c[:, 1] * 19349663) ^ (c[:, 2] * 83492791) ^ (seed * 2654435761)
                h = (h * 0x9E3779B1) & 0xFFFFFFFF
                val = (h % 100003) / 100003.0
                wgt = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
                out += wgt * val
    return out


def surface_albedo(n_surfaces: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed + 31337).uniform(0.2, 0.9, size=(n_surfaces, 3))


def render_rgbd(scene: RoomScene, cam: Camera, T_wc: np.ndarray, seed: int):
    """FP64 ray cast returning (depth (H, W) FP32, rgb (H, W, 3) FP32): colour = per-surface albedo
    (uniform in [0.2, 0.9] per channel) times 0.6 + 0.4 * 3-octave value noise of the hit point."""
    dc = cam.ray_dirs_cam()
    d = dc @ T_wc[:3, :3].T
    o = T_wc[:3, 3]
    t, sid = scene.raycast_id(o, d)
    hit = np.isfinite(t)
    depth = np.where(hit, t, 0.0)
    pts = o + d * np.where(hit, t, 0.0)[:, None]
    noise = (_value_noise(pts, seed, 0.2) + 0.5 * _value_noise(pts, seed + 1, 0.1) +
             0.25 * _value_noise(pts, seed + 2, 0.05)) / 1.75
    alb = surface_albedo(6 + len(scene.spheres) + len(scene.boxes), seed)[sid]
    rgb = alb * (0.6 + 0.4 * noise)[:, None]
    rgb = np.where(hit[:, None], rgb, 0.0)
    return (depth.reshape(cam.height, cam.width).astype(np.float32),
            rgb.reshape(cam.height, cam.width, 3).astype(np.float32))


@dataclasses.dataclass
class KeyframeSet:
    cam: Camera
    scene: RoomScene
    poses: list
    depths: np.ndarray  # (F, H, W)
    rgbs: np.ndarray  # (F, H, W, 3)
    voxel_size: float


def keyframes(seed: int = 2, n_keyframes: int = 10, stride: int = 10, cam: Camera = KINECT_640,
              voxel_size: float = 0.01) -> KeyframeSet:
    """RGB-D keyframes (every `stride`-th frame of the room trajectory), noise-free depth."""
    scene = make_room(seed)
    poses_all = room_trajectory(scene, n_keyframes * stride, seed)
    poses = poses_all[::stride][:n_keyframes]
    depths = np.empty((n_keyframes, cam.height, cam.width), np.float32)
    rgbs = np.empty((n_keyframes, cam.height, cam.width, 3), np.float32)
    for i, T in enumerate(poses):
        depths[i], rgbs[i] = render_rgbd(scene, cam, T, seed)
    return KeyframeSet(cam, scene, poses, depths, rgbs, voxel_size)
