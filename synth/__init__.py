"""Seeded synthetic inputs for the equirectangular splatting path.

This module only draws random numbers and lays them out. It holds none of the rendering arithmetic (no projection,
no covariance, no blending), so that the FP64 oracle and the CUDA path can both take their inputs from here without
sharing any of the method's code.

Scene shapes follow the workloads the paper measures on (egocentric captures inside a room, Sec. 5.3; roaming
captures through connected rooms, Sec. 5.2). The datasets themselves are not available, so these generators stand in
for them with the same geometry classes. Attribute distributions (per Gaussian):

* log-scale ~ N(-3, 0.5) per axis, stored as linear scale exp(.)
* quaternion (w, x, y, z) = normalise(N(0, I4))
* opacity = sigmoid(N(0, 1))
* SH degree 3: DC ~ N(0.5, 0.2), higher bands ~ N(0, 0.3)

All arrays are float32 and C-contiguous.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SH_COEFFS = {0: 1, 1: 4, 2: 9, 3: 16}


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # [N, 3] world position m
    scales: np.ndarray     # [N, 3] linear scale S (positive)
    quats: np.ndarray      # [N, 4] rotation q, (w, x, y, z), unit norm
    opacity: np.ndarray    # [N]    opacity o in (0, 1)
    sh: np.ndarray         # [N, K, 3] SH coefficients, K = (degree + 1)^2
    sh_degree: int = 3

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return self.means, self.scales, self.quats, self.opacity, self.sh

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity[idx].copy(), self.sh[idx].copy(), self.sh_degree)


def _attributes(rng: np.random.Generator, n: int, sh_degree: int, log_scale_mean=-3.0, log_scale_std=0.5):
    scales = np.exp(rng.normal(log_scale_mean, log_scale_std, size=(n, 3)))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.0, size=n)))
    k = SH_COEFFS[sh_degree]
    sh = rng.normal(0.0, 0.3, size=(n, k, 3))
    sh[:, 0, :] = rng.normal(0.5, 0.2, size=(n, 3))
    return (scales.astype(np.float32), q.astype(np.float32), opacity.astype(np.float32), sh.astype(np.float32))


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def shell_scene(n: int, seed: int, r_min: float = 0.5, r_max: float = 5.0, sh_degree: int = 3,
                log_scale_mean: float = -3.0) -> Scene:
    """Means uniform in the volume of a spherical shell around the origin (camera at the origin)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(r_min ** 3, r_max ** 3, size=n)
    means = _unit_vectors(rng, n) * np.cbrt(u)[:, None]
    scales, quats, opacity, sh = _attributes(rng, n, sh_degree, log_scale_mean=log_scale_mean)
    return Scene(means.astype(np.float32), scales, quats, opacity, sh, sh_degree)


# Room used by the egocentric workload: 10 x 3 x 8 m (x, y, z), y pointing down as in the camera convention.
ROOM_HALF = np.array([5.0, 1.5, 4.0])


def _box_surface_points(rng: np.random.Generator, n: int, lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Points uniform on the 6 faces of an axis-aligned box, area-weighted."""
    ext = hi - lo
    areas = np.array([ext[1] * ext[2], ext[1] * ext[2], ext[0] * ext[2], ext[0] * ext[2], ext[0] * ext[1], ext[0] * ext[1]])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    pts = lo + rng.uniform(size=(n, 3)) * ext
    axis = face // 2
    side = face % 2
    pts[np.arange(n), axis] = np.where(side == 0, lo[axis], hi[axis])
    return pts


def room_scene(n: int, seed: int, surface_frac: float = 0.7, sh_degree: int = 3) -> Scene:
    """Egocentric room: `surface_frac` of the means on the walls/floor/ceiling, the rest uniform inside."""
    rng = np.random.default_rng(seed)
    n_surf = int(round(surface_frac * n))
    surf = _box_surface_points(rng, n_surf, -ROOM_HALF, ROOM_HALF)
    inner = rng.uniform(-ROOM_HALF, ROOM_HALF, size=(n - n_surf, 3))
    means = np.concatenate([surf, inner], axis=0)
    means = means[rng.permutation(n)]
    scales, quats, opacity, sh = _attributes(rng, n, sh_degree)
    return Scene(means.astype(np.float32), scales, quats, opacity, sh, sh_degree)


def corridor_scene(n: int, seed: int, rooms: int = 5, room_len: float = 12.0, sh_degree: int = 3) -> Scene:
    """Roaming layout: `rooms` boxes of 8 x 3 x room_len m chained along +z (a 60 m corridor of rooms), 70 % of
    the means on the walls, floor and ceiling, 30 % inside; a 2 x 2.1 m doorway is cut into every wall that two
    rooms share (the surface points there are moved inside the rooms), so poses along the centre line see through."""
    rng = np.random.default_rng(seed)
    half = np.array([4.0, 1.5, room_len / 2.0])
    n_surf = int(round(0.7 * n))
    which = rng.integers(0, rooms, size=n)
    centers = np.stack([np.zeros(rooms), np.zeros(rooms), (np.arange(rooms) + 0.5) * room_len], axis=1)
    surf = _box_surface_points(rng, n_surf, -half, half)
    inner = rng.uniform(-half, half, size=(n - n_surf, 3))
    local = np.concatenate([surf, inner], axis=0)
    # doorways: |x| < 1, y from the floor (+1.5, y points down) up to 2.1 m above it, on shared z walls
    on_wall = np.abs(np.abs(local[:, 2]) - half[2]) < 1e-9
    shared = np.where(local[:, 2] > 0, which < rooms - 1, which > 0)
    door = on_wall & shared & (np.abs(local[:, 0]) < 1.0) & (local[:, 1] > 1.5 - 2.1)
    local[door] = rng.uniform(-half, half, size=(int(door.sum()), 3))
    means = local + centers[which]
    scales, quats, opacity, sh = _attributes(rng, n, sh_degree)
    return Scene(means.astype(np.float32), scales, quats, opacity, sh, sh_degree)


def perturbed_copy(scene: Scene, seed: int, mean_std: float = 0.01, dc_std: float = 0.05) -> Scene:
    """Copy with means + N(0, mean_std) and SH DC + N(0, dc_std): the source of a training target image."""
    rng = np.random.default_rng(seed)
    s = scene.subset(slice(None))
    s.means = (s.means + rng.normal(0.0, mean_std, size=s.means.shape)).astype(np.float32)
    s.sh[:, 0, :] = (s.sh[:, 0, :] + rng.normal(0.0, dc_std, size=s.sh[:, 0, :].shape)).astype(np.float32)
    return s


# ---------------------------------------------------------------- poses (world -> camera, 4x4 row-major T_cw)

def _rot_y(a: float) -> np.ndarray:
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def viewmat_from(rot_cw: np.ndarray, cam_center: np.ndarray) -> np.ndarray:
    """T_cw with rotation `rot_cw` (world->camera) for a camera centred at `cam_center` (world)."""
    m = np.eye(4)
    m[:3, :3] = rot_cw
    m[:3, 3] = -rot_cw @ cam_center
    return m


def identity_viewmats(v: int = 1) -> np.ndarray:
    return np.repeat(np.eye(4, dtype=np.float32)[None], v, axis=0)


def room_viewmats(v: int, seed: int, radius: float = 1.0) -> np.ndarray:
    """`v` cameras uniform in a ball of `radius` around the room centre, random yaw about the y axis."""
    rng = np.random.default_rng(seed)
    out = np.empty((v, 4, 4))
    for i in range(v):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        c = d * radius * np.cbrt(rng.uniform())
        out[i] = viewmat_from(_rot_y(rng.uniform(0.0, 2.0 * np.pi)).T, c)
    return out.astype(np.float32)


def corridor_viewmats(v: int, seed: int, rooms: int = 5, room_len: float = 12.0) -> np.ndarray:
    """`v` cameras at equal arc length along the corridor centre line, random yaw."""
    rng = np.random.default_rng(seed)
    zs = (np.arange(v) + 0.5) * (rooms * room_len / v)
    out = np.empty((v, 4, 4))
    for i in range(v):
        out[i] = viewmat_from(_rot_y(rng.uniform(0.0, 2.0 * np.pi)).T, np.array([0.0, 0.0, zs[i]]))
    return out.astype(np.float32)


def random_viewmats(v: int, seed: int, max_offset: float = 0.3) -> np.ndarray:
    """Random full rotations (uniform on SO(3), drawn by scipy) and small offsets around the origin."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    rots = Rotation.random(v, random_state=rng).as_matrix()
    out = np.empty((v, 4, 4))
    for i in range(v):
        out[i] = viewmat_from(rots[i], rng.uniform(-max_offset, max_offset, size=3))
    return out.astype(np.float32)


def cube_face_viewmats(viewmats: np.ndarray) -> np.ndarray:
    """Six 90-degree pinhole views per pose (the faces of a cube map: looking along +z, +x, -z, -x, -y, +y of each
    camera), pose-major: the perspective split of an equirectangular capture."""
    faces = []
    for yaw in (0.0, 0.5 * np.pi, np.pi, 1.5 * np.pi):
        faces.append(_rot_y(yaw))
    c, s = np.cos(0.5 * np.pi), np.sin(0.5 * np.pi)
    faces.append(np.array([[1, 0, 0], [0, c, -s], [0, s, c]]))   # looking up (-y, y points down)
    faces.append(np.array([[1, 0, 0], [0, c, s], [0, -s, c]]))   # looking down
    out = []
    for vm in np.asarray(viewmats, np.float64):
        for F in faces:
            m = np.eye(4)
            m[:3, :3] = F @ vm[:3, :3]
            m[:3, 3] = F @ vm[:3, 3]
            out.append(m)
    return np.array(out, np.float32)


# ---------------------------------------------------------------- projected splats for stage-level tests

SPLAT_FIELDS = ("px", "py", "c0", "c1", "c2", "opacity", "r", "g", "b", "depth", "rx", "ry")


def random_splats(v: int, n: int, width: int, height: int, seed: int, *, max_radius: int = 40,
                  opacity_range=(0.05, 0.99), depth_ties: float = 0.1, cull_frac: float = 0.05,
                  seam_frac: float = 0.1, pole_frac: float = 0.05, wide_frac: float = 0.02,
                  aniso_frac: float = 0.4) -> dict:
    """Per-(view, Gaussian) screen-space records drawn directly (not projected from 3D).

    Each record is a centre (px, py) in [0, W) x [0, H), an instance box of half-extents (rx, ry), an SPD inverse
    covariance (c0, c1, c2) whose 3-sigma ellipse fits inside that box (standard deviations along x and y at most
    rx / 3 and ry / 3, any correlation), an opacity, an RGB colour and a depth. A fraction of the boxes is
    anisotropic (ry drawn below rx or the other way round), and a fraction of the records is placed on the longitude
    seam, near the poles, made wider than the image, or culled (rx = ry = 0); a fraction shares its depth with
    another record so that ties occur. Arrays are float32 (rx, ry int32), flattened over (view, Gaussian).
    """
    rng = np.random.default_rng(seed)
    m = v * n
    px = rng.uniform(0.0, width, size=m)
    py = rng.uniform(0.0, height, size=m)
    seam = rng.uniform(size=m) < seam_frac
    px[seam] = np.where(rng.uniform(size=seam.sum()) < 0.5, rng.uniform(0, 3, size=seam.sum()),
                        width - rng.uniform(1e-3, 3, size=seam.sum()))
    pole = rng.uniform(size=m) < pole_frac
    py[pole] = np.where(rng.uniform(size=pole.sum()) < 0.5, rng.uniform(0, 2, size=pole.sum()),
                        height - rng.uniform(1e-3, 2, size=pole.sum()))
    rx = rng.integers(1, max_radius + 1, size=m)
    ry = rx.copy()
    aniso = rng.uniform(size=m) < aniso_frac
    short = rng.integers(1, max_radius + 1, size=m)
    flip = rng.uniform(size=m) < 0.5
    ry[aniso & ~flip] = np.minimum(rx, short)[aniso & ~flip]
    rx[aniso & flip] = np.minimum(ry, short)[aniso & flip]
    wide = rng.uniform(size=m) < wide_frac
    rx[wide] = rng.integers(width // 2, width + 8, size=wide.sum())
    # standard deviations along x and y no larger than a third of the half-extents (at least 0.3 px)
    sx = np.maximum(rx / 3.0 * rng.uniform(0.3, 1.0, size=m), 0.3)
    sy = np.maximum(ry / 3.0 * rng.uniform(0.3, 1.0, size=m), 0.3)
    sx = np.minimum(sx, rx / 3.0)
    sy = np.minimum(sy, ry / 3.0)
    rho = rng.uniform(-0.9, 0.9, size=m)
    s00, s11, s01 = sx * sx, sy * sy, rho * sx * sy
    det = s00 * s11 - s01 * s01
    c0, c1, c2 = s11 / det, -s01 / det, s00 / det
    opacity = rng.uniform(*opacity_range, size=m)
    rgb = rng.uniform(0.0, 1.0, size=(m, 3))
    depth = rng.uniform(0.2, 20.0, size=m)
    tie = rng.uniform(size=m) < depth_ties
    depth[tie] = depth[rng.integers(0, m, size=tie.sum())]
    cull = rng.uniform(size=m) < cull_frac
    rx[cull] = 0
    ry[cull] = 0
    f32 = np.float32
    return dict(px=px.astype(f32), py=py.astype(f32), c0=c0.astype(f32), c1=c1.astype(f32), c2=c2.astype(f32),
                opacity=opacity.astype(f32), r=rgb[:, 0].astype(f32), g=rgb[:, 1].astype(f32),
                b=rgb[:, 2].astype(f32), depth=depth.astype(f32), rx=rx.astype(np.int32), ry=ry.astype(np.int32))


def random_image_grad(v: int, width: int, height: int, seed: int) -> np.ndarray:
    """Upstream gradient dL/dC ~ N(0, 1), layout [V, 3, H, W]."""
    return np.random.default_rng(seed).normal(size=(v, 3, height, width)).astype(np.float32)


def random_image(v: int, width: int, height: int, seed: int) -> np.ndarray:
    """A target image with values uniform in [0, 1], layout [V, 3, H, W]."""
    return np.random.default_rng(seed).uniform(size=(v, 3, height, width)).astype(np.float32)
