"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: it only draws parameters,
poses and images from seeded numpy generators, in the shapes of the scenes the
paper evaluates on (Replica-sized 1200x680 monocular frames, TUM-sized 640x480
RGB-D frames).  The datasets themselves are not available; these scenes stand
in for them.

Scene recipe (every count, distribution and seed is fixed here):
  tiny       4,096 Gaussians, means uniform in a 2 m cube centred at (0, 0, 3),
             160x120 camera, fx = fy = 150, identity pose.
  room       Gaussians uniform in a 6 x 3 x 4 m room centred at the origin
             (x in [-3, 3], y in [-1.5, 1.5], z in [-2, 2]).
  common     log-scales N(-4, 0.5); unit quaternions = normalised N(0, I4);
             opacity logits N(0, 1); SH DC U(-1, 1), higher bands N(0, 0.1).
  perturbed  every parameter + N(0, 0.05) (seed 1); targets render the
             unperturbed set.
  trajectory Lissajous path inside the central 2 x 1 x 1 m, yaw within +-60
             degrees (seed 2), 50 poses.
Seeds: scene 0, perturbation 1, trajectory 2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SH_PLANES = 12  # 48 floats per Gaussian as 12 float4 planes


@dataclass
class Params:
    mean_op: np.ndarray   # (N, 4) float32: x, y, z, opacity logit
    quat: np.ndarray      # (N, 4) float32: w, x, y, z
    logscale: np.ndarray  # (N, 4) float32: 3 log-scales + zero pad
    sh: np.ndarray        # (12, N, 4) float32: coefficient-major SH

    @property
    def n(self) -> int:
        return self.mean_op.shape[0]

    def copy(self) -> "Params":
        return Params(self.mean_op.copy(), self.quat.copy(), self.logscale.copy(), self.sh.copy())


@dataclass
class Camera:
    R: np.ndarray  # (3, 3) world -> camera rotation
    t: np.ndarray  # (3,) world -> camera translation
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_array(self) -> np.ndarray:
        """16 float32: R row-major, t, fx, fy, cx, cy."""
        return np.concatenate([self.R.reshape(9), self.t.reshape(3),
                               [self.fx, self.fy, self.cx, self.cy]]).astype(np.float32)


def _draw(rng: np.random.Generator, n: int, lo, hi) -> Params:
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    mean = lo + (hi - lo) * rng.random((n, 3))
    opac = rng.standard_normal(n)
    ls = rng.normal(-4.0, 0.5, (n, 3))
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    sh48 = np.empty((n, 48))
    sh48[:, 0:3] = rng.uniform(-1.0, 1.0, (n, 3))
    sh48[:, 3:] = rng.normal(0.0, 0.1, (n, 45))
    return Params(
        mean_op=np.concatenate([mean, opac[:, None]], 1).astype(np.float32),
        quat=q.astype(np.float32),
        logscale=np.concatenate([ls, np.zeros((n, 1))], 1).astype(np.float32),
        sh=np.ascontiguousarray(sh48.reshape(n, SH_PLANES, 4).transpose(1, 0, 2)).astype(np.float32),
    )


def tiny_scene(n: int = 4096, seed: int = 0) -> Params:
    rng = np.random.default_rng(seed)
    return _draw(rng, n, (-1.0, -1.0, 2.0), (1.0, 1.0, 4.0))


def room_scene(n: int, seed: int = 0) -> Params:
    rng = np.random.default_rng(seed)
    return _draw(rng, n, (-3.0, -1.5, -2.0), (3.0, 1.5, 2.0))  # ROOM_LO, ROOM_HI


ROOM_LO, ROOM_HI = (-3.0, -1.5, -2.0), (3.0, 1.5, 2.0)  # the 6 x 3 x 4 m room


def _quat_from_matrix(R: np.ndarray) -> np.ndarray:
    """(N, 3, 3) rotations -> (N, 4) unit quaternions (w, x, y, z), w >= 0."""
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    q = np.empty((R.shape[0], 4))
    # Shepperd's method: take the largest of 4w^2, 4x^2, 4y^2, 4z^2
    c = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1)
    k = c.argmax(1)
    for i in range(R.shape[0]):
        r = R[i]
        if k[i] == 0:
            w = np.sqrt(1.0 + tr[i]) / 2
            q[i] = [w, (r[2, 1] - r[1, 2]) / (4 * w), (r[0, 2] - r[2, 0]) / (4 * w), (r[1, 0] - r[0, 1]) / (4 * w)]
        elif k[i] == 1:
            x = np.sqrt(1.0 + r[0, 0] - r[1, 1] - r[2, 2]) / 2
            q[i] = [(r[2, 1] - r[1, 2]) / (4 * x), x, (r[0, 1] + r[1, 0]) / (4 * x), (r[0, 2] + r[2, 0]) / (4 * x)]
        elif k[i] == 2:
            y = np.sqrt(1.0 - r[0, 0] + r[1, 1] - r[2, 2]) / 2
            q[i] = [(r[0, 2] - r[2, 0]) / (4 * y), (r[0, 1] + r[1, 0]) / (4 * y), y, (r[1, 2] + r[2, 1]) / (4 * y)]
        else:
            z = np.sqrt(1.0 - r[0, 0] - r[1, 1] + r[2, 2]) / 2
            q[i] = [(r[1, 0] - r[0, 1]) / (4 * z), (r[0, 2] + r[2, 0]) / (4 * z), (r[1, 2] + r[2, 1]) / (4 * z), z]
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    return q


def wall_scene(n: int, seed: int = 0) -> Params:
    """The room's Gaussians on its six walls instead of filling its volume
    (surface-like, as indoor scenes are): faces drawn by area, positions
    uniform on the face with 1 cm of normal jitter, two in-plane log-scales
    N(-4, 0.5) and a 2 mm thickness along the wall normal (the local z axis,
    turned onto the normal with a random spin about it), opacity logits
    N(1, 1), colours as in room_scene."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(ROOM_LO), np.asarray(ROOM_HI)
    size = hi - lo
    faces = []  # (axis, side)
    areas = []
    for ax in range(3):
        o = [a for a in range(3) if a != ax]
        for side in (0, 1):
            faces.append((ax, side))
            areas.append(size[o[0]] * size[o[1]])
    areas = np.asarray(areas) / np.sum(areas)
    f = rng.choice(len(faces), size=n, p=areas)
    mean = lo + size * rng.random((n, 3))
    normal = np.zeros((n, 3))
    for i, (ax, side) in enumerate(faces):
        sel = f == i
        mean[sel, ax] = (hi[ax] if side else lo[ax])
        normal[sel, ax] = -1.0 if side else 1.0  # pointing into the room
    mean += normal * rng.normal(0.0, 0.01, (n, 1))
    # rotation taking e_z to the face normal (one per face), then a random
    # spin about the normal: q = q_face * (cos(th/2), 0, 0, sin(th/2))
    ez = np.array([0.0, 0.0, 1.0])
    Rf = np.empty((len(faces), 3, 3))
    for i, (ax, side) in enumerate(faces):
        nz = np.zeros(3)
        nz[ax] = -1.0 if side else 1.0
        a = np.cross(ez, nz)
        s_, c_ = np.linalg.norm(a), float(ez @ nz)
        if s_ < 1e-12:
            Rf[i] = np.eye(3) if c_ > 0 else np.diag([1.0, -1.0, -1.0])
        else:
            K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]]) / s_
            ang = np.arctan2(s_, c_)
            Rf[i] = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * (K @ K)
    qf = _quat_from_matrix(Rf)[f]
    th = rng.uniform(0, 2 * np.pi, n)
    cs, sn = np.cos(th / 2), np.sin(th / 2)
    w1, x1, y1, z1 = qf.T
    q = np.stack([w1 * cs - z1 * sn, x1 * cs + y1 * sn, y1 * cs - x1 * sn, z1 * cs + w1 * sn], 1)
    ls = np.empty((n, 3))
    ls[:, :2] = rng.normal(-4.0, 0.5, (n, 2))
    ls[:, 2] = np.log(0.002)
    opac = rng.normal(1.0, 1.0, n)
    sh48 = np.empty((n, 48))
    sh48[:, 0:3] = rng.uniform(-1.0, 1.0, (n, 3))
    sh48[:, 3:] = rng.normal(0.0, 0.1, (n, 45))
    return Params(
        mean_op=np.concatenate([mean, opac[:, None]], 1).astype(np.float32),
        quat=q.astype(np.float32),
        logscale=np.concatenate([ls, np.zeros((n, 1))], 1).astype(np.float32),
        sh=np.ascontiguousarray(sh48.reshape(n, SH_PLANES, 4).transpose(1, 0, 2)).astype(np.float32),
    )


def perturb(p: Params, sigma: float = 0.05, seed: int = 1) -> Params:
    rng = np.random.default_rng(seed)
    q = p.copy()
    q.mean_op += rng.normal(0, sigma, q.mean_op.shape).astype(np.float32)
    q.quat += rng.normal(0, sigma, q.quat.shape).astype(np.float32)
    q.logscale[:, :3] += rng.normal(0, sigma, (p.n, 3)).astype(np.float32)
    q.sh += rng.normal(0, sigma, q.sh.shape).astype(np.float32)
    return q


def tiny_camera() -> Camera:
    return Camera(np.eye(3), np.zeros(3), 150.0, 150.0, 80.0, 60.0, 160, 120)


def _yaw(theta: float) -> np.ndarray:
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def pose_camera(position, yaw, fx, fy, width, height) -> Camera:
    """Camera at `position` looking along +z rotated by `yaw` about +y."""
    Rcw = _yaw(yaw)               # camera -> world
    R = Rcw.T                     # world -> camera
    t = -R @ np.asarray(position, np.float64)
    return Camera(R, t, float(fx), float(fy), width / 2.0, height / 2.0, int(width), int(height))


def trajectory(k: int, n_poses: int = 50, seed: int = 2):
    """(position, yaw) of pose k on the seeded Lissajous path."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, 4)
    s = 2 * np.pi * (k % n_poses) / n_poses
    pos = np.array([1.0 * np.sin(s + ph[0]), 0.5 * np.sin(2 * s + ph[1]), 0.5 * np.sin(3 * s + ph[2])])
    yaw = (np.pi / 3) * np.sin(s + ph[3])
    return pos, yaw


def replica_camera(k: int = 0) -> Camera:
    """1200x680, fx = fy = 600: the Replica frame shape, on the trajectory."""
    pos, yaw = trajectory(k)
    return pose_camera(pos, yaw, 600.0, 600.0, 1200, 680)


def tum_camera(k: int = 0) -> Camera:
    """640x480, fx = fy = 525: the TUM RGB-D frame shape, on the trajectory."""
    pos, yaw = trajectory(k)
    return pose_camera(pos, yaw, 525.0, 525.0, 640, 480)


def camera_at_level(cam: Camera, level: int) -> Camera:
    """Intrinsics of pyramid level `level` (each level halves, sizes round up)."""
    s = 2 ** level
    w, h = cam.width, cam.height
    for _ in range(level):
        w, h = (w + 1) // 2, (h + 1) // 2
    return Camera(cam.R, cam.t, cam.fx / s, cam.fy / s, cam.cx / s, cam.cy / s, w, h)


def random_image(C: int, H: int, W: int, seed: int = 5, smooth: int = 2) -> np.ndarray:
    """Seeded image in [0, 1], box-smoothed noise (float32, planar C x H x W)."""
    rng = np.random.default_rng(seed)
    x = rng.random((C, H + 2 * smooth, W + 2 * smooth))
    if smooth > 0:
        k = 2 * smooth + 1
        c = np.cumsum(np.cumsum(np.pad(x, ((0, 0), (1, 0), (1, 0))), 1), 2)
        x = (c[:, k:, k:] - c[:, :-k, k:] - c[:, k:, :-k] + c[:, :-k, :-k]) / (k * k)
    return np.ascontiguousarray(x[:, :H, :W]).astype(np.float32)


def random_grad_image(C: int, H: int, W: int, seed: int = 6) -> np.ndarray:
    """Seeded upstream gradient dL/dimage, N(0, 1) (float32, planar)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((C, H, W)).astype(np.float32)


# ---------------------------------------------------------------- keypoints
def project_points(xyz: np.ndarray, cam: Camera):
    """(u, v, depth) of world points in `cam` (FP64)."""
    pc = np.asarray(xyz, np.float64) @ np.asarray(cam.R, np.float64).T + np.asarray(cam.t, np.float64)
    z = pc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = cam.fx * pc[:, 0] / z + cam.cx
        v = cam.fy * pc[:, 1] / z + cam.cy
    return u, v, z


def orb_angle(img: np.ndarray, u: float, v: float, half: int = 8) -> float:
    """Orientation of a keypoint by the intensity centroid of the 16 x 16
    luminance patch around it (the ORB definition): atan2(m01, m10)."""
    C, H, W = img.shape
    lum = 0.299 * img[0] + 0.587 * img[1] + 0.114 * img[2]
    cx, cy = int(round(u)), int(round(v))
    ys = np.clip(np.arange(cy - half, cy + half), 0, H - 1)
    xs = np.clip(np.arange(cx - half, cx + half), 0, W - 1)
    patch = lum[np.ix_(ys, xs)]
    off = np.arange(-half, half) + 0.5
    m10 = float((patch * off[None, :]).sum())
    m01 = float((patch * off[:, None]).sum())
    return float(np.arctan2(m01, m10))


def held_out_keypoints(p: Params, cams, per_keyframe: int, seed: int = 5, margin: float = 8.0,
                       min_depth: float = 0.5):
    """Seeded held-out primitives for densification tests: for each keyframe in
    turn, `per_keyframe` (None: all) not-yet-chosen Gaussians whose centre
    projects inside the image (with a margin) in front of the camera.  Returns a list of
    (indices, keypoints (M, 5) float32 without angles) per keyframe; the
    keypoint is the exact projection of the centre, with its depth."""
    rng = np.random.default_rng(seed)
    taken = np.zeros(p.n, bool)
    out = []
    for cam in cams:
        u, v, z = project_points(p.mean_op[:, :3], cam)
        ok = (~taken) & (z > min_depth) & (u >= margin) & (u <= cam.width - 1 - margin) & (v >= margin) & \
             (v <= cam.height - 1 - margin)
        cand = np.flatnonzero(ok)
        take = len(cand) if per_keyframe is None else min(per_keyframe, len(cand))
        pick = np.sort(rng.choice(cand, size=take, replace=False))
        taken[pick] = True
        kp = np.stack([u[pick], v[pick], z[pick], np.zeros(len(pick)), np.zeros(len(pick))], 1).astype(np.float32)
        out.append((pick, kp))
    return out


def densify_scene(p: Params, cams, per_keyframe: int, seed: int):
    """The map layout of a densification experiment: `p` permuted so that the
    held-out primitives of keyframe k (chosen by held_out_keypoints) occupy
    slots offsets[k] .. offsets[k] + M_k - 1 at the end of the map.  Returns
    (permuted params, offsets, keypoints per keyframe (M_k, 5) float32)."""
    held = held_out_keypoints(p, cams, per_keyframe, seed=seed)
    new = np.concatenate([h[0] for h in held]) if held else np.zeros(0, np.int64)
    rest = np.setdiff1d(np.arange(p.n), new)
    order = np.concatenate([rest, new]).astype(np.int64)
    q = Params(p.mean_op[order].copy(), p.quat[order].copy(), p.logscale[order].copy(), p.sh[:, order].copy())
    offsets, off = [], len(rest)
    for idx, _ in held:
        offsets.append(off)
        off += len(idx)
    return q, offsets, [h[1] for h in held]


def stereo_pair(k: int, baseline: float = 0.11, f: float = 376.0, width: int = 752, height: int = 480):
    """(left, right) cameras of a rectified stereo rig at pose k of the
    trajectory: the right camera sits `baseline` metres along the left
    camera's +x axis (EuRoC-shaped 752 x 480 monochrome views)."""
    pos, yaw = trajectory(k)
    left = pose_camera(pos, yaw, f, f, width, height)
    right = Camera(left.R.copy(), left.t - np.array([baseline, 0.0, 0.0]), left.fx, left.fy, left.cx, left.cy,
                   width, height)
    return left, right
