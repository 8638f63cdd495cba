"""The seeded input generators (no method arithmetic): keypoints of held-out
primitives project from their centres, the map permutation keeps every
Gaussian once, and the ORB intensity-centroid angle points at the bright
side of a patch."""
import numpy as np

import synthetic as S


def test_densify_scene_layout():
    p = S.room_scene(20000, seed=3)
    cams = [S.tum_camera(k * 50 // 4) for k in range(4)]
    q, offs, kps = S.densify_scene(p, cams, 300, seed=4)
    # a permutation: the same multiset of rows
    a = np.sort(p.mean_op.view(np.uint32).reshape(p.n, -1), axis=0)
    b = np.sort(q.mean_op.view(np.uint32).reshape(q.n, -1), axis=0)
    assert np.array_equal(a, b)
    assert offs == sorted(offs) and offs[-1] + len(kps[-1]) == p.n
    for off, kp, cam in zip(offs, kps, cams):
        u, v, z = S.project_points(q.mean_op[off:off + len(kp), :3], cam)
        assert np.allclose(u, kp[:, 0], atol=1e-3) and np.allclose(v, kp[:, 1], atol=1e-3)
        assert np.allclose(z, kp[:, 2], rtol=1e-6) and (z > 0.5).all()
        assert (kp[:, 0] >= 8).all() and (kp[:, 0] <= cam.width - 9).all()


def test_orb_angle_points_to_the_bright_side():
    img = np.zeros((3, 40, 40))
    img[:, :, 25:] = 1.0  # bright to the right of (20, 20)
    assert abs(S.orb_angle(img, 20, 20)) < 1e-9
    img = np.zeros((3, 40, 40))
    img[:, 25:, :] = 1.0  # bright below
    assert abs(S.orb_angle(img, 20, 20) - np.pi / 2) < 1e-9


def test_stereo_pair_baseline():
    left, right = S.stereo_pair(3)
    cl = -left.R.T @ left.t
    cr = -right.R.T @ right.t
    assert np.isclose(np.linalg.norm(cr - cl), 0.11)
    # the right centre lies along the left camera's x axis
    assert np.allclose(left.R @ (cr - cl), [0.11, 0.0, 0.0])


def test_wall_scene_lies_on_the_walls():
    """The sensitivity variant: every mean within the 1 cm jitter (5 sigma) of
    a wall of the room, the thin axis along that wall's normal (away from the
    room's edges, where the nearest wall is ambiguous), unit quaternions."""
    w = S.wall_scene(20000, seed=3)
    m = w.mean_op[:, :3].astype(np.float64)
    lo, hi = np.array(S.ROOM_LO), np.array(S.ROOM_HI)
    d = np.minimum(np.abs(m - lo), np.abs(m - hi))
    assert d.min(1).max() <= 0.05
    q = w.quat.astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-6)
    qw, x, y, z = q.T
    local_z = np.stack([2 * (x * z + qw * y), 2 * (y * z - qw * x), 1 - 2 * (x * x + y * y)], 1)
    ax = d.argmin(1)
    clear = np.sort(d, 1)[:, 1] > 0.1
    assert np.abs(local_z[np.arange(len(ax)), ax])[clear].min() > 0.9999
    assert np.allclose(w.logscale[:, 2], np.log(0.002))
