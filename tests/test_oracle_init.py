"""Pins of the oracle's default initialisation of new primitives (Sec. 3.3.1
densification at keypoints; the 3D-Gaussian-splatting convention as the
reading): nearest-neighbour scale on lattices whose neighbour distances are
known exactly, back-projection checked by projecting forward again, the DC
colour checked through the oracle's own spherical-harmonics evaluation
(Legendre-derived basis), pixel rounding and degenerate maps."""
import numpy as np
import pytest

import oracle
import synthetic as S


def _cam_identity(W=64, H=48, f=50.0):
    return S.Camera(np.eye(3), np.zeros(3), f, f, W / 2.0, H / 2.0, W, H)


def _kp_for(points, cam):
    """Exact keypoints (u, v, depth, 0, 0) of world points seen by `cam`."""
    pc = points @ cam.R.T + cam.t
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    return np.stack([u, v, pc[:, 2], np.zeros(len(u)), np.zeros(len(u))], 1).astype(np.float32)


def _lattice(a, n=5, origin=(-0.2, -0.2, 2.0)):
    g = np.arange(n) * a
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1) + np.asarray(origin)


def test_lattice_site_has_log_spacing_scale():
    a = 0.125
    pts = _lattice(a)
    cam = _cam_identity()
    site = 62  # interior site (2, 2, 2) of the 5^3 lattice: six neighbours at distance a
    kp = _kp_for(pts[site:site + 1], cam)
    img = np.zeros((3, cam.height, cam.width))
    out = oracle.default_init(img, kp, cam.as_array(), pts, site)
    assert np.allclose(out["logscale"], np.log(a), atol=1e-6)


def test_cube_centre_has_log_half_diagonal_scale():
    a = 0.25
    pts = _lattice(a, n=4)
    centre = pts[0] + a * np.array([1.5, 1.5, 1.5])  # centre of an interior cube: 8 corners at a sqrt(3) / 2
    cam = _cam_identity()
    ref = np.vstack([pts, centre[None]])
    kp = _kp_for(centre[None], cam)
    out = oracle.default_init(np.zeros((3, cam.height, cam.width)), kp, cam.as_array(), ref, len(pts))
    assert np.allclose(out["logscale"], np.log(a * np.sqrt(3.0) / 2.0), atol=1e-6)


def test_sparse_maps():
    cam = _cam_identity()
    p = np.array([[0.1, -0.05, 2.5]])
    kp = _kp_for(p, cam)
    img = np.zeros((3, cam.height, cam.width))
    alone = oracle.default_init(img, kp, cam.as_array(), p, 0)
    assert np.allclose(alone["logscale"], np.log(0.01))   # no other point: 1 cm
    other = np.array([[0.1 + 0.3, -0.05, 2.5]])
    two = oracle.default_init(img, kp, cam.as_array(), np.vstack([p, other]), 0)
    assert np.allclose(two["logscale"], np.log(0.3), atol=1e-6)  # one neighbour: its distance
    dup = oracle.default_init(img, kp, cam.as_array(), np.vstack([p, p]), 0)
    assert np.allclose(dup["logscale"], 0.5 * np.log(1e-7))       # coincident points: the floor


def test_back_projection_round_trip_and_fixed_fields():
    rng = np.random.default_rng(4)
    cam = S.pose_camera((0.3, -0.2, 0.1), 0.4, 300.0, 280.0, 320, 240)
    kp = np.stack([rng.uniform(0, 320, 20), rng.uniform(0, 240, 20), rng.uniform(0.5, 4.0, 20),
                   np.zeros(20), np.zeros(20)], 1).astype(np.float32)
    ref = rng.uniform(-2, 2, (50, 3))
    out = oracle.default_init(rng.uniform(0, 1, (3, 240, 320)), kp, cam.as_array(), np.vstack([ref, np.zeros((20, 3))]),
                              50)
    ca = cam.as_array().astype(np.float64)
    R, t = ca[:9].reshape(3, 3), ca[9:12]
    pc = out["mean"] @ R.T + t
    # R is stored in FP32, so R^T inverts it only to ~1e-7: the round trip holds to that
    assert np.allclose(pc[:, 2], kp[:, 2], rtol=1e-6)
    assert np.allclose(ca[12] * pc[:, 0] / pc[:, 2] + ca[14], kp[:, 0], atol=1e-4)
    assert np.allclose(ca[13] * pc[:, 1] / pc[:, 2] + ca[15], kp[:, 1], atol=1e-4)
    assert np.all(out["quat"] == np.array([1.0, 0.0, 0.0, 0.0]))
    assert np.allclose(1.0 / (1.0 + np.exp(-out["logit"])), 0.1, rtol=1e-14)
    assert np.all(out["sh"][:, 3:] == 0.0)


@pytest.mark.parametrize("u,v,px,py", [(10.5, 7.49, 11, 7), (10.4999, 7.5, 10, 8), (-3.0, 500.0, 0, 47),
                                       (63.7, 0.2, 63, 0)])
def test_dc_colour_reproduces_the_keypoint_pixel(u, v, px, py):
    """The oracle's SH evaluation (basis from associated Legendre functions)
    of the initialised primitive returns the pixel's colour in every view."""
    cam = _cam_identity()
    rng = np.random.default_rng(8)
    img = rng.uniform(0.05, 0.95, (3, cam.height, cam.width))
    kp = np.array([[u, v, 2.0, 0.0, 0.0]], np.float32)
    out = oracle.default_init(img, kp, cam.as_array(), np.zeros((1, 3)), 0)
    mo = np.concatenate([out["mean"], out["logit"][:, None]], 1)
    ls = np.concatenate([out["logscale"], np.zeros((1, 1))], 1)
    sh = out["sh"].reshape(1, 12, 4).transpose(1, 0, 2).copy()
    sc = oracle.Scene64(mo, out["quat"], ls, sh, 3)
    for view in (cam, S.pose_camera((0.5, 0.2, -1.0), 0.7, 50.0, 50.0, 64, 48)):
        pr = oracle.project(sc, view.as_array(), view.width, view.height, np.ones(1, np.uint8))
        assert np.allclose(pr[0, 13:16], img[:, py, px], atol=1e-12)


def test_three_nearest_by_mean_square():
    """Neighbours at 0.1, 0.2, 0.3, 0.4 m: the scale is sqrt((0.01 + 0.04 +
    0.09) / 3), not the mean distance (0.2) nor any other neighbour count."""
    cam = _cam_identity()
    q = np.array([0.05, 0.02, 2.2])
    ref = np.vstack([q, q + [0.1, 0, 0], q + [0, -0.2, 0], q + [0, 0, 0.3], q + [-0.4, 0, 0]])
    out = oracle.default_init(np.zeros((3, cam.height, cam.width)), _kp_for(q[None], cam), cam.as_array(), ref, 0)
    assert np.allclose(out["logscale"], 0.5 * np.log((0.01 + 0.04 + 0.09) / 3.0), atol=1e-6)
