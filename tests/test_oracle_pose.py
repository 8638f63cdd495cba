"""Pins for the oracle's camera pose gradient (dL/dR, dL/dt and the
left-rotation gradient dL/dphi), the pose-refinement extension of the
render backward (the camera (R, t) of Eq. 3's projection is the variable).

* finite differences of the loss through the render (Eq. 3 and Eq. 4) with
  respect to every entry of R and t, the FP64 camera perturbed below FP32
  resolution so the FP32 decisions stay frozen;
* finite differences along exp([phi]x) applied to (R, t) (Rodrigues);
* the translation gauge: moving every mean by d and t by -R d changes
  nothing, so sum_i dL/dmean_i = R^T dL/dt exactly;
* the two forms agree: dL/dphi_k = <dL/dR, [e_k]x R> + dL/dt . (e_k x t).
"""
import numpy as np
import pytest

import oracle
import synthetic as S

W = H = 16


def _rot(axis, angle):
    """Rodrigues' formula."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


def _hat(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]], np.float64)


def _cam(R, t):
    return oracle.camera_array(R, t, 20.0, 20.0, 8.0, 8.0).astype(np.float64)


def _scene(seed, n=7):
    rng = np.random.default_rng(seed)
    mean_op = np.zeros((n, 4), np.float32)
    mean_op[:, 0:2] = rng.uniform(-0.45, 0.45, (n, 2))
    mean_op[:, 2] = rng.uniform(2.5, 3.5, n)
    mean_op[:, 3] = rng.normal(0, 1, n)
    mean_op[n - 1, 0:3] = [1.8, 0.1, 3.0]  # x/z = 0.6, beyond the Jacobian clamp
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    ls = np.zeros((n, 4), np.float32)
    ls[:, :3] = np.log(rng.uniform(0.12, 0.3, (n, 3)))
    ls[n - 1, :3] = np.log(0.5)
    sh = np.zeros((n, 48))
    sh[:, 0:3] = rng.uniform(0.5, 1.5, (n, 3))
    sh[:, 3:] = rng.normal(0, 0.15, (n, 45))
    sh = np.ascontiguousarray(sh.reshape(n, 12, 4).transpose(1, 0, 2)).astype(np.float32)
    return mean_op, quat, ls, sh


def _setup(seed, orthonormal=False):
    """orthonormal: R orthonormal in FP64 (the FP32 decisions then see its
    rounding); else R is FP32-representable."""
    mean_op, quat, ls, sh = _scene(seed)
    R = _rot((0.3, -1.0, 0.4), 0.06)
    t = np.array([0.04, -0.03, 0.08])
    cam = _cam(R, t)  # FP32-representable values, held in FP64
    if orthonormal:
        cam[:9] = R.reshape(9)
    dec = oracle.decide(mean_op, quat, ls, cam, W, H)
    sc = oracle.Scene64(mean_op, quat, ls, sh)
    img, _, _, mg = oracle.render(sc, cam, W, H, dec)
    assert dec.visible.sum() == sc.n
    assert mg.min() > 1e-3, "a pixel decision sits too close to its threshold for FD"
    pr = oracle.project(sc, cam, W, H, dec.visible)
    assert np.abs(pr[:, 13:16]).min() > 1e-3  # colour clamp inactive
    gt = S.random_image(3, H, W, seed=seed + 20).astype(np.float64)
    assert np.abs(img - gt).min() > 1e-5  # |.| of the L1 term differentiable
    return sc, dec, cam, img, gt


def _loss(sc, dec, cam, gt):
    im, _, _, _ = oracle.render(sc, cam, W, H, dec)
    return oracle.loss(im, gt, 0.2, grad=False)


def _analytic(sc, dec, cam, img, gt):
    _, dimg = oracle.loss(img, gt, 0.2)
    g, g2 = oracle.render_bwd(sc, cam, W, H, dec, dimg)
    return g, oracle.pose_grad(sc, cam, W, H, dec, g2)


@pytest.mark.parametrize("seed", [2, 7])
def test_pose_gradient_matches_fd_on_R_and_t(seed):
    sc, dec, cam, img, gt = _setup(seed)
    _, pose = _analytic(sc, dec, cam, img, gt)
    fd = np.zeros(12)
    h = 1e-6
    for k in range(12):
        cp, cm = cam.copy(), cam.copy()
        cp[k] += h
        cm[k] -= h
        fd[k] = (_loss(sc, dec, cp, gt) - _loss(sc, dec, cm, gt)) / (2 * h)
    print("analytic", pose[:12], "\nfd      ", fd)
    np.testing.assert_allclose(pose[:12], fd, rtol=2e-5, atol=2e-7 * np.abs(fd).max())
    assert np.abs(pose[:12]).max() > 1e-3  # not vacuous


@pytest.mark.parametrize("seed", [4, 8])
def test_pose_gradient_matches_fd_along_left_rotation(seed):
    sc, dec, cam, img, gt = _setup(seed)
    _, pose = _analytic(sc, dec, cam, img, gt)
    R, t = cam[:9].reshape(3, 3), cam[9:12]
    fd = np.zeros(3)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        vals = []
        for s in (h, -h):
            Q = _rot(e, s)
            c = cam.copy()
            c[:9] = (Q @ R).reshape(9)
            c[9:12] = Q @ t
            vals.append(_loss(sc, dec, c, gt))
        fd[k] = (vals[0] - vals[1]) / (2 * h)
    print("analytic", pose[12:], "\nfd      ", fd)
    np.testing.assert_allclose(pose[12:], fd, rtol=2e-5, atol=2e-7 * np.abs(fd).max())


def test_translation_gauge():
    sc, dec, cam, img, gt = _setup(4, orthonormal=True)
    g, pose = _analytic(sc, dec, cam, img, gt)
    R = cam[:9].reshape(3, 3)
    lhs = g[:, 0:3].sum(0)
    rhs = R.T @ pose[9:12]
    print(lhs, rhs)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-14 * np.abs(lhs).max())


def test_rotation_forms_agree():
    sc, dec, cam, img, gt = _setup(9)
    _, pose = _analytic(sc, dec, cam, img, gt)
    R, t = cam[:9].reshape(3, 3), cam[9:12]
    GR, Gt = pose[:9].reshape(3, 3), pose[9:12]
    via_raw = np.array([(GR * (_hat(e) @ R)).sum() + Gt @ np.cross(e, t) for e in np.eye(3)])
    np.testing.assert_allclose(pose[12:], via_raw, rtol=1e-9, atol=1e-12 * np.abs(via_raw).max())


def test_pose_gradient_is_linear_and_zero_without_screen_gradient():
    sc, dec, cam, img, gt = _setup(11)
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal((sc.n, 9)), rng.standard_normal((sc.n, 9))
    pa, pb, pab = (oracle.pose_grad(sc, cam, W, H, dec, x) for x in (a, b, 2 * a - b))
    np.testing.assert_allclose(pab, 2 * pa - pb, atol=1e-12 * np.abs(pab).max())
    assert np.abs(oracle.pose_grad(sc, cam, W, H, dec, np.zeros((sc.n, 9)))).max() == 0.0
