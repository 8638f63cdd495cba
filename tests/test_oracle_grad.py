"""Finite-difference pins for the oracle's analytic backward (Eq. 3 and Eq. 4 gradients).

Tiny scenes (<= 8 Gaussians, 16 x 16 pixels) whose discrete decisions (cull,
pixel box, alpha clamp / skip, termination, colour clamp, Jacobian clamp) do
not move under the +-h perturbation: the FP32 decision set is frozen from the
unperturbed parameters and the oracle's reported margins are checked.  Every
one of the 59 parameters of every Gaussian is differentiated.
"""
import numpy as np
import pytest

import oracle
import synthetic as S

W = H = 16


def _cam():
    return oracle.camera_array(np.eye(3), np.zeros(3), 20.0, 20.0, 8.0, 8.0)


def _scene(seed, n=7, with_clamped_jacobian=True, opaque=False):
    rng = np.random.default_rng(seed)
    mean_op = np.zeros((n, 4), np.float32)
    mean_op[:, 0:2] = rng.uniform(-0.5, 0.5, (n, 2))
    mean_op[:, 2] = rng.uniform(2.5, 3.5, n)
    mean_op[:, 3] = rng.normal(0, 1, n)
    if opaque:
        mean_op[0, 3] = 7.0
    if with_clamped_jacobian:
        mean_op[n - 1, 0:3] = [1.8, 0.1, 3.0]  # x/z = 0.6 beyond the 1.3 tan(fov/2) clamp
    quat = rng.standard_normal((n, 4)).astype(np.float32)
    ls = np.zeros((n, 4), np.float32)
    ls[:, :3] = np.log(rng.uniform(0.12, 0.3, (n, 3)))
    if with_clamped_jacobian:
        ls[n - 1, :3] = np.log(0.5)
    sh = np.zeros((n, 48))
    sh[:, 0:3] = rng.uniform(0.5, 1.5, (n, 3))
    sh[:, 3:] = rng.normal(0, 0.15, (n, 45))
    sh = np.ascontiguousarray(sh.reshape(n, 12, 4).transpose(1, 0, 2)).astype(np.float32)
    return mean_op, quat, ls, sh


def _flat(sc):
    return [sc.mean_op, sc.quat, sc.logscale, sc.sh]


def _fd_grad(fun, sc, h=1e-6):
    """Central differences of fun(sc) w.r.t. every parameter, in the (N, 60) layout."""
    n = sc.n
    out = np.zeros((n, 60))
    arrays = _flat(sc)
    for a_idx, arr in enumerate(arrays):
        for idx in np.ndindex(arr.shape):
            if a_idx == 2 and idx[1] == 3:
                continue  # log-scale pad is not a parameter
            old = arr[idx]
            step = h * max(1.0, abs(old))
            arr[idx] = old + step
            fp = fun(sc)
            arr[idx] = old - step
            fm = fun(sc)
            arr[idx] = old
            g = (fp - fm) / (2 * step)
            if a_idx < 3:
                out[idx[0], 4 * a_idx + idx[1]] = g
            else:
                plane, i, e = idx
                out[i, 12 + 4 * plane + e] = g
    return out


def _setup(seed, flags, **kw):
    mean_op, quat, ls, sh = _scene(seed, **kw)
    cam = _cam()
    dec = oracle.decide(mean_op, quat, ls, cam, W, H)
    sc = oracle.Scene64(mean_op, quat, ls, sh)
    img, T, nc, mg = oracle.render(sc, cam, W, H, dec, flags=flags)
    pr = oracle.project(sc, cam, W, H, dec.visible)
    if flags == 0:
        assert mg.min() > 1e-3, "a pixel decision sits too close to its threshold for FD"
    assert np.abs(pr[dec.visible > 0, 13:16]).min() > 1e-3  # colour clamp inactive
    return cam, dec, sc, img


@pytest.mark.parametrize("seed,flags,opaque", [(1, oracle.NO_CLAMP | oracle.NO_SKIP | oracle.NO_TERM, False),
                                               (2, 0, False), (3, 0, True)])
def test_render_backward_matches_fd(seed, flags, opaque):
    cam, dec, sc, img = _setup(seed, flags, opaque=opaque)
    assert dec.visible.sum() == sc.n
    dimg = S.random_grad_image(3, H, W, seed=seed).astype(np.float64)

    def fun(s):
        im, _, _, _ = oracle.render(s, cam, W, H, dec, flags=flags)
        return float((dimg * im).sum())

    g, g2 = oracle.render_bwd(sc, cam, W, H, dec, dimg, flags=flags)
    fd = _fd_grad(fun, sc)
    scale = np.abs(fd).max()
    np.testing.assert_allclose(g, fd, rtol=2e-5, atol=2e-7 * scale)
    assert np.abs(g[:, 11]).max() == 0


def test_loss_through_render_matches_fd():
    cam, dec, sc, img = _setup(4, 0)
    gt = S.random_image(3, H, W, seed=9).astype(np.float64)
    assert np.abs(img - gt).min() > 1e-5

    def fun(s):
        im, _, _, _ = oracle.render(s, cam, W, H, dec)
        return oracle.loss(im, gt, 0.2, grad=False)

    _, dimg = oracle.loss(img, gt, 0.2)
    g, _ = oracle.render_bwd(sc, cam, W, H, dec, dimg)
    fd = _fd_grad(fun, sc)
    np.testing.assert_allclose(g, fd, rtol=2e-5, atol=2e-7 * np.abs(fd).max())


def test_chain_is_linear_in_screen_space_gradient():
    cam, dec, sc, img = _setup(5, 0)
    rng = np.random.default_rng(1)
    a, b = rng.standard_normal((sc.n, 9)), rng.standard_normal((sc.n, 9))
    ga, gb, gab = oracle.chain(sc, cam, W, H, dec, a), oracle.chain(sc, cam, W, H, dec, b), \
        oracle.chain(sc, cam, W, H, dec, 2 * a - b)
    np.testing.assert_allclose(gab, 2 * ga - gb, atol=1e-12)
