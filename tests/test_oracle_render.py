"""Closed-form pins for the oracle render (Eq. 3, with the product index read as (1 - alpha_j)).

On the optical axis with identity rotation J is diagonal, so one isotropic
Gaussian of scale s at depth z renders exactly
    sigma * c * exp(-rho^2 / (2 (f^2 s^2 / z^2 + 0.3)))
inside its 3-sigma pixel box.  Stacks of on-axis Gaussians give alpha_i =
sigma_i at the centre pixel, so the blend reduces to the closed product form.
"""
import math

import numpy as np
import pytest

import oracle

Y00 = 0.5 / math.sqrt(math.pi)
W = H = 33
F = 30.0


def _cam():
    return oracle.camera_array(np.eye(3), np.zeros(3), F, F, 16.0, 16.0)


def _gaussians(zs, scales, logits, dc):
    n = len(zs)
    mean_op = np.zeros((n, 4), np.float32)
    mean_op[:, 2] = zs
    mean_op[:, 3] = logits
    quat = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1))
    ls = np.zeros((n, 4), np.float32)
    ls[:, :3] = np.log(np.asarray(scales, np.float64))[:, None]
    sh = np.zeros((12, n, 4), np.float32)
    dcs = np.asarray(dc, np.float32).reshape(n, 3)
    sh[0, :, 0:3] = dcs
    return mean_op, quat, ls, sh


def _render(g, flags=0):
    mean_op, quat, ls, sh = g
    cam = _cam()
    dec = oracle.decide(mean_op, quat, ls, cam, W, H)
    sc = oracle.Scene64(mean_op, quat, ls, sh)
    return oracle.render(sc, cam, W, H, dec, flags=flags), dec, sc


def _sig(x):
    return 1 / (1 + math.exp(-x))


def test_single_isotropic_gaussian_profile():
    z, s, logit, dc = 3.0, 0.08, 0.3, (0.4, -0.2, 0.9)
    g = _gaussians([z], [s], [logit], [dc])
    (img, T, nc, mg), dec, sc = _render(g)
    s32 = float(np.float32(math.exp(float(np.float32(math.log(s))))))
    var = (F * s32 / z) ** 2 + 0.3
    # isotropic: the eigenvalue bound mid + sqrt(max(0.1, mid^2 - det)) is var + sqrt(0.1)
    r = math.ceil(3 * math.sqrt(var + math.sqrt(0.1)))
    assert dec.radius[0] == r
    sigma = _sig(float(np.float32(logit)))
    col = [max(0.0, Y00 * float(np.float32(c)) + 0.5) for c in dc]
    for py in range(H):
        for px in range(W):
            rho2 = (px - 16) ** 2 + (py - 16) ** 2
            a = sigma * math.exp(-rho2 / (2 * var))
            inside = abs(px - 16) <= r and abs(py - 16) <= r and a >= 1 / 255
            for ch in range(3):
                exp_val = a * col[ch] if inside else 0.0
                assert img[ch, py, px] == pytest.approx(exp_val, abs=1e-12, rel=1e-6)
            assert T[py, px] == pytest.approx(1 - a if inside else 1.0, rel=1e-6)


def test_footprint_box_excludes_pixels_beyond_three_sigma():
    # 2D variance chosen so that 3 sqrt(var + sqrt(0.1)) = 11.9: the first pixel
    # beyond the box is then only ~3.3 sigma out, where alpha is still > 1/255
    var = (11.9 / 3) ** 2 - math.sqrt(0.1)
    s = math.sqrt(var - 0.3) * 3.0 / F
    g = _gaussians([3.0], [s], [8.0], [(1.0, 1.0, 1.0)])
    (img, T, nc, mg), dec, sc = _render(g)
    r = int(dec.radius[0])
    assert r == 12
    a_out = _sig(8.0) * math.exp(-((r + 1) ** 2) / (2 * var))
    assert a_out > 1 / 255          # alpha would clear the cutoff ...
    assert img[0, 16, 16 + r + 1] == 0.0  # ... but the pixel is outside the box
    assert img[0, 16, 16 + r] > 0.0


def test_opaque_front_gaussian_occludes_all_but_one_percent():
    zs, scales, logits = [2.0, 4.0], [0.3, 0.1], [12.0, 0.5]
    dcs = [(0.2, 0.3, 0.4), (1.5, -0.5, 0.7)]
    g = _gaussians(zs, scales, logits, dcs)
    (img, T, nc, mg), dec, sc = _render(g)
    cf = [Y00 * float(np.float32(c)) + 0.5 for c in dcs[0]]
    cb = [max(0.0, Y00 * float(np.float32(c)) + 0.5) for c in dcs[1]]
    ab = _sig(float(np.float32(0.5)))
    for ch in range(3):
        # front alpha clamps to 0.99 at the centre pixel (G = 1): back adds 0.01 * alpha_b * c_b
        assert img[ch, 16, 16] == pytest.approx(0.99 * cf[ch] + 0.01 * ab * cb[ch], rel=1e-12)
    assert T[16, 16] == pytest.approx(0.01 * (1 - ab), rel=1e-12)


def test_transmittance_is_product_and_blend_uses_earlier_alphas():
    rng = np.random.default_rng(7)
    for _ in range(5):
        k = int(rng.integers(2, 7))
        zs = np.sort(rng.uniform(1.5, 6.0, k))
        logits = rng.uniform(-3, 0.5, k)
        dcs = rng.uniform(-0.5, 1.5, (k, 3))
        g = _gaussians(zs, np.full(k, 0.2), logits, dcs)
        (img, T, nc, mg), dec, sc = _render(g)
        sig = [_sig(float(np.float32(l))) for l in logits]
        cols = [[max(0.0, Y00 * float(np.float32(c)) + 0.5) for c in row] for row in dcs]
        Tp = 1.0
        Cexp = np.zeros(3)
        for i in range(k):
            Cexp += np.array(cols[i]) * sig[i] * Tp
            Tp *= 1 - sig[i]
        assert T[16, 16] == pytest.approx(Tp, rel=1e-12)
        np.testing.assert_allclose(img[:, 16, 16], Cexp, rtol=1e-12)
        assert nc[16, 16] == k


def test_input_order_does_not_matter():
    rng = np.random.default_rng(9)
    k = 12
    mean_op = np.zeros((k, 4), np.float32)
    mean_op[:, 0:2] = rng.uniform(-0.3, 0.3, (k, 2))
    mean_op[:, 2] = rng.uniform(2, 5, k)
    mean_op[:, 3] = rng.normal(0, 1, k)
    quat = rng.standard_normal((k, 4)).astype(np.float32)
    ls = np.zeros((k, 4), np.float32)
    ls[:, :3] = rng.normal(-2.5, 0.3, (k, 3))
    sh = rng.normal(0, 0.3, (12, k, 4)).astype(np.float32)
    (img, T, _, _), _, _ = _render((mean_op, quat, ls, sh))
    perm = rng.permutation(k)
    (img2, T2, _, _), _, _ = _render((mean_op[perm].copy(), quat[perm].copy(), ls[perm].copy(),
                                      sh[:, perm].copy()))
    assert np.array_equal(img, img2) and np.array_equal(T, T2)


def test_termination_stops_before_transmittance_drops_below_threshold():
    k = 6
    g = _gaussians(np.linspace(2, 4, k), np.full(k, 0.3), np.full(k, math.log(0.95 / 0.05)),
                   np.full((k, 3), 1.0))
    (img, T, nc, mg), dec, sc = _render(g)
    s = _sig(float(np.float32(math.log(0.95 / 0.05))))
    assert nc[16, 16] == 3                  # (1-0.95)^3 >= 1e-4 > (1-0.95)^4
    assert T[16, 16] == pytest.approx((1 - s) ** 3, rel=1e-12)
    (img_nt, T_nt, nc_nt, _), _, _ = _render(g, flags=oracle.NO_TERM)
    assert nc_nt[16, 16] == k


def test_alpha_below_cutoff_is_skipped():
    g = _gaussians([3.0], [0.1], [-6.0], [(1.0, 1.0, 1.0)])  # sigmoid(-6) ~ 0.0025 < 1/255
    (img, T, nc, mg), _, _ = _render(g)
    assert np.all(img == 0) and np.all(T == 1)
    (img2, T2, _, _), _, _ = _render(g, flags=oracle.NO_SKIP)
    assert img2[0, 16, 16] > 0
