"""Pins for the oracle's Gaussian pyramid (Eq. 5), Adam step and PSNR."""
import math

import numpy as np
import pytest
from scipy.ndimage import convolve

import oracle
import synthetic as S


def test_pyramid_constant_image_stays_constant():
    x = np.full((3, 17, 22), 0.37)
    y = oracle.pyramid_down(x)
    assert y.shape == (3, 9, 11)
    np.testing.assert_allclose(y, 0.37, rtol=0, atol=1e-15)


def test_pyramid_matches_scipy_mirror_convolution():
    x = S.random_image(3, 21, 30, seed=8).astype(np.float64)
    k1 = np.array([1, 4, 6, 4, 1]) / 16.0
    k = np.outer(k1, k1)
    ref = np.stack([convolve(x[c], k, mode="mirror")[::2, ::2] for c in range(3)])
    np.testing.assert_allclose(oracle.pyramid_down(x), ref, atol=1e-15)


def test_pyramid_impulse_response_is_binomial():
    x = np.zeros((1, 20, 20))
    x[0, 10, 10] = 1.0
    y = oracle.pyramid_down(x)
    k1 = np.array([1, 4, 6, 4, 1]) / 16.0
    # output (i, j) samples input (2i, 2j): the impulse at (10, 10) reaches i, j in {4, 5, 6}
    for i in range(10):
        for j in range(10):
            di, dj = 10 - 2 * i + 2, 10 - 2 * j + 2
            ref = k1[di] * k1[dj] if 0 <= di < 5 and 0 <= dj < 5 else 0.0
            assert y[0, i, j] == pytest.approx(ref, abs=1e-16)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(0)
    g = rng.standard_normal(50)
    p = rng.standard_normal(50)
    lr = np.full(50, 1e-3)
    p1, m1, v1 = oracle.adam(p, g, np.zeros(50), np.zeros(50), lr, 1)
    # step 1: m_hat = g, v_hat = g^2 -> p - lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-15), rtol=1e-14)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-14)


def test_adam_second_step_by_hand():
    g1, g2 = 0.5, -2.0
    p1, m1, v1 = oracle.adam([1.0], [g1], [0.0], [0.0], [0.1], 1)
    p2, m2, v2 = oracle.adam(p1, [g2], m1, v1, [0.1], 2)
    m = 0.9 * 0.1 * g1 + 0.1 * g2
    v = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    mh, vh = m / (1 - 0.81), v / (1 - 0.999 ** 2)
    assert p2[0] == pytest.approx(p1[0] - 0.1 * mh / (math.sqrt(vh) + 1e-15), rel=1e-14)


def test_psnr_known_mse():
    gt = np.zeros(100)
    img = np.full(100, 0.1)
    assert oracle.psnr(img, gt) == pytest.approx(20.0, rel=1e-14)
    img2 = np.full(100, 1.7)  # clamped to 1 -> MSE 1 -> 0 dB
    assert oracle.psnr(img2, gt) == pytest.approx(0.0, abs=1e-14)
