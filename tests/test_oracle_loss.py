"""Pins for the oracle's Eq. 4 loss: (1 - lambda) mean|I_r - I_gt| + lambda (1 - SSIM), lambda = 0.2 (Sec. 4.1).

SSIM is tied to an independent SciPy implementation (separable Gaussian
window, zero padding), to its constant-image closed form and to SSIM(I, I) = 1;
the gradient to central finite differences.
"""
import numpy as np
import pytest
from scipy.signal import correlate2d
from scipy.signal.windows import gaussian

import oracle
import synthetic as S


def _scipy_ssim_map(x, y):
    w = gaussian(11, 1.5)
    w = w / w.sum()
    k = np.outer(w, w)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    out = np.zeros_like(x)
    for c in range(x.shape[0]):
        f = lambda a: correlate2d(a, k, mode="same", boundary="fill", fillvalue=0)
        mx, my = f(x[c]), f(y[c])
        sxx = f(x[c] * x[c]) - mx * mx
        syy = f(y[c] * y[c]) - my * my
        sxy = f(x[c] * y[c]) - mx * my
        out[c] = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return out


def test_ssim_map_matches_scipy():
    x = S.random_image(3, 23, 31, seed=1).astype(np.float64)
    y = S.random_image(3, 23, 31, seed=2).astype(np.float64)
    np.testing.assert_allclose(oracle.ssim_map(x, y), _scipy_ssim_map(x, y), atol=1e-12)


def test_identical_images_have_zero_loss_and_gradient():
    x = S.random_image(3, 20, 24, seed=3)
    L, d = oracle.loss(x, x, 0.2)
    assert L == pytest.approx(0.0, abs=1e-14)
    assert np.abs(d).max() < 1e-14


def test_l1_only_and_constant_images():
    x = np.full((3, 30, 30), 0.25)
    y = np.full((3, 30, 30), 0.75)
    assert oracle.loss(x, y, 0.0, grad=False) == pytest.approx(0.5, abs=1e-15)
    s = oracle.ssim_map(x, y)
    C1 = 0.01 ** 2
    # away from the zero-padded border the variances vanish: S = (2ab + C1) / (a^2 + b^2 + C1)
    assert s[0, 15, 15] == pytest.approx((2 * 0.25 * 0.75 + C1) / (0.25 ** 2 + 0.75 ** 2 + C1), rel=1e-12)
    L = oracle.loss(x, y, 0.2, grad=False)
    assert L == pytest.approx(0.8 * 0.5 + 0.2 * (1 - s.mean()), rel=1e-14)


def test_gradient_matches_central_differences():
    x = S.random_image(3, 9, 12, seed=4).astype(np.float64)
    y = S.random_image(3, 9, 12, seed=5).astype(np.float64)
    assert np.abs(x - y).min() > 1e-4  # stay off the |.| kink
    _, d = oracle.loss(x, y, 0.2)
    h = 1e-6
    fd = np.zeros_like(x)
    for idx in np.ndindex(x.shape):
        xp = x.copy()
        xp[idx] += h
        xm = x.copy()
        xm[idx] -= h
        fd[idx] = (oracle.loss(xp, y, 0.2, grad=False) - oracle.loss(xm, y, 0.2, grad=False)) / (2 * h)
    np.testing.assert_allclose(d, fd, rtol=1e-6, atol=1e-11)


def test_luma_weights():
    """Gray stays gray (the weights sum to one); each pure channel gives its
    BT.601 weight."""
    g = np.full((3, 4, 5), 0.37)
    assert np.allclose(oracle.luma(g), 0.37, atol=1e-15)
    for c, w in enumerate((0.299, 0.587, 0.114)):
        e = np.zeros((3, 2, 2))
        e[c] = 1.0
        assert np.allclose(oracle.luma(e), w, atol=1e-15)
