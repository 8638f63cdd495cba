"""Pins for the oracle's real spherical-harmonic basis (colour of Eq. 3, Sec. 3.1 SH in R^16).

The oracle builds Y_lm from associated-Legendre polynomials; these tests tie it
to (a) SciPy's complex spherical harmonics, (b) textbook closed forms written
out by hand, (c) orthonormality on the sphere by Gauss-Legendre quadrature and
(d) finite differences of its own direction gradient.
"""
import numpy as np
import pytest
from scipy.special import sph_harm_y

import oracle


def _dirs(n, seed=11):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_matches_scipy_complex_sh():
    # real Y_{l,+m} = sqrt2 Re Y_l^m, Y_{l,-m} = sqrt2 Im Y_l^m (Condon-Shortley phase in both)
    for v in _dirs(40):
        Y, _ = oracle.sh_basis(v, 3)
        theta = np.arccos(np.clip(v[2], -1, 1))
        phi = np.arctan2(v[1], v[0])
        for l in range(4):
            for m in range(-l, l + 1):
                c = sph_harm_y(l, abs(m), theta, phi)
                ref = c.real if m == 0 else (np.sqrt(2) * (c.real if m > 0 else c.imag))
                assert Y[l * l + l + m] == pytest.approx(float(ref), abs=1e-13)


def test_textbook_closed_forms():
    pi = np.pi
    for x, y, z in _dirs(20, seed=3):
        Y, _ = oracle.sh_basis(np.array([x, y, z]), 3)
        ref = [
            0.5 / np.sqrt(pi),
            -np.sqrt(3 / (4 * pi)) * y, np.sqrt(3 / (4 * pi)) * z, -np.sqrt(3 / (4 * pi)) * x,
            0.5 * np.sqrt(15 / pi) * x * y, -0.5 * np.sqrt(15 / pi) * y * z,
            0.25 * np.sqrt(5 / pi) * (3 * z * z - 1),
            -0.5 * np.sqrt(15 / pi) * x * z, 0.25 * np.sqrt(15 / pi) * (x * x - y * y),
            -0.25 * np.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
            0.5 * np.sqrt(105 / pi) * x * y * z,
            -0.25 * np.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
            0.25 * np.sqrt(7 / pi) * z * (5 * z * z - 3),
            -0.25 * np.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
            0.25 * np.sqrt(105 / pi) * z * (x * x - y * y),
            -0.25 * np.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y),
        ]
        np.testing.assert_allclose(Y, ref, atol=1e-13)


def test_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        s = np.sqrt(1 - z * z)
        for ph in phis:
            Y, _ = oracle.sh_basis(np.array([s * np.cos(ph), s * np.sin(ph), z]), 3)
            G += w * (2 * np.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_degree_limits_and_degree0_constant():
    for v in _dirs(5):
        Y0, dY0 = oracle.sh_basis(v, 0)
        assert Y0[0] == pytest.approx(0.5 / np.sqrt(np.pi), abs=1e-15)
        assert np.all(Y0[1:] == 0) and np.all(dY0 == 0)
        Y1, _ = oracle.sh_basis(v, 1)
        assert np.all(Y1[4:] == 0)


def test_gradient_of_polynomial_extension_fd():
    h = 1e-6
    for v in _dirs(10, seed=5):
        _, dY = oracle.sh_basis(v, 3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            Yp, _ = oracle.sh_basis(v + e, 3)
            Ym, _ = oracle.sh_basis(v - e, 3)
            np.testing.assert_allclose(dY[:, a], (Yp - Ym) / (2 * h), atol=1e-8)


def test_band_energy_rotation_invariant():
    # sum_m Y_lm(u) Y_lm(v) depends only on u.v (addition theorem): (2l+1)/(4pi) P_l(u.v)
    from numpy.polynomial.legendre import legval
    d = _dirs(12, seed=8)
    for u, v in zip(d[:6], d[6:]):
        Yu, _ = oracle.sh_basis(u, 3)
        Yv, _ = oracle.sh_basis(v, 3)
        for l in range(4):
            sl = slice(l * l, (l + 1) * (l + 1))
            coef = np.zeros(l + 1)
            coef[l] = 1
            ref = (2 * l + 1) / (4 * np.pi) * legval(float(u @ v), coef)
            assert float(Yu[sl] @ Yv[sl]) == pytest.approx(ref, abs=1e-13)
