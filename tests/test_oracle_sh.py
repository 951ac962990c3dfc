"""Pins of the oracle's real spherical harmonics (colour model, Sec. 3).

The oracle has two derivations (associated-Legendre recurrence in spherical
angles, and Cartesian polynomials); they are checked against each other,
against orthonormality on the sphere, against textbook closed forms, and the
Cartesian gradient against finite differences.
"""
import numpy as np
import pytest


def _dirs(n, seed=0):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_two_derivations_agree(orc):
    for d in _dirs(200):
        a = orc.sh_spherical(3, d)
        b, _ = orc.sh_cartesian(3, d)
        np.testing.assert_allclose(a, b, atol=1e-13)


def test_orthonormal_on_sphere(orc):
    # Gauss-Legendre in cos(theta) x uniform in phi integrates polynomials of
    # degree <= 6 on the sphere exactly.
    x, w = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for z, wz in zip(x, w):
        s = np.sqrt(1 - z * z)
        for ph in phis:
            Y = orc.sh_spherical(3, [s * np.cos(ph), s * np.sin(ph), z])
            G += wz * (2 * np.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_textbook_closed_forms(orc):
    pi = np.pi
    for x, y, z in _dirs(20, 1):
        Y, _ = orc.sh_cartesian(3, [x, y, z])
        # Condon-Shortley phase: Y_1^{+1} = -sqrt(3/4pi) x, Y_1^{-1} = -sqrt(3/4pi) y
        expect = {
            0: 0.5 / np.sqrt(pi),
            1: -np.sqrt(3 / (4 * pi)) * y,
            2: np.sqrt(3 / (4 * pi)) * z,
            3: -np.sqrt(3 / (4 * pi)) * x,
            4: 0.5 * np.sqrt(15 / pi) * x * y,
            6: 0.25 * np.sqrt(5 / pi) * (3 * z * z - 1),
            8: 0.25 * np.sqrt(15 / pi) * (x * x - y * y),
            12: 0.25 * np.sqrt(7 / pi) * z * (5 * z * z - 3),
            10: 0.5 * np.sqrt(105 / pi) * x * y * z,
        }
        for k, v in expect.items():
            assert abs(Y[k] - v) < 1e-13, (k, Y[k], v)


def test_cartesian_gradient_matches_fd(orc):
    h = 1e-6
    for d in _dirs(30, 2):
        _, dY = orc.sh_cartesian(3, d)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            Yp, _ = orc.sh_cartesian(3, d + e)
            Ym, _ = orc.sh_cartesian(3, d - e)
            np.testing.assert_allclose((Yp - Ym) / (2 * h), dY[:, a], atol=1e-8)


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_lower_degrees_are_prefixes(orc, deg):
    d = _dirs(1, 3)[0]
    np.testing.assert_array_equal(orc.sh_spherical(deg, d), orc.sh_spherical(3, d)[: (deg + 1) ** 2])
