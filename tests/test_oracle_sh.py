"""Pins of the oracle's real spherical harmonics (colour model, Sec. 3).

The oracle has two derivations (associated-Legendre recurrence in spherical
angles, and Cartesian polynomials); they are checked against each other,
against orthonormality on the sphere, against textbook closed forms, and the
Cartesian gradient against finite differences; the preprocess colour against
the closed form at a known view direction.
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


def test_colour_follows_the_view_direction(orc):
    """The colour of Sec. 3's primitives is the SH expansion at the unit
    direction from the camera centre c = -R^T t to the mean, plus 0.5,
    clamped at 0. A camera turned about y and moved off the origin sees a
    degree-1 splat on its optical axis, where that direction is R's third
    row; the expected colour is written with the textbook degree-0/1
    functions. The opposite direction, or a centre taken as t, fails."""
    from paper_2503_01199_gb300 import scenegen
    ph = 0.7
    R = np.array([[np.cos(ph), 0.0, -np.sin(ph)], [0.0, 1.0, 0.0], [np.sin(ph), 0.0, np.cos(ph)]])
    centre = np.array([0.4, -0.3, -2.0])
    t = -R @ centre
    cam = scenegen.pinhole_camera(64, 64, 64.0, R=R, t=t)
    R32 = np.asarray(cam["R"], np.float64)
    c32 = -R32.T @ np.asarray(cam["t"], np.float64)   # the camera as stored (float32)
    mean = c32 + R32.T @ np.array([0.0, 0.0, 3.0])
    sh = np.array([[[0.3, 0.1, -0.2], [0.5, -0.4, 0.2], [0.6, 0.3, -0.9], [-0.8, 0.2, 0.4]]])
    scene = {"mean": mean[None], "log_scale": np.full((1, 3), np.log(0.05)),
             "quat": np.array([[1.0, 0, 0, 0]]), "logit": np.zeros(1), "sh": sh, "sh_degree": 1}
    sp = orc.preprocess(scene, cam)
    assert sp["radius"][0] > 0
    np.testing.assert_allclose(sp["uv"][0], [32.0, 32.0], atol=1e-9)

    def colour(d):
        x, y, z = d / np.linalg.norm(d)
        s = np.sqrt(3 / (4 * np.pi))
        Y = np.array([0.5 / np.sqrt(np.pi), -s * y, s * z, -s * x])
        return np.maximum(0.0, 0.5 + Y @ sh[0])

    d = R32[2]
    want = colour(d)
    assert want.min() == 0.0 < want.max()            # one channel clamped
    np.testing.assert_allclose(sp["rgb"][0], want, rtol=1e-12, atol=1e-14)
    assert np.abs(colour(-d) - want).max() > 0.05
    assert np.abs(colour(mean - np.asarray(cam["t"], np.float64)) - want).max() > 0.05
