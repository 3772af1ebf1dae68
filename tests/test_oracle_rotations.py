"""Pins of the oracle's Wigner matrices and of the App. B.1/B.2 rotations.

The Wigner elements are checked against Wigner's explicit sum (an independent
formula, evaluated here with exact rationals), d(0) = I, orthogonality and the
j = 1 closed forms; the rotations are checked against the expansions of
rotated point sets, which needs no reference implementation."""
import math
from fractions import Fraction

import numpy as np
import pytest


def wigner_explicit(j, m, k, beta):
    """Wigner's explicit sum for d^j_{m k}(beta) = <j m|exp(-i beta J_y)|j k>."""
    c, s = math.cos(beta / 2), math.sin(beta / 2)
    tot = 0.0
    for t in range(0, 2 * j + 1):
        a, b, cc, d = j + k - t, t, m - k + t, j - m - t
        if min(a, b, cc, d) < 0:
            continue
        coef = Fraction(math.factorial(j + m) * math.factorial(j - m) * math.factorial(j + k) * math.factorial(j - k))
        den = math.factorial(a) * math.factorial(b) * math.factorial(cc) * math.factorial(d)
        tot += (-1) ** (m - k + t) * math.sqrt(coef) / den * c ** (2 * j + k - m - 2 * t) * s ** (m - k + 2 * t)
    return tot


@pytest.mark.parametrize("beta", [0.0, 0.37, 1.2, math.pi / 2, 2.9, -0.8])
def test_wigner_matches_explicit_sum(orc, beta):
    p = 7
    d = orc.wigner_d(p, beta)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            for k in range(-n, n + 1):
                assert d[n, m + p, k + p] == pytest.approx(wigner_explicit(n, m, k, beta), abs=2e-14)


def test_wigner_identity_orthogonality_and_j1(orc):
    p = 10
    I = orc.wigner_d(p, 0.0)
    for n in range(p + 1):
        blk = I[n, p - n:p + n + 1, p - n:p + n + 1]
        np.testing.assert_allclose(blk, np.eye(2 * n + 1), atol=1e-15)
    b = 1.234
    d = orc.wigner_d(p, b)
    for n in range(p + 1):
        blk = d[n, p - n:p + n + 1, p - n:p + n + 1]
        np.testing.assert_allclose(blk @ blk.T, np.eye(2 * n + 1), atol=1e-13)
    # j = 1 closed forms
    c, s = math.cos(b), math.sin(b)
    assert d[1, p + 1, p + 1] == pytest.approx((1 + c) / 2)
    assert d[1, p + 1, p + 0] == pytest.approx(-s / math.sqrt(2))
    assert d[1, p + 1, p - 1] == pytest.approx((1 - c) / 2)
    assert d[1, p + 0, p + 0] == pytest.approx(c)
    assert d[1, p + 0, p + 1] == pytest.approx(s / math.sqrt(2))


def _rot_z(a):
    return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1.0]])


def _rot_y(a):
    return np.array([[math.cos(a), 0, math.sin(a)], [0, 1.0, 0], [-math.sin(a), 0, math.cos(a)]])


@pytest.fixture
def cloud():
    rng = np.random.default_rng(11)
    return rng.uniform(-0.5, 0.5, (9, 3)), rng.uniform(-1, 1, 9)


@pytest.mark.parametrize("angle", [0.7, -2.1, 3.0])
def test_azimuthal_rotation_equals_rotated_points(orc, cloud, angle):
    """App. B.1: coefficients after a turn of the frame by +angle about z equal
    those of the points turned by -angle."""
    pts, q = cloud
    p = 8
    Rz = _rot_z(-angle)
    C = orc.p2m(p, pts, q, np.zeros(3))
    np.testing.assert_allclose(orc.rotate_azimuthal(p, C, angle), orc.p2m(p, pts @ Rz.T, q, np.zeros(3)), atol=1e-15)
    far = pts + np.array([2.0, -1.0, 1.5])
    D = orc.p2l(p, far, q, np.zeros(3))
    np.testing.assert_allclose(orc.rotate_azimuthal(p, D, angle, local=True),
                               orc.p2l(p, far @ Rz.T, q, np.zeros(3)), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("angle", [0.9, -1.7, 2.6])
def test_polar_rotation_equals_rotated_points(orc, cloud, angle):
    """App. B.2 with d^{|m|}_{n,k} read as the Wigner element d^n_{|m|,k}."""
    pts, q = cloud
    p = 8
    Ry = _rot_y(-angle)
    C = orc.p2m(p, pts, q, np.zeros(3))
    np.testing.assert_allclose(orc.rotate_polar(p, C, angle), orc.p2m(p, pts @ Ry.T, q, np.zeros(3)), atol=1e-14)
    far = pts + np.array([2.0, -1.0, 1.5])
    D = orc.p2l(p, far, q, np.zeros(3))
    got = orc.rotate_polar(p, D, angle, local=True)
    want = orc.p2l(p, far @ Ry.T, q, np.zeros(3))
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13 * np.abs(want).max())


def test_rotation_round_trip(orc):
    p = 10
    rng = np.random.default_rng(5)
    C = rng.normal(size=(p + 1) ** 2)
    for local in (False, True):
        back = orc.rotate_polar(p, orc.rotate_polar(p, C, 1.1, local), -1.1, local)
        np.testing.assert_allclose(back, C, atol=1e-12)
        back = orc.rotate_azimuthal(p, orc.rotate_azimuthal(p, C, 0.4, local), -0.4, local)
        np.testing.assert_allclose(back, C, atol=1e-13)
