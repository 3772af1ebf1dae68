"""Pins of the oracle's basis functions (App. A) against closed forms, the
complex definitions via scipy's associated Legendre functions, finite
differences and the addition theorem."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import lpmv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "basis_low_order.txt")


def test_golden_low_order(orc):
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 20
    for r in rows:
        x, y, z = (float(v) for v in r[:3])
        kind, n, m = r[3], int(r[4]), int(r[5])
        want = float(Fraction(r[6]))
        if kind == "R":
            got = orc.rhat(2, (x, y, z))[orc.idx(n, m)]
        elif kind == "S":
            got = orc.shat(2, (x, y, z))[orc.idx(n, m)]
        else:
            c = int(kind[1])
            got = orc.grad_rhat(2, (x, y, z))[1][orc.idx(n, m), c]
        assert got == pytest.approx(want, rel=1e-15, abs=1e-16), r


def _complex_R(n, m, v):
    """App. A.1 definition: alpha r^n P^|m|_n(cos th) e^{i m phi}, alpha = (-1)^m/(n+|m|)!."""
    x, y, z = v
    r = math.sqrt(x * x + y * y + z * z)
    th, ph = math.acos(z / r), math.atan2(y, x)
    return (-1) ** m / math.factorial(n + abs(m)) * r**n * lpmv(abs(m), n, math.cos(th)) * np.exp(1j * m * ph)


def _complex_S(n, m, v):
    """App. A.2 definition: beta r^-(n+1) P^|m|_n e^{i m phi}, beta = (-1)^m (n-|m|)!."""
    x, y, z = v
    r = math.sqrt(x * x + y * y + z * z)
    th, ph = math.acos(z / r), math.atan2(y, x)
    return (-1) ** m * math.factorial(n - abs(m)) * r ** (-(n + 1)) * lpmv(abs(m), n, math.cos(th)) * np.exp(1j * m * ph)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_regular_basis_matches_complex_definition(orc, seed):
    p = 10
    v = np.random.default_rng(seed).normal(size=3)
    R = orc.rhat(p, v)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            c = _complex_R(n, m, v)
            want = c.real if m >= 0 else c.imag
            assert R[orc.idx(n, m)] == pytest.approx(want, rel=1e-11, abs=1e-14 * np.linalg.norm(v) ** n)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_singular_basis_matches_complex_definition(orc, seed):
    p = 10
    v = np.random.default_rng(seed).normal(size=3)
    S = orc.shat(p, v)
    r = np.linalg.norm(v)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            # App. A.2: Re(S^m_n) for m >= 0, Im(S^|m|_n) for m < 0
            want = _complex_S(n, m, v).real if m >= 0 else _complex_S(n, -m, v).imag
            scale = math.factorial(n) * r ** (-(n + 1))
            assert S[orc.idx(n, m)] == pytest.approx(want, rel=1e-10, abs=1e-13 * scale)


def test_regular_closed_forms(orc):
    v = (0.3, -0.7, 1.1)
    x, y, z = v
    R = orc.rhat(6, v)
    assert R[orc.idx(1, 0)] == pytest.approx(z)
    assert R[orc.idx(2, 0)] == pytest.approx((2 * z * z - x * x - y * y) / 4)
    for n in range(1, 7):
        w = (x + 1j * y) ** n / (2**n * math.factorial(n))
        assert R[orc.idx(n, n)] == pytest.approx(w.real, rel=1e-13)
        assert R[orc.idx(n, -n)] == pytest.approx(-w.imag, rel=1e-13)


def test_gradient_matches_finite_differences(orc):
    """App. A.3 with the diagonal sign obtained from App. A.1 (the printed
    leading minus would fail this test at n >= 2)."""
    p, h = 10, 1e-6
    v = np.array([0.31, -0.52, 0.44])
    _, G = orc.grad_rhat(p, v)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd = (orc.rhat(p, v + e) - orc.rhat(p, v - e)) / (2 * h)
        np.testing.assert_allclose(G[:, c], fd, rtol=1e-7, atol=1e-10)
    # the R^2_2 = (x^2 - y^2)/8 case written out
    x, y, _ = v
    assert G[orc.idx(2, 2)] == pytest.approx([x / 4, -y / 4, 0.0])


def test_addition_theorem_converges(orc):
    """sum (2 - delta_0m) sgn(m) R(r') S(r) -> 1/|r - r'| (Eq. 6 in the real basis)."""
    rp = np.array([0.2, -0.1, 0.15])
    r = np.array([0.9, 0.6, -0.8])
    exact = 1.0 / np.linalg.norm(r - rp)
    errs = []
    for p in (2, 4, 6, 8, 10, 12):
        R, S = orc.rhat(p, rp), orc.shat(p, r)
        s = 0.0
        for n in range(p + 1):
            for m in range(-n, n + 1):
                w = 1.0 if m == 0 else (2.0 if m > 0 else -2.0)
                s += w * R[orc.idx(n, m)] * S[orc.idx(n, m)]
        errs.append(abs(s - exact) / exact)
    ratio = np.linalg.norm(rp) / np.linalg.norm(r)
    assert errs[-1] < 1e-8
    for a, b in zip(errs, errs[1:]):
        assert b < a * ratio * 1.5
