"""Pins of the oracle's complete operators (P2M, M2M, M2L, L2L, L2P; Sec. II.C,
II.D, App. B.3).  M2M and L2L are exact for truncated expansions, and M2L of a
monopole equals the local expansion of that charge, so rotations, Wigner
matrices, the diagonal transforms and their signs are pinned together."""
import numpy as np
import pytest


def _cloud(seed, n=12, half=0.3):
    rng = np.random.default_rng(seed)
    return rng.uniform(-half, half, (n, 3)), rng.uniform(-1, 1, n)


def test_p2m_monopole_and_dipole(orc):
    pts, q = _cloud(0)
    C = orc.p2m(4, pts, q, np.zeros(3))
    assert C[orc.idx(0, 0)] == pytest.approx(q.sum())
    assert C[orc.idx(1, 1)] == pytest.approx((q * pts[:, 0]).sum() / 2)
    assert C[orc.idx(1, -1)] == pytest.approx(-(q * pts[:, 1]).sum() / 2)
    assert C[orc.idx(1, 0)] == pytest.approx((q * pts[:, 2]).sum())


def test_single_charge_far_and_near(orc):
    """One charge: M2P far away and P2L->L2P near the centre reproduce q/|x - r0|."""
    r0 = np.array([0.1, -0.05, 0.08])
    q = np.array([1.7])
    x_far = np.array([2.5, 1.0, -1.5])
    exact = 1.7 / np.linalg.norm(x_far - r0)
    for p, tol in ((4, 1e-5), (8, 1e-8), (12, 1e-11)):
        C = orc.p2m(p, r0[None, :], q, np.zeros(3))
        assert orc.m2p(p, C, np.zeros(3), x_far) == pytest.approx(exact, rel=tol)
        D = orc.p2l(p, x_far[None, :], q, np.zeros(3))
        assert orc.l2p(p, D, np.zeros(3), r0) == pytest.approx(exact, rel=tol)


@pytest.mark.parametrize("shift", [(0.21, -0.33, 0.12), (0, 0, 0.4), (0, 0, -0.4), (0.3, 0, 0), (0, 0, 0)])
def test_m2m_is_exact(orc, shift):
    pts, q = _cloud(1)
    p = 10
    c_child = np.array([0.05, -0.02, 0.03])
    c_par = c_child + np.array(shift)
    got = orc.m2m(p, orc.p2m(p, pts, q, c_child), c_child, c_par)
    want = orc.p2m(p, pts, q, c_par)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


@pytest.mark.parametrize("shift", [(0.1, -0.2, 0.13), (0, 0, 0.25), (0, 0, -0.25), (0, 0, 0)])
def test_l2l_is_exact(orc, shift):
    pts, q = _cloud(2)
    p = 10
    c_old = np.array([4.0, -1.0, 2.0])
    c_new = c_old + np.array(shift)
    D = orc.p2l(p, pts, q, c_old)
    Dn = orc.l2l(p, D, c_old, c_new)
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = c_new + rng.uniform(-0.1, 0.1, 3)
        assert orc.l2p(p, Dn, c_new, x) == pytest.approx(orc.l2p(p, D, c_old, x), rel=1e-12)


def test_l2l_composes_exactly(orc):
    """Translations of a degree-p local expansion compose without truncation:
    L2L(A -> leaf) equals L2L(parent -> leaf) after L2L(A -> parent), and the
    chain over three levels equals the direct translation (the GPU applies the
    level-by-level L2L of Sec. II.C in this direct form)."""
    p = 10
    rng = np.random.default_rng(11)
    D = rng.normal(size=(p + 1) ** 2)
    cA = np.array([0.0, 0.0, 0.0])
    cP = cA + np.array([0.21, -0.13, 0.17])
    cG = cP + np.array([-0.08, 0.11, 0.06])
    cL = cG + np.array([0.03, -0.04, -0.05])
    chain = orc.l2l(p, orc.l2l(p, orc.l2l(p, D, cA, cP), cP, cG), cG, cL)
    direct = orc.l2l(p, D, cA, cL)
    np.testing.assert_allclose(chain, direct, rtol=1e-11, atol=1e-12 * np.abs(direct).max())
    # with M2L sums at every level: the leaf's local is its own sum plus the
    # direct translations of its ancestors' own sums
    own = {c: rng.normal(size=(p + 1) ** 2) for c in ("A", "P", "G", "L")}
    lev = orc.l2l(p, own["A"], cA, cP) + own["P"]
    lev = orc.l2l(p, lev, cP, cG) + own["G"]
    lev = orc.l2l(p, lev, cG, cL) + own["L"]
    direct = (own["L"] + orc.l2l(p, own["G"], cG, cL) + orc.l2l(p, own["P"], cP, cL)
              + orc.l2l(p, own["A"], cA, cL))
    np.testing.assert_allclose(lev, direct, rtol=1e-11, atol=1e-12 * np.abs(direct).max())


@pytest.mark.parametrize("c_trg", [(2.0, -1.5, 1.2), (0, 0, -3.0), (0, 0, 3.0), (-2.2, 0.1, 0.0)])
def test_m2l_monopole_is_exact(orc, c_trg):
    p = 10
    C = np.zeros((p + 1) ** 2)
    C[0] = 1.7
    cS = np.array([0.2, 0.1, -0.3])
    got = orc.m2l(p, C, cS, np.array(c_trg))
    want = 1.7 * orc.shat(p, cS - np.array(c_trg))
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13 * np.abs(want).max())


def test_m2l_converges_to_p2l(orc):
    """A shrinking source cluster: M2L(P2M) -> P2L with error ~ (size/d)^(p+1);
    the sign factor sgn(m)(-1)^(k+m) of App. B.3 matters at m != 0."""
    pts, q = _cloud(4)
    p = 6
    cS, cT = np.zeros(3), np.array([2.0, -1.5, 1.2])
    errs = []
    for scale in (1e-1, 1e-2):
        P = pts * scale
        D = orc.m2l(p, orc.p2m(p, P, q, cS), cS, cT)
        Dx = orc.p2l(p, P, q, cT)
        errs.append(np.abs(D - Dx).max() / np.abs(Dx).max())
    assert errs[1] < 1e-13
    assert errs[0] < 1e-8


def test_m2l_then_l2p_matches_direct(orc):
    pts, q = _cloud(5)
    cS, cT = np.zeros(3), np.array([1.6, 1.1, -2.0])
    rng = np.random.default_rng(6)
    xs = cT + rng.uniform(-0.3, 0.3, (6, 3))
    exact = np.array([np.sum(q / np.linalg.norm(x - pts, axis=1)) for x in xs])
    prev = None
    for p in (4, 8, 12):
        D = orc.m2l(p, orc.p2m(p, pts, q, cS), cS, cT)
        err = max(abs(orc.l2p(p, D, cT, x) - e) / abs(e) for x, e in zip(xs, exact))
        if prev is not None:
            assert err < prev / 10
        prev = err
    assert prev < 1e-7
