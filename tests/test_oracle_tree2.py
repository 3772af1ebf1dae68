"""Pins of the oracle's separate source and target hierarchies (Sec. II.B,
final part): coverage of every (target leaf, source leaf) pair by brute force,
Eq. 4 on every list entry, the transposition symmetry of the tie rule, the
reduction to the single-tree lists when sources and targets coincide, and
the potential and field at targets against the direct sum."""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads


def _ws(ca, ra, cb, rb, theta):
    d = np.linalg.norm(ca - cb)
    R, r = max(ra, rb), min(ra, rb)
    return d > 0 and R + theta * r <= theta * d


def _targets(n, seed, lo=-0.2, hi=1.2):
    return lo + (hi - lo) * np.random.default_rng(seed).random((n, 3))


def _anc(H, leaf, l):
    return H.level_offset(l) + (leaf >> (H.s * (H.L - l)))


@pytest.mark.parametrize("n_src,n_trg,s", [(700, 150, 2), (120, 900, 2), (600, 600, 3), (400, 50, 1)])
def test_tree2_lists_cover_every_pair_once(orc, n_src, n_trg, s):
    sp, _ = workloads.gaussian_clusters(n_src, seed=3, n_clusters=3, sigma=0.1)
    tp = _targets(n_trg, 4)
    theta = 0.6
    T = orc.Tree2(sp, tp, 10, s, theta)
    S, G = T.src, T.trg
    nbs = S.n_boxes
    m2l = set(zip(T.m2l_trg.tolist(), T.m2l_src.tolist()))
    p2p = set(zip(T.p2p_trg.tolist(), T.p2p_src.tolist()))
    assert len(m2l) == T.n_m2l and len(p2p) == T.n_p2p
    for gt, gs in m2l:
        assert nbs <= gt < nbs + G.n_boxes and 0 <= gs < nbs
        assert _ws(S.center[gs], S.radius[gs], G.center[gt - nbs], G.radius[gt - nbs], theta)
    lt_off, ls_off = G.level_offset(G.L), S.level_offset(S.L)
    for t, s_ in p2p:
        assert not _ws(S.center[ls_off + s_], S.radius[ls_off + s_], G.center[lt_off + t], G.radius[lt_off + t], theta)
    for t in range(G.n_leaves):
        for s_ in range(S.n_leaves):
            hits = sum((nbs + _anc(G, t, lt), _anc(S, s_, ls)) in m2l
                       for lt in range(G.L + 1) for ls in range(S.L + 1))
            assert hits + ((t, s_) in p2p) == 1, (t, s_)
    key = T.m2l_trg.astype(np.int64) * (nbs + G.n_boxes) + T.m2l_src
    assert np.all(np.diff(key) > 0)


def test_tree2_tie_rule_transposes_with_roles(orc):
    """The criterion is symmetric, so swapping the roles of the two point sets
    and the tie rule together transposes the lists."""
    a, _ = workloads.uniform_cube(2048, 1)      # same count: equal radii ties occur
    b, _ = workloads.uniform_cube(2048, 2)
    A = orc.Tree2(a, b, 16, 2, 0.5, tie_target=False)
    B = orc.Tree2(b, a, 16, 2, 0.5, tie_target=True)
    na, nb = A.src.n_boxes, B.src.n_boxes
    ea = {(int(t) - na, int(s)) for t, s in zip(A.m2l_trg, A.m2l_src)}
    eb = {(int(s), int(t) - nb) for t, s in zip(B.m2l_trg, B.m2l_src)}
    assert ea == eb
    assert set(zip(A.p2p_trg.tolist(), A.p2p_src.tolist())) == set(zip(B.p2p_src.tolist(), B.p2p_trg.tolist()))


def test_tree2_with_equal_sets_is_the_single_tree(orc):
    pos, q = workloads.plummer_sphere(5000, 5)
    T = orc.Tree(pos, 32, 2, 0.5)
    T2 = orc.Tree2(pos, pos, 32, 2, 0.5)
    np.testing.assert_array_equal(T2.m2l_trg, T.m2l_trg + T.n_boxes)
    np.testing.assert_array_equal(T2.m2l_src, T.m2l_src)
    np.testing.assert_array_equal(T2.p2p_trg, T.p2p_trg)
    np.testing.assert_array_equal(T2.p2p_src, T.p2p_src)
    u1, f1 = T.eval(q, 6, field=True)
    u2, f2 = T2.eval(q, 6, field=True)
    np.testing.assert_allclose(u2, u1, rtol=0, atol=1e-15 * np.abs(u1).max())
    np.testing.assert_allclose(f2, f1, rtol=0, atol=1e-15 * np.abs(f1).max())


@pytest.mark.parametrize("kind", ["cube_halo", "shell_in_cube", "far"])
def test_tree2_potential_and_field_at_targets(orc, kind):
    sp, q = workloads.uniform_cube(6000, 7)
    if kind == "cube_halo":
        tp = _targets(2500, 8)
    elif kind == "shell_in_cube":
        v = np.random.default_rng(9).normal(size=(1800, 3))
        tp = 0.5 + 0.3 * v / np.linalg.norm(v, axis=1, keepdims=True)
    else:
        tp = _targets(700, 10) + np.array([6.0, 0.0, 0.0])
    T = orc.Tree2(sp, tp, 24, 2, 0.5)
    ud, fd = orc.direct2(sp, q, tp, field=True)
    errs = []
    for p in (3, 6, 9):
        u, f = T.eval(q, p, field=True)
        errs.append(np.linalg.norm(u - ud) / np.linalg.norm(ud))
        ef = np.linalg.norm(f - fd) / np.linalg.norm(fd)
        assert ef < 50 * 0.5 ** (p + 1) / 0.25
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5
    if kind == "far":
        # every target box is far from the source root: one root-level pair, no near field
        assert T.n_p2p == 0


def test_tree2_target_on_a_source(orc):
    """A target that coincides with a source point sees every other charge but
    not the coincident one (zero distances contribute nothing)."""
    sp, q = workloads.uniform_cube(3000, 11)
    tp = np.concatenate([sp[[5, 17, 2999]], _targets(300, 12)])
    T = orc.Tree2(sp, tp, 16, 2, 0.5)
    u = T.eval(q, 10)
    ud = orc.direct2(sp, q, tp)
    assert np.all(np.isfinite(u))
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-5
    # the coincident charge would dominate with a finite-distance treatment
    np.testing.assert_allclose(u[:3], ud[:3], rtol=1e-5)


def test_tree2_level_pairs_follow_the_march(orc):
    """Every M2L pair sits on the level path of Sec. II.B's rules: the side
    whose level has the larger average radius advances (ties: the source), the
    other side once one has no finer level."""
    sp, _ = workloads.plummer_sphere(4000, 13)
    tp = _targets(900, 14, -1.0, 1.0)
    T = orc.Tree2(sp, tp, 12, 2, 0.5)
    S, G = T.src, T.trg
    path, ls, lt = {(0, 0)}, 0, 0
    while ls < S.L or lt < G.L:
        if ls < S.L and lt < G.L:
            adv_src = S.level_avg_radius[ls] >= G.level_avg_radius[lt]
        else:
            adv_src = ls < S.L
        ls, lt = (ls + 1, lt) if adv_src else (ls, lt + 1)
        path.add((ls, lt))
    lev = lambda H, g: max(l for l in range(H.L + 1) if H.level_offset(l) <= g)
    seen = {(lev(S, int(s_)), lev(G, int(t) - S.n_boxes)) for t, s_ in zip(T.m2l_trg, T.m2l_src)}
    assert seen <= path
    assert len(seen) >= 3
