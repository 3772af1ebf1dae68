"""Pins of the oracle's hierarchy (Sec. II.A, Listing 2) and interaction lists
(Sec. II.B, Eq. 4): balance counts, brute-force median splits, leaf order,
bounding-box geometry, and the coverage invariant of the lists."""
import itertools

import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads


def _levels_ref(n, leaf, s):
    L = 0
    while -(-n // (1 << (s * L))) > leaf:
        L += 1
    return L


@pytest.mark.parametrize("n,leaf,s", [(1, 4, 2), (4, 4, 2), (5, 4, 2), (97, 8, 2), (1000, 16, 2),
                                      (4097, 64, 2), (777, 8, 1), (3001, 16, 3)])
def test_balance_counts(orc, n, leaf, s):
    """Level-l boxes hold ceil(N/2^(l s)) or floor(N/2^(l s)) points."""
    pos, _ = workloads.uniform_cube(n, seed=n)
    T = orc.Tree(pos, leaf, s, 0.5)
    assert T.L == _levels_ref(n, leaf, s) == orc.num_levels(n, leaf, s)
    assert sorted(T.perm.tolist()) == list(range(n))
    for l in range(T.L + 1):
        off, nb = T.level_offset(l), 1 << (s * l)
        cnt = T.box_count[off:off + nb]
        assert set(cnt.tolist()) <= {-(-n // nb), n // nb}
        assert cnt.sum() == n
        assert T.box_start[off] == 0
        np.testing.assert_array_equal(T.box_start[off + 1:off + nb], np.cumsum(cnt)[:-1])


def _check_splits(pos, T, s):
    """Every box's lower child holds the ceil(n/2) smallest points by
    (coordinate on the longest bbox axis, original index), recursively."""
    perm = T.perm
    n_rounds = T.L * s
    for l in range(T.L + 1):
        off, nb = T.level_offset(l), 1 << (s * l)
        for b in range(nb):
            a, c = T.box_start[off + b], T.box_count[off + b]
            members = set(perm[a:a + c].tolist())
            # descend the s bisections of this box by brute force
            segs = [sorted(members)]
            for _ in range(s if l < T.L else 0):
                nxt = []
                for seg in segs:
                    P = pos[seg]
                    ext = P.max(0) - P.min(0)
                    ax = int(np.argmax(ext))
                    order = sorted(seg, key=lambda i: (pos[i, ax], i))
                    h = (len(order) + 1) // 2
                    nxt += [order[:h], order[h:]]
                segs = nxt
            if l < T.L:
                coff = T.level_offset(l + 1)
                for k, seg in enumerate(segs):
                    g = coff + (b << s) + k
                    child = perm[T.box_start[g]:T.box_start[g] + T.box_count[g]]
                    assert set(child.tolist()) == set(seg)
    assert n_rounds == T.L * s


@pytest.mark.parametrize("n,leaf,s", [(300, 8, 2), (257, 5, 1), (600, 16, 3)])
def test_median_splits_brute_force(orc, n, leaf, s):
    pos, _ = workloads.uniform_cube(n, seed=3)
    T = orc.Tree(pos, leaf, s, 0.5)
    _check_splits(pos, T, s)


def test_ties_and_signed_zero(orc):
    """Grid points with many equal coordinates, and -0.0 next to +0.0: ties go
    by original index, -0.0 equals +0.0."""
    g = np.arange(6, dtype=float)
    pos = np.array(list(itertools.product(g, g, [0.0, 1.0])))
    pos[::7, 2] = -0.0
    T = orc.Tree(pos, 4, 2, 0.5)
    _check_splits(pos, T, 2)
    pos2 = pos.copy()
    pos2[pos2 == 0.0] = 0.0  # all +0.0
    T2 = orc.Tree(pos2, 4, 2, 0.5)
    np.testing.assert_array_equal(T.perm, T2.perm)
    np.testing.assert_array_equal(T.center.view(np.uint64), T2.center.view(np.uint64))
    assert not np.any(np.signbit(T.center) & (T.center == 0.0))


def test_leaf_order_and_geometry(orc):
    pos, _ = workloads.plummer_sphere(3000, seed=4)
    T = orc.Tree(pos, 16, 2, 0.5)
    off = T.level_offset(T.L)
    for b in range(T.n_leaves):
        a, c = T.box_start[off + b], T.box_count[off + b]
        leaf = T.perm[a:a + c]
        assert np.all(np.diff(leaf) > 0)
    for g in range(T.n_boxes):
        P = pos[T.perm[T.box_start[g]:T.box_start[g] + T.box_count[g]]]
        lo, hi = P.min(0), P.max(0)
        np.testing.assert_array_equal(T.center[g], (lo + hi) * 0.5)
        assert T.radius[g] == pytest.approx(0.5 * np.linalg.norm(hi - lo), rel=1e-15)
        assert np.linalg.norm(P - T.center[g], axis=1).max() <= T.radius[g] * (1 + 1e-15)


def test_single_leaf_tree(orc):
    pos, _ = workloads.uniform_cube(50, 0)
    T = orc.Tree(pos, 64, 2, 0.5)
    assert T.L == 0 and T.n_m2l == 0 and T.n_p2p == 1
    assert (T.p2p_trg[0], T.p2p_src[0]) == (0, 0)


def _ancestor(T, leaf, l):
    return T.level_offset(l) + (leaf >> (T.s * (T.L - l)))


def _level_of(T, g):
    l = 0
    while T.level_offset(l + 1) <= g:
        l += 1
    return l


def _ws(T, gs, gt, theta):
    d = np.linalg.norm(T.center[gs] - T.center[gt])
    R, r = max(T.radius[gs], T.radius[gt]), min(T.radius[gs], T.radius[gt])
    return d > 0 and R + theta * r <= theta * d


@pytest.mark.parametrize("kind", ["cube", "plummer", "clusters"])
@pytest.mark.parametrize("theta", [0.4, 0.7])
def test_lists_cover_every_leaf_pair_once(orc, kind, theta):
    n = 1500
    pos = {"cube": workloads.uniform_cube, "plummer": workloads.plummer_sphere,
           "clusters": workloads.gaussian_clusters}[kind](n, seed=9)[0]
    T = orc.Tree(pos, 12, 2, theta)
    m2l = set(zip(T.m2l_trg.tolist(), T.m2l_src.tolist()))
    p2p = set(zip(T.p2p_trg.tolist(), T.p2p_src.tolist()))
    assert len(m2l) == T.n_m2l and len(p2p) == T.n_p2p
    for (gt, gs) in m2l:
        assert _ws(T, gs, gt, theta)
    for (t, s_) in p2p:
        assert not _ws(T, T.level_offset(T.L) + s_, T.level_offset(T.L) + t, theta)
    for t in range(T.n_leaves):
        for s_ in range(T.n_leaves):
            hits = sum((_ancestor(T, t, lt), _ancestor(T, s_, ls)) in m2l
                       for lt in range(T.L + 1) for ls in range(T.L + 1))
            assert hits + ((t, s_) in p2p) == 1, (t, s_)


def test_list_order_and_level_march(orc):
    pos, _ = workloads.uniform_cube(4000, 2)
    T = orc.Tree(pos, 16, 2, 0.5)
    key = T.m2l_trg.astype(np.int64) * T.n_boxes + T.m2l_src
    assert np.all(np.diff(key) > 0)
    key = T.p2p_trg.astype(np.int64) * T.n_leaves + T.p2p_src
    assert np.all(np.diff(key) > 0)
    # same tree on both sides, equal radii advance the source: ls in {lt, lt+1}
    for gt, gs in zip(T.m2l_trg, T.m2l_src):
        assert _level_of(T, gs) - _level_of(T, gt) in (0, 1)


def test_tie_rule_flag_swaps_roles(orc):
    """With identical source and target trees the criterion is symmetric, so
    advancing the target on ties yields the transposed lists."""
    pos, _ = workloads.gaussian_clusters(2500, 7)
    A = orc.Tree(pos, 16, 2, 0.6, tie_target=False)
    B = orc.Tree(pos, 16, 2, 0.6, tie_target=True)
    assert set(zip(A.m2l_trg.tolist(), A.m2l_src.tolist())) == set(zip(B.m2l_src.tolist(), B.m2l_trg.tolist()))
    assert set(zip(A.p2p_trg.tolist(), A.p2p_src.tolist())) == set(zip(B.p2p_src.tolist(), B.p2p_trg.tolist()))
    for gt, gs in zip(B.m2l_trg, B.m2l_src):
        assert _level_of(B, gt) - _level_of(B, gs) in (0, 1)


def test_average_radius_per_level(orc):
    pos, _ = workloads.uniform_cube(3000, 1)
    T = orc.Tree(pos, 16, 2, 0.5)
    for l in range(T.L + 1):
        off, nb = T.level_offset(l), 1 << (2 * l)
        assert T.level_avg_radius[l] == pytest.approx(T.radius[off:off + nb].mean(), rel=1e-14)
    assert np.all(np.diff(T.level_avg_radius) < 0)


@pytest.mark.parametrize("s", [2, 3])
def test_same_level_lists_brute_force(orc, s):
    """Same-level lists (Sec. II.B steps 1-3) against their definition: a pair
    of boxes on one level is weakly coupled when it is well separated and no
    pair of their ancestors on a coarser level is; the leaf pairs with no
    well-separated ancestor pair at any level are strongly coupled."""
    pos, _ = workloads.double_helix(700, seed=4, turns=3.0, pitch=2.0)
    theta = 0.6
    T = orc.Tree(pos, 10, s, theta, same_level=True)
    nl = 1 << (s * T.L)
    m2l_ref, p2p_ref = set(), set()
    for t in range(nl):
        for s_ in range(nl):
            hit = None
            for l in range(T.L + 1):
                gt, gs = _ancestor(T, t, l), _ancestor(T, s_, l)
                if _ws(T, gs, gt, theta):
                    hit = (gt, gs)
                    break
            if hit is None:
                p2p_ref.add((t, s_))
            else:
                m2l_ref.add(hit)
    assert set(zip(T.m2l_trg.tolist(), T.m2l_src.tolist())) == m2l_ref
    assert set(zip(T.p2p_trg.tolist(), T.p2p_src.tolist())) == p2p_ref
    assert T.n_m2l == len(m2l_ref) and T.n_p2p == len(p2p_ref)
    key = T.m2l_trg.astype(np.int64) * T.n_boxes + T.m2l_src
    assert np.all(np.diff(key) > 0)


def test_same_vs_cross_level_on_helix(orc):
    """The comparison of Sec. II.B on a double helix with s = 3: the level
    march needs fewer weakly coupled pairs than same-level lists, by moving
    pairs to coarser target or source levels; the leaves covered are the
    same, and the root-level interactions agree."""
    pos, q = workloads.double_helix(6000, seed=0, turns=5.0, pitch=3.4, tube=0.1)
    A = orc.Tree(pos, 12, 3, 0.77, same_level=True)
    B = orc.Tree(pos, 12, 3, 0.77)
    assert B.n_m2l < A.n_m2l
    lv = lambda T, g: _level_of(T, g)
    la = {(lv(A, t), lv(A, s_)) for t, s_ in zip(A.m2l_trg, A.m2l_src)}
    assert all(a == b for a, b in la)
    lb = {(lv(B, t), lv(B, s_)) for t, s_ in zip(B.m2l_trg, B.m2l_src)}
    assert any(a != b for a, b in lb)
    first = min(l for l, _ in la)
    na = sum(1 for t in A.m2l_trg if lv(A, t) == first)
    nb = sum(1 for t, s_ in zip(B.m2l_trg, B.m2l_src) if lv(B, t) == first and lv(B, s_) == first)
    assert na == nb
    # both are complete, so the FMM results agree to the expansion error
    sub = workloads.sample_targets(len(q), 200)
    ua = A.eval(q, 6, targets=sub)
    ub = B.eval(q, 6, targets=sub)
    ud = orc.direct(pos, q, targets=sub)
    for u in (ua, ub):
        assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-3
