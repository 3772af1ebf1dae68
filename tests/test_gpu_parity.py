"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

Tree, geometry and interaction lists must be bit-identical; FP64 potentials,
fields and gradients must match the oracle FMM to 1e-12 relative L2 (1e-11
for fields and position gradients, which carry an extra cancellation); the
FP32-compensated path must match the FP64 oracle FMM to the FP32 budget
derived in the tests below.
"""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# FP32C budget against the FP64 oracle FMM (same tree, same p).  The unit
# roundoff u = 2^-24 = 6e-8 enters (i) the near field through FP32 offsets
# from the leaf centres (a pair at distance r in a leaf of radius R carries
# about 2u R / r) with compensated sums, and (ii) the far field through about
# ten rounded operations per coefficient and translation along an M2M - M2L -
# L2L chain whose depth grows with the level count L, in a basis scaled by
# the box radii so that no coefficient over- or underflows.  A random walk of
# those roundings, u sqrt(10 (2L + 1)), is 6e-7 to 1.2e-6 for L = 3..8 on
# well-spread point sets (uniform cube, Plummer sphere, film; measured 7e-8
# to 4e-7), so their bar is 1e-6.  Mixed-sign charges in tight clusters
# cancel: a potential far smaller than the sum of its terms' magnitudes
# carries the terms' rounding relative to that smaller value (measured up to
# 9.4e-7 on Gaussian clusters with s = 3 and 1.6e-6 on the helix), so
# clustered sets get 4e-6.  Fields and position gradients are one derivative
# of the same sums with one more cancellation (measured up to 2.8e-6 and
# 8.5e-6): 1e-5 and 3e-5.  The named workloads carry their own bars, each
# 3-5x its measured error: cube4k_p4 5e-7 (1.2e-7), cube1m_p8 1e-6 (1.8e-7),
# plummer4m_p10 1e-6 (2.6e-7).
TOL_FP64 = 1e-12
TOL_FP64_FIELD = 1e-11
TOL_FP32 = 1e-6
TOL_FP32_CLUSTERED = 4e-6
TOL_FP32_FIELD = 1e-5
TOL_FP32_GRAD = 3e-5
TOL_FP32_CFG = {"cube4k_p4": 5e-7, "cube1m_p8": 1e-6, "plummer4m_p10": 1e-6, "clusters_s3_p6": TOL_FP32_CLUSTERED}


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15269_gb300 import build, fmm
    build.build()
    fmm.lib()
    return fmm


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def build_both(F, orc, pos, p, leaf, s=2, theta=0.5, prec=1, flags=0):
    T = F.fmm_build_tree(cuda(pos), p, leaf, s, theta, prec, flags)
    O = orc.Tree(pos, leaf, s, theta, tie_target=bool(flags & F.FMM_TIE_TARGET),
                 same_level=bool(flags & F.FMM_SAME_LEVEL))
    return T, O


def assert_same_tree(F, T, O):
    ex = F.fmm_tree_export(T)
    st = F.fmm_tree_stats(T)
    assert (st["levels"], st["n_boxes"], st["n_m2l"], st["n_p2p"]) == (O.L, O.n_boxes, O.n_m2l, O.n_p2p)
    np.testing.assert_array_equal(ex["perm"], O.perm)
    np.testing.assert_array_equal(ex["box_start"], O.box_start)
    np.testing.assert_array_equal(ex["box_count"], O.box_count)
    np.testing.assert_array_equal(ex["center"].view(np.uint64), O.center.view(np.uint64))
    np.testing.assert_array_equal(ex["radius"].view(np.uint64), O.radius.view(np.uint64))
    np.testing.assert_array_equal(ex["level_avg_radius"].view(np.uint64), O.level_avg_radius.view(np.uint64))
    np.testing.assert_array_equal(ex["m2l_trg"], O.m2l_trg)
    np.testing.assert_array_equal(ex["m2l_src"], O.m2l_src)
    np.testing.assert_array_equal(ex["p2p_trg"], O.p2p_trg)
    np.testing.assert_array_equal(ex["p2p_src"], O.p2p_src)
    leaf_counts = O.box_count[O.level_offset(O.L):].astype(np.int64)
    pairs = int(np.sum(leaf_counts[O.p2p_trg] * leaf_counts[O.p2p_src]))
    assert st["n_p2p_pairs"] == pairs


def dup_grid(n, seed):
    rng = np.random.default_rng(seed)
    return np.round(rng.random((n, 3)) * 8) / 8  # many exact duplicates


def random_dups(n, seed):
    # exact copies of random FP64 points, which land in other leaves too
    rng = np.random.default_rng(seed)
    base = rng.random((n - n // 6, 3))
    return np.concatenate([base, base[rng.choice(len(base), n // 6)]])


TREE_CASES = [
    ("cube4k_cfg", lambda: workloads.uniform_cube(4096, 0)[0], 64, 2, 0.4, 0),
    ("plummer30k", lambda: workloads.plummer_sphere(30000, 1)[0], 64, 2, 0.5, 0),
    ("film40", lambda: workloads.thin_film(40, 2)[0], 32, 2, 0.5, 0),
    ("clusters_s3", lambda: workloads.gaussian_clusters(10000, 3)[0], 16, 3, 0.6, 0),
    ("cube_s1", lambda: workloads.uniform_cube(5000, 4)[0], 8, 1, 0.5, 0),
    ("clusters_tie_target", lambda: workloads.gaussian_clusters(8000, 5)[0], 32, 2, 0.6, 1),
    ("n1", lambda: np.array([[0.3, -0.2, 0.1]]), 64, 2, 0.5, 0),
    ("n2", lambda: np.array([[0.3, -0.2, 0.1], [0.1, 0.1, 0.1]]), 4, 2, 0.5, 0),
    ("n50_single_leaf", lambda: workloads.uniform_cube(50, 6)[0], 64, 2, 0.5, 0),
    ("n2049", lambda: workloads.uniform_cube(2049, 7)[0], 16, 2, 0.5, 0),
    ("n4097", lambda: workloads.uniform_cube(4097, 8)[0], 8, 2, 0.5, 0),
    ("duplicates", lambda: dup_grid(3000, 9), 16, 2, 0.5, 0),
    ("cube250k", lambda: workloads.uniform_cube(250000, 10)[0], 64, 2, 0.5, 0),
    ("helix_same_level_s3", lambda: workloads.double_helix(6000, 0, 5.0, 1.0, 3.4, 0.1)[0], 12, 3, 0.77, 2),
    ("helix_cross_s3", lambda: workloads.double_helix(6000, 0, 5.0, 1.0, 3.4, 0.1)[0], 12, 3, 0.77, 0),
    ("cube_same_level", lambda: workloads.uniform_cube(20000, 11)[0], 32, 2, 0.5, 2),
    ("clusters_same_level_tie", lambda: workloads.gaussian_clusters(7000, 12)[0], 16, 2, 0.6, 3),
]


@pytest.mark.parametrize("name,mk,leaf,s,theta,flags", TREE_CASES, ids=[c[0] for c in TREE_CASES])
def test_tree_and_lists_bit_exact(F, orc, name, mk, leaf, s, theta, flags):
    pos = mk()
    T, O = build_both(F, orc, pos, 4, leaf, s, theta, 1, flags)
    assert_same_tree(F, T, O)
    F.fmm_tree_status(T)


POT_CASES = [
    ("cube4k_p4", lambda: workloads.uniform_cube(4096, 0), 4, 64, 2, 0.4),
    ("plummer20k_p8", lambda: workloads.plummer_sphere(20000, 1), 8, 64, 2, 0.5),
    ("film30_p8", lambda: workloads.thin_film(30, 2), 8, 32, 2, 0.5),
    ("cube12k_p10", lambda: workloads.uniform_cube(12000, 3), 10, 32, 2, 0.5),
    ("clusters_s3_p6", lambda: workloads.gaussian_clusters(9000, 4), 6, 32, 3, 0.6),
    ("cube6k_s1_p3", lambda: workloads.uniform_cube(6000, 5), 3, 16, 1, 0.5),
    ("cube3k_p1", lambda: workloads.uniform_cube(3000, 6), 1, 32, 2, 0.5),
    ("ragged_p5_leaf200", lambda: workloads.uniform_cube(7777, 7), 5, 200, 2, 0.5),
    ("duplicates_p6", lambda: (dup_grid(5000, 8), np.random.default_rng(8).uniform(-1, 1, 5000)), 6, 16, 2, 0.5),
    ("random_duplicates_p6", lambda: (random_dups(6000, 9), np.random.default_rng(9).uniform(-1, 1, 6000)), 6, 16, 2,
     0.5),
]


@pytest.mark.parametrize("name,mk,p,leaf,s,theta", POT_CASES, ids=[c[0] for c in POT_CASES])
def test_potential_parity(F, orc, name, mk, p, leaf, s, theta):
    pos, q = mk()
    T, O = build_both(F, orc, pos, p, leaf, s, theta, F.FMM_FP64)
    u_o = O.eval(q, p)
    u64 = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    e64 = rel_l2(u64, u_o)
    F.fmm_tree_set_precision(T, F.FMM_FP32C)
    u32 = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    e32 = rel_l2(u32, u_o)
    F.fmm_tree_status(T)
    print("%s: fp64 vs oracle %.3e, fp32c vs oracle %.3e" % (name, e64, e32))
    assert e64 <= TOL_FP64
    assert e32 <= TOL_FP32_CFG.get(name, TOL_FP32)


def test_same_level_potential_parity(F, orc):
    pos, q = workloads.double_helix(30000, 1, 5.0, 1.0, 3.4, 0.1)
    T, O = build_both(F, orc, pos, 8, 24, 3, 0.6, F.FMM_FP64, F.FMM_SAME_LEVEL)
    u_o = O.eval(q, 8)
    assert rel_l2(F.fmm_eval_potential(T, cuda(q)).cpu().numpy(), u_o) <= TOL_FP64
    F.fmm_tree_set_precision(T, F.FMM_FP32C)
    assert rel_l2(F.fmm_eval_potential(T, cuda(q)).cpu().numpy(), u_o) <= TOL_FP32_CLUSTERED
    F.fmm_tree_status(T)


@pytest.mark.parametrize("name,mk,p,leaf,s,theta", POT_CASES, ids=[c[0] for c in POT_CASES])
def test_fp64df_potential_parity(F, orc, name, mk, p, leaf, s, theta):
    """FP64 accuracy with the double-float near field: same bar as FP64."""
    pos, q = mk()
    T, O = build_both(F, orc, pos, p, leaf, s, theta, F.FMM_FP64DF)
    u_o = O.eval(q, p)
    u = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    F.fmm_tree_status(T)
    e = rel_l2(u, u_o)
    print("%s: fp64df vs oracle %.3e" % (name, e))
    # double-float values carry about 48 bits (2^-48 ~ 3.6e-15 per operation);
    # sums over thousands of near-field terms and the M2L's few hundred
    # operations per coefficient stay within about 1e-13, an order of
    # magnitude inside the FP64 bar (measured up to 4.8e-14 on these cases)
    assert e <= 2e-13


@pytest.mark.parametrize("name,mk,p,leaf,s,theta", POT_CASES[:4], ids=[c[0] for c in POT_CASES[:4]])
def test_field_parity(F, orc, name, mk, p, leaf, s, theta):
    pos, q = mk()
    T, O = build_both(F, orc, pos, p, leaf, s, theta, F.FMM_FP64)
    u_o, f_o = O.eval(q, p, field=True)
    u64, f64 = (x.cpu().numpy() for x in F.fmm_eval_field(T, cuda(q)))
    F.fmm_tree_set_precision(T, F.FMM_FP32C)
    u32, f32 = (x.cpu().numpy() for x in F.fmm_eval_field(T, cuda(q)))
    print("%s field: fp64 %.3e fp32c %.3e" % (name, rel_l2(f64, f_o), rel_l2(f32, f_o)))
    assert rel_l2(u64, u_o) <= TOL_FP64
    assert rel_l2(f64, f_o) <= TOL_FP64_FIELD
    assert rel_l2(u32, u_o) <= TOL_FP32
    assert rel_l2(f32, f_o) <= TOL_FP32_FIELD


def test_backward_matches_oracle(F, orc):
    pos, q = workloads.thin_film(24, 1)
    g = np.random.default_rng(2).normal(size=len(q))
    p = 8
    T, O = build_both(F, orc, pos, p, 32, 2, 0.5, F.FMM_FP64)
    # oracle FMM vjp: dq = K g, dpos = g grad u + q grad v = -(g E_q + q E_g)
    _, fq = O.eval(q, p, field=True)
    v, fg = O.eval(g, p, field=True)
    dq_o = v
    dp_o = -(g[:, None] * fq + q[:, None] * fg)
    gq, gp = F.fmm_backward(T, cuda(q), cuda(g))
    assert rel_l2(gq.cpu().numpy(), dq_o) <= TOL_FP64
    assert rel_l2(gp.cpu().numpy(), dp_o) <= TOL_FP64_FIELD
    # and the exact direct-sum gradient within the FMM truncation
    dq_d, dp_d = orc.direct_vjp(pos, q, g)
    assert rel_l2(gq.cpu().numpy(), dq_d) < 1e-4
    assert rel_l2(gp.cpu().numpy(), dp_d) < 1e-3


@pytest.mark.parametrize("kind,leaf", [("film", 32), ("cube", 64), ("clusters", 100), ("cube", 200)])
def test_backward_fp32c_matches_oracle(F, orc, kind, leaf):
    """FP32C backward (fused near-field sweep for leaves up to 128 points, two
    field evaluations above) against the oracle FMM's vector-Jacobian product."""
    if kind == "film":
        pos, q = workloads.thin_film(24, 1)
    elif kind == "cube":
        pos, q = workloads.uniform_cube(9000, 3)
    else:
        pos, q = workloads.gaussian_clusters(9000, 4)
    g = np.random.default_rng(2).normal(size=len(q))
    p = 8
    T, O = build_both(F, orc, pos, p, leaf, 2, 0.5, F.FMM_FP32C)
    _, fq = O.eval(q, p, field=True)
    v, fg = O.eval(g, p, field=True)
    dp_o = -(g[:, None] * fq + q[:, None] * fg)
    gq, gp = F.fmm_backward(T, cuda(q), cuda(g))
    F.fmm_tree_status(T)
    e_q, e_p = rel_l2(gq.cpu().numpy(), v), rel_l2(gp.cpu().numpy(), dp_o)
    print("%s leaf %d: dq %.2e dpos %.2e" % (kind, leaf, e_q, e_p))
    assert e_q <= (TOL_FP32_CLUSTERED if kind == "clusters" else TOL_FP32)
    assert e_p <= TOL_FP32_GRAD


def test_autograd_function(F, orc):
    pos, q = workloads.uniform_cube(3000, 3)
    T = F.fmm_build_tree(cuda(pos), 8, 32, 2, 0.5, F.FMM_FP64)
    P = cuda(pos).requires_grad_(True)
    Q = cuda(q).requires_grad_(True)
    u = F.FMMPotential.apply(P, Q, T)
    loss = 0.5 * (Q * u).sum()
    loss.backward()
    O = orc.Tree(pos, 32, 2, 0.5)
    uo, fo = O.eval(q, 8, field=True)
    # L = 1/2 q.u: dL/dq = u/2 + K(q/2) = u;  dL/dr = -(q/2 E_q + q E_{q/2}) = -q E_q
    assert rel_l2(Q.grad.cpu().numpy(), uo) <= 1e-11
    assert rel_l2(P.grad.cpu().numpy(), -q[:, None] * fo) <= TOL_FP64_FIELD


def test_host_buffer_entry_point(F):
    pos, q = workloads.uniform_cube(5000, 4)
    T = F.fmm_build_tree(cuda(pos), 6, 64, 2, 0.5, F.FMM_FP32C)
    u_dev = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    qh = torch.from_numpy(q).pin_memory()
    u_host = F.fmm_eval_potential_host(T, qh).numpy()
    np.testing.assert_array_equal(u_host, u_dev)


def test_edge_cases(F, orc):
    # one point: no other charge, potential 0
    T = F.fmm_build_tree(cuda(np.array([[0.5, 0.5, 0.5]])), 4, 64, 2, 0.5, F.FMM_FP64)
    assert F.fmm_eval_potential(T, cuda(np.array([3.0]))).item() == 0.0
    # coincident points contribute nothing to each other
    pos = np.array([[0.1, 0.2, 0.3]] * 3 + [[0.9, 0.8, 0.7]])
    q = np.array([1.0, 2.0, 3.0, 4.0])
    for prec in (F.FMM_FP64, F.FMM_FP32C, F.FMM_FP64DF):
        T = F.fmm_build_tree(cuda(pos), 4, 4, 2, 0.5, prec)
        u = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
        np.testing.assert_allclose(u, orc.direct(pos, q), rtol=1e-6)
    # all points identical: zero radius everywhere
    pos = np.zeros((40, 3)) + 0.25
    for prec in (F.FMM_FP64, F.FMM_FP32C, F.FMM_FP64DF):
        T = F.fmm_build_tree(cuda(pos), 4, 4, 2, 0.5, prec)
        assert np.all(F.fmm_eval_potential(T, cuda(np.ones(40))).cpu().numpy() == 0.0)
    # non-finite positions are rejected
    bad = workloads.uniform_cube(100, 0)[0]
    bad[7, 1] = np.nan
    with pytest.raises(F.FmmError) as ei:
        F.fmm_build_tree(cuda(bad), 4, 16, 2, 0.5, F.FMM_FP64)
    assert ei.value.code == F.FMM_ERR_INVALID_ARG


def test_cube1m_p8_full_size(F, orc):
    """Uniform cube N = 2^20, p = 8, leaf 128, theta 0.4: bit-exact hierarchy,
    FP32C within 1e-6 relative L2 of the FP64 direct sum on sampled targets,
    FP64 within 1e-12 of the oracle FMM there."""
    c = workloads.CONFIGS["cube1m_p8"]
    pos, q = workloads.uniform_cube(c["n"], 0)
    T, O = build_both(F, orc, pos, c["p"], c["leaf_size"], c["s"], c["theta"], F.FMM_FP32C)
    assert_same_tree(F, T, O)
    tg = workloads.sample_targets(c["n"], 512, seed=1)
    ud = orc.direct(pos, q, targets=tg)
    u32 = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()[tg]
    F.fmm_tree_set_precision(T, F.FMM_FP64)
    u64 = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()[tg]
    uo = O.eval(q, c["p"], targets=tg)
    F.fmm_tree_status(T)
    print("cube1m: fp32c vs direct %.3e, fp64 vs direct %.3e, fp64 vs oracle fmm %.3e, fp32c vs oracle fmm %.3e"
          % (rel_l2(u32, ud), rel_l2(u64, ud), rel_l2(u64, uo), rel_l2(u32, uo)))
    assert rel_l2(u64, uo) <= TOL_FP64
    assert rel_l2(u32, uo) <= TOL_FP32_CFG["cube1m_p8"]
    assert rel_l2(u32, ud) <= 1e-6


def leaf_targets(O, n_leaves, seed):
    """Every point of `n_leaves` random leaves of the oracle tree (original
    indices, sorted): the oracle FMM then needs M2L and L2L only for those
    leaves and their ancestors."""
    rng = np.random.default_rng(seed)
    off = O.level_offset(O.L)
    leaves = rng.choice(O.n_leaves, n_leaves, replace=False)
    tg = np.concatenate([O.perm[O.box_start[off + l]:O.box_start[off + l] + O.box_count[off + l]] for l in leaves])
    return np.sort(tg.astype(np.int64))


def test_plummer4m_p10_full_size(F, orc):
    """Highly non-uniform N = 2^22 (70% Plummer + 30% sphere surface), p = 10,
    leaf 64, theta 0.5, depth 8, in the launch configuration the benchmark
    times: the hierarchy bit for bit against the oracle, and FP64, FP64DF and
    FP32C potentials against the oracle FMM at every point of 12 random leaves
    (the deepest tree the benchmark evaluates, where the FP32 radius scaling
    is stressed most), plus FP32C against the FP64 direct sum."""
    c = workloads.CONFIGS["plummer4m_p10"]
    pos, q = workloads.plummer_sphere(c["n"], seed=0)
    T, O = build_both(F, orc, pos, c["p"], c["leaf_size"], c["s"], c["theta"], F.FMM_FP32C)
    assert O.L == 8
    assert_same_tree(F, T, O)
    tg = leaf_targets(O, 12, seed=1)
    uo = O.eval(q, c["p"], targets=tg)
    ud = orc.direct(pos, q, targets=tg)
    qd = cuda(q)
    errs = {}
    for name, prec in (("fp32c", F.FMM_FP32C), ("fp64", F.FMM_FP64), ("fp64df", F.FMM_FP64DF)):
        F.fmm_tree_set_precision(T, prec)
        errs[name] = rel_l2(F.fmm_eval_potential(T, qd).cpu().numpy()[tg], uo)
    F.fmm_tree_set_precision(T, F.FMM_FP32C)
    e32d = rel_l2(F.fmm_eval_potential(T, qd).cpu().numpy()[tg], ud)
    F.fmm_tree_status(T)
    print("plummer4m vs oracle fmm (%d targets):" % len(tg), {k: "%.3e" % v for k, v in errs.items()},
          "fp32c vs direct %.3e, oracle fmm vs direct %.3e" % (e32d, rel_l2(uo, ud)))
    assert errs["fp64"] <= TOL_FP64
    assert errs["fp64df"] <= 2e-13
    assert errs["fp32c"] <= TOL_FP32_CFG["plummer4m_p10"]
    assert e32d <= 3e-6  # truncation (about 1.4e-6 at theta 0.5) plus the FP32 budget


def test_batched64_p6_full_size(F, orc):
    """64 charge sets of log-uniform size in [1e4, 5e5] (7.9 M points), p = 6,
    theta 0.6, merged into one batch and replayed from a CUDA graph as the
    benchmark does: every set's potential against its own direct sum on
    sampled targets, and the batch equal to the sets evaluated alone."""
    from paper_2511_15269_gb300 import autotune
    c = workloads.CONFIGS["batched64_p6"]
    sets = workloads.batched_sets(64, seed=0)
    B = autotune.build_batch([p for p, _ in sets], c["p"], 64, c["s"], c["theta"], F.FMM_FP32C)
    qd = cuda(np.concatenate([q for _, q in sets]))
    u = torch.empty_like(qd)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        F.fmm_eval_potential(B, qd, u)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        F.fmm_eval_potential(B, qd, u)
    u.zero_()
    graph.replay()
    torch.cuda.synchronize()
    uu = u.cpu().numpy()
    off = F.fmm_tree_point_offsets(B)
    rng = np.random.default_rng(3)
    num = den = 0.0
    for k, (pos, q) in enumerate(sets):
        tg = np.sort(rng.choice(len(q), 32, replace=False)).astype(np.int64)
        ud = orc.direct(pos, q, targets=tg)
        num += float(np.sum((uu[off[k] + tg] - ud) ** 2))
        den += float(np.sum(ud ** 2))
        if k % 16 == 0:  # a few sets alone, bit for bit
            T = F.fmm_build_tree(cuda(pos), c["p"], 64, c["s"], c["theta"], F.FMM_FP32C)
            np.testing.assert_array_equal(uu[off[k]:off[k + 1]], F.fmm_eval_potential(T, cuda(q)).cpu().numpy())
    F.fmm_tree_status(B)
    err = (num / den) ** 0.5
    print("batched64: rel L2 vs direct %.3e" % err)
    assert err < 1e-3


def test_empty_input_rejected(F):
    with pytest.raises(F.FmmError) as ei:
        F.fmm_build_tree(torch.zeros((0, 3), dtype=torch.float64, device="cuda"), 4, 16, 2, 0.5, F.FMM_FP32C)
    assert ei.value.code == F.FMM_ERR_INVALID_ARG
