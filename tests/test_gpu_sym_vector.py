"""Symmetric near field of the field and of the backward pass (FP32C).

Pairs listed both ways are evaluated once: every 1/r and d / r^3 serves both
points (the field of the charges; the backward pass's potential of dL/du and
its pair-symmetric position gradient).  Checked against the oracle FMM at
the FP32C field and gradient bars, against the one-sided kernels
(FMM_OPT_NEAR_SYMMETRIC = 0) at the same bars, on leaves of 32, 64 and 128
points (the three register layouts), with coincident points (masked pairs),
and with the workspace rules (the slot buffers are made by the first such
evaluation; beside a caller's workspace nothing is allocated and the
one-sided kernel runs).
"""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# FP32C bars of the single-tree parity tests: fields 1e-5, position
# gradients 3e-5, potentials 1e-6 (4e-6 on clustered sets)
TOL_FP32 = 1e-6
TOL_FP32_CLUSTERED = 4e-6
TOL_FP32_FIELD = 1e-5
TOL_FP32_GRAD = 3e-5


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


def dup_points(n, seed):
    # exact copies of random points (coincident pairs inside and across leaves)
    rng = np.random.default_rng(seed)
    base = rng.random((n - n // 5, 3))
    pos = np.concatenate([base, base[rng.choice(len(base), n // 5)]])
    q = rng.uniform(-1.0, 1.0, len(pos))
    return pos, q


CASES = [
    ("cube_leaf32", lambda: workloads.uniform_cube(12000, 31), 32, 6),
    ("cube_leaf64", lambda: workloads.uniform_cube(20000, 32), 64, 6),
    ("cube_leaf128", lambda: workloads.uniform_cube(40000, 33), 128, 8),
    ("clusters_leaf64", lambda: workloads.gaussian_clusters(15000, 34), 64, 6),
    ("duplicates_leaf32", lambda: dup_points(6000, 35), 32, 5),
]


@pytest.mark.parametrize("name,mk,leaf,p", CASES, ids=[c[0] for c in CASES])
def test_symmetric_field_matches_oracle_and_one_sided(F, orc, name, mk, leaf, p):
    pos, q = mk()
    T = F.fmm_build_tree(cuda(pos), p, leaf, 2, 0.5, F.FMM_FP32C)
    O = orc.Tree(pos, leaf, 2, 0.5)
    u_o, f_o = O.eval(q, p, field=True)
    u_s, f_s = (x.cpu().numpy() for x in F.fmm_eval_field(T, cuda(q)))
    F.fmm_tree_status(T)
    F.fmm_tree_set_option(T, F.FMM_OPT_NEAR_SYMMETRIC, 0)
    u_1, f_1 = (x.cpu().numpy() for x in F.fmm_eval_field(T, cuda(q)))
    ub = TOL_FP32_CLUSTERED if name.startswith("clusters") else TOL_FP32
    print("%s: field sym %.2e one-sided %.2e, u sym %.2e" % (name, rel_l2(f_s, f_o), rel_l2(f_1, f_o),
                                                             rel_l2(u_s, u_o)))
    assert rel_l2(u_s, u_o) <= ub
    assert rel_l2(f_s, f_o) <= TOL_FP32_FIELD
    assert rel_l2(f_s, f_1) <= TOL_FP32_FIELD
    assert rel_l2(u_s, u_1) <= ub
    # the potential of the field evaluation agrees with the potential
    # evaluation (both symmetric; different kernels, same sums up to rounding)
    F.fmm_tree_set_option(T, F.FMM_OPT_NEAR_SYMMETRIC, 1)
    u_p = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    assert rel_l2(u_s, u_p) <= ub


@pytest.mark.parametrize("name,mk,leaf,p", CASES, ids=[c[0] for c in CASES])
def test_symmetric_backward_matches_oracle_and_one_sided(F, orc, name, mk, leaf, p):
    pos, q = mk()
    g = np.random.default_rng(7).normal(size=len(q))
    T = F.fmm_build_tree(cuda(pos), p, leaf, 2, 0.5, F.FMM_FP32C)
    O = orc.Tree(pos, leaf, 2, 0.5)
    _, fq = O.eval(q, p, field=True)
    v, fg = O.eval(g, p, field=True)
    dp_o = -(g[:, None] * fq + q[:, None] * fg)
    gq_s, gp_s = (x.cpu().numpy() for x in F.fmm_backward(T, cuda(q), cuda(g)))
    F.fmm_tree_status(T)
    F.fmm_tree_set_option(T, F.FMM_OPT_NEAR_SYMMETRIC, 0)
    gq_1, gp_1 = (x.cpu().numpy() for x in F.fmm_backward(T, cuda(q), cuda(g)))
    ub = TOL_FP32_CLUSTERED if name.startswith("clusters") else TOL_FP32
    print("%s: dq %.2e dpos %.2e (one-sided %.2e)" % (name, rel_l2(gq_s, v), rel_l2(gp_s, dp_o),
                                                      rel_l2(gp_1, dp_o)))
    assert rel_l2(gq_s, v) <= ub
    assert rel_l2(gp_s, dp_o) <= TOL_FP32_GRAD
    assert rel_l2(gq_s, gq_1) <= ub
    assert rel_l2(gp_s, gp_1) <= TOL_FP32_GRAD


def test_backward_position_gradient_only(F, orc):
    # dL/dq not requested: the combine writes dL/dx alone
    pos, q = workloads.uniform_cube(8000, 36)
    g = np.random.default_rng(8).normal(size=len(q))
    T = F.fmm_build_tree(cuda(pos), 6, 64, 2, 0.5, F.FMM_FP32C)
    gq, gp = F.fmm_backward(T, cuda(q), cuda(g), need_q=False)
    F.fmm_tree_status(T)
    assert gq is None
    O = orc.Tree(pos, 64, 2, 0.5)
    _, fq = O.eval(q, 6, field=True)
    _, fg = O.eval(g, 6, field=True)
    dp_o = -(g[:, None] * fq + q[:, None] * fg)
    assert rel_l2(gp.cpu().numpy(), dp_o) <= TOL_FP32_GRAD


def test_field_slot_buffers_and_caller_workspace(F, orc):
    pos, q = workloads.uniform_cube(20000, 37)
    O = orc.Tree(pos, 64, 2, 0.5)
    u_o, f_o = O.eval(q, 6, field=True)
    # (a) the first field evaluation makes the slot buffers: the workspace grows
    T = F.fmm_build_tree(cuda(pos), 6, 64, 2, 0.5, F.FMM_FP32C)
    w0 = F.fmm_tree_workspace_bytes(T)
    F.fmm_eval_field(T, cuda(q))
    w1 = F.fmm_tree_workspace_bytes(T)
    assert w1 > w0
    # ... and a caller's workspace of that size keeps the symmetric field
    ws = torch.empty(w1, dtype=torch.uint8, device="cuda")
    F.fmm_tree_set_workspace(T, ws)
    u, f = (x.cpu().numpy() for x in F.fmm_eval_field(T, cuda(q)))
    assert rel_l2(f, f_o) <= TOL_FP32_FIELD and rel_l2(u, u_o) <= TOL_FP32
    assert F.fmm_tree_workspace_bytes(T) == w1
    # (b) a caller's workspace attached before any field evaluation: nothing
    # is allocated, the one-sided kernel runs
    T2 = F.fmm_build_tree(cuda(pos), 6, 64, 2, 0.5, F.FMM_FP32C)
    ws2 = torch.empty(F.fmm_tree_workspace_bytes(T2), dtype=torch.uint8, device="cuda")
    F.fmm_tree_set_workspace(T2, ws2)
    before = F.fmm_device_memory_in_use()
    u2, f2 = (x.cpu().numpy() for x in F.fmm_eval_field(T2, cuda(q)))
    gq2, gp2 = (x.cpu().numpy() for x in F.fmm_backward(T2, cuda(q), cuda(q)))
    assert F.fmm_device_memory_in_use() == before
    assert F.fmm_tree_workspace_bytes(T2) == w0
    assert rel_l2(f2, f_o) <= TOL_FP32_FIELD and rel_l2(u2, u_o) <= TOL_FP32
    # cotangent g = q: dL/dq = K q = u, dL/dx = -(q E_q + q E_q) = -2 q E
    assert rel_l2(gq2, u_o) <= TOL_FP32
    assert rel_l2(gp2, -2 * q[:, None] * f_o) <= TOL_FP32_GRAD


@pytest.mark.parametrize("n,leaf", [(8348, 64), (16484, 128)])
def test_half_width_layout_mixed_leaves(F, orc, n, leaf):
    # leaves of floor / ceil(n / 4^L) points straddling half of the warp's
    # target slots (32 | 33 points with 64 slots, 64 | 65 with 128): the
    # potential kernel runs both layouts in one launch
    pos, q = workloads.uniform_cube(n, 38)
    T = F.fmm_build_tree(cuda(pos), 6, leaf, 2, 0.5, F.FMM_FP32C)
    O = orc.Tree(pos, leaf, 2, 0.5)
    u_o = O.eval(q, 6)
    u = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    F.fmm_tree_status(T)
    F.fmm_tree_set_option(T, F.FMM_OPT_NEAR_SYMMETRIC, 0)
    u1 = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    print("n %d leaf %d: sym %.2e one-sided %.2e" % (n, leaf, rel_l2(u, u_o), rel_l2(u1, u_o)))
    assert rel_l2(u, u_o) <= TOL_FP32
    assert rel_l2(u, u1) <= TOL_FP32
