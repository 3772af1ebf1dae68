"""The rest of the C-ABI boundary: positions as three arrays (FMM_POS_SOA),
a caller-owned evaluation workspace (fmm_tree_workspace_bytes /
fmm_tree_set_workspace) and batched charge sets (fmm_eval_batched), each
against the plain entry points on the same inputs."""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15269_gb300 import build, fmm
    build.build()
    fmm.lib()
    return fmm


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_soa_positions_build_the_same_tree(F):
    pos, q = workloads.plummer_sphere(30000, seed=31)
    A = F.fmm_build_tree(cuda(pos), 6, 32, 2, 0.5, F.FMM_FP32C)
    B = F.fmm_build_tree(cuda(pos.T), 6, 32, 2, 0.5, F.FMM_FP32C, F.FMM_POS_SOA)
    ea, eb = F.fmm_tree_export(A), F.fmm_tree_export(B)
    for k in ("perm", "box_start", "box_count", "m2l_trg", "m2l_src", "p2p_trg", "p2p_src"):
        np.testing.assert_array_equal(ea[k], eb[k])
    np.testing.assert_array_equal(ea["center"].view(np.uint64), eb["center"].view(np.uint64))
    qd = cuda(q)
    np.testing.assert_array_equal(F.fmm_eval_potential(A, qd).cpu().numpy(),
                                  F.fmm_eval_potential(B, qd).cpu().numpy())
    F.fmm_tree_status(B)


def test_soa_two_hierarchies(F, orc):
    sp, q = workloads.uniform_cube(8000, seed=32)
    tp = workloads.uniform_cube(3000, seed=33)[0]
    A = F.fmm_build_tree2(cuda(sp), cuda(tp), 6, 32, 2, 0.5, F.FMM_FP64)
    B = F.fmm_build_tree2(cuda(sp.T), cuda(tp.T), 6, 32, 2, 0.5, F.FMM_FP64, F.FMM_POS_SOA)
    qd = cuda(q)
    np.testing.assert_array_equal(F.fmm_eval_potential(A, qd).cpu().numpy(),
                                  F.fmm_eval_potential(B, qd).cpu().numpy())


@pytest.mark.parametrize("precision", [1, 0])
def test_caller_workspace(F, orc, precision):
    pos, q = workloads.uniform_cube(40000, seed=34)
    T = F.fmm_build_tree(cuda(pos), 6, 64, 2, 0.5, precision)
    qd = cuda(q)
    ref = F.fmm_eval_potential(T, qd).cpu().numpy()
    own = F.fmm_tree_stats(T)["device_bytes"]
    nb = F.fmm_tree_workspace_bytes(T)
    assert 0 < nb < own
    with pytest.raises(F.FmmError) as ei:
        F.fmm_tree_set_workspace(T, torch.empty(nb - 256, dtype=torch.uint8, device="cuda"))
    assert ei.value.code == F.FMM_ERR_CAPACITY
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    F.fmm_tree_set_workspace(T, ws)
    assert F.fmm_tree_stats(T)["device_bytes"] <= own - nb + 8192
    for _ in range(2):
        np.testing.assert_array_equal(F.fmm_eval_potential(T, qd).cpu().numpy(), ref)
    F.fmm_tree_status(T)
    F.fmm_tree_set_workspace(T, None)
    np.testing.assert_array_equal(F.fmm_eval_potential(T, qd).cpu().numpy(), ref)
    F.fmm_tree_status(T)


def test_caller_workspace_and_a_new_precision(F, orc):
    pos, q = workloads.uniform_cube(20000, seed=35)
    T = F.fmm_build_tree(cuda(pos), 6, 64, 2, 0.5, F.FMM_FP32C)
    F.fmm_tree_set_workspace(T, torch.empty(F.fmm_tree_workspace_bytes(T), dtype=torch.uint8, device="cuda"))
    with pytest.raises(F.FmmError) as ei:
        F.fmm_tree_set_precision(T, F.FMM_FP64)
    assert ei.value.code == F.FMM_ERR_INVALID_ARG
    F.fmm_tree_set_workspace(T, None)
    F.fmm_tree_set_precision(T, F.FMM_FP64)
    F.fmm_tree_set_workspace(T, torch.empty(F.fmm_tree_workspace_bytes(T), dtype=torch.uint8, device="cuda"))
    u = F.fmm_eval_potential(T, cuda(q)).cpu().numpy()
    F.fmm_tree_status(T)
    assert rel_l2(u, orc.Tree(pos, 64, 2, 0.5).eval(q, 6)) <= 1e-12


def test_eval_batched_matches_the_concatenated_evaluation(F):
    sets = [workloads.uniform_cube(12000, seed=36), workloads.gaussian_clusters(7000, seed=37),
            workloads.plummer_sphere(20000, seed=38)]
    trees = [F.fmm_build_tree(cuda(p), 6, 32, 2, 0.6, F.FMM_FP32C) for p, _ in sets]
    B = F.fmm_tree_merge(trees)
    q_sets = [cuda(q) for _, q in sets]
    ref = F.fmm_eval_potential(B, torch.cat(q_sets)).cpu().numpy()
    off = F.fmm_tree_point_offsets(B)
    u_sets = F.fmm_eval_batched(B, q_sets)
    for k, u in enumerate(u_sets):
        np.testing.assert_array_equal(u.cpu().numpy(), ref[off[k]:off[k + 1]])
    # captured once in a CUDA graph and replayed with new charges in place
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        F.fmm_eval_batched(B, q_sets, u_sets)
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.fmm_eval_batched(B, q_sets, u_sets)
    rng = np.random.default_rng(39)
    new = [rng.uniform(-1, 1, len(q)) for _, q in sets]
    for k in range(3):
        q_sets[k].copy_(cuda(new[k]))
    g.replay()
    torch.cuda.synchronize()
    ref2 = F.fmm_eval_potential(B, torch.cat(q_sets)).cpu().numpy()
    for k, u in enumerate(u_sets):
        np.testing.assert_array_equal(u.cpu().numpy(), ref2[off[k]:off[k + 1]])
    F.fmm_tree_status(B)
    with pytest.raises(F.FmmError):
        F.fmm_eval_batched(B, q_sets[:2])


def test_pool_retention(F):
    # unused pool memory after a tree is freed: kept up to the retention,
    # given back with retention 0; a rebuild from kept memory gives the same
    # tree
    pos, q = workloads.uniform_cube(300000, seed=41)
    pd, qd = cuda(pos), cuda(q)
    torch.cuda.synchronize()
    F.fmm_set_pool_retention(0)
    free0 = torch.cuda.mem_get_info()[0]
    try:
        F.fmm_set_pool_retention(2 << 30)
        T = F.fmm_build_tree(pd, 6, 64, 2, 0.5, F.FMM_FP32C)
        tree_bytes = F.fmm_tree_stats(T)["device_bytes"]
        u_a = F.fmm_eval_potential(T, qd).cpu().numpy()
        T.free()
        kept = free0 - torch.cuda.mem_get_info()[0]
        assert tree_bytes <= kept <= (2 << 30) + (64 << 20)
        T = F.fmm_build_tree(pd, 6, 64, 2, 0.5, F.FMM_FP32C)
        u_b = F.fmm_eval_potential(T, qd).cpu().numpy()
        np.testing.assert_array_equal(u_a, u_b)
        T.free()
        F.fmm_set_pool_retention(0)
        assert free0 - torch.cuda.mem_get_info()[0] <= (64 << 20)
    finally:
        F.fmm_set_pool_retention(2 << 30)
