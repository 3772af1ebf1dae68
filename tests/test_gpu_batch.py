"""Batches of independent charge sets (fmm_tree_merge): one evaluation over a
merged batch must reproduce, bit for bit, the evaluations of its trees one by
one (every stage computes each tree's boxes and leaves the same way, only in
one launch), in both precisions, for potentials, fields and gradients; a
CUDA-graph replay must reproduce the eager result."""
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


def batch_inputs():
    sets = [(workloads.uniform_cube(3000, 1), 16), (workloads.gaussian_clusters(5000, 2), 32),
            (workloads.plummer_sphere(8000, 3), 64), (workloads.thin_film(20, 4), 8),
            (workloads.uniform_cube(60, 5), 64), (workloads.gaussian_clusters(12000, 6), 128)]
    return sets


@pytest.mark.parametrize("precision", [1, 0])
def test_batch_matches_single_trees(F, orc, precision):
    p = 6
    sets = batch_inputs()
    trees = [F.fmm_build_tree(cuda(pos), p, leaf, 2, 0.6, precision) for (pos, q), leaf in sets]
    B = F.fmm_tree_merge(trees)
    st = F.fmm_tree_stats(B)
    assert st["n_trees"] == len(sets)
    assert st["n"] == sum(len(q) for (pos, q), _ in sets)
    assert st["n_m2l"] == sum(F.fmm_tree_stats(t)["n_m2l"] for t in trees)
    off = F.fmm_tree_point_offsets(B)
    q_all = np.concatenate([q for (pos, q), _ in sets])
    u_b = F.fmm_eval_potential(B, cuda(q_all)).cpu().numpy()
    ub_f, fb = (x.cpu().numpy() for x in F.fmm_eval_field(B, cuda(q_all)))
    g_all = np.random.default_rng(7).normal(size=len(q_all))
    gq_b, gp_b = (x.cpu().numpy() for x in F.fmm_backward(B, cuda(q_all), cuda(g_all)))
    for k, (t, ((pos, q), leaf)) in enumerate(zip(trees, sets)):
        sl = slice(off[k], off[k + 1])
        np.testing.assert_array_equal(u_b[sl], F.fmm_eval_potential(t, cuda(q)).cpu().numpy())
        u1, f1 = (x.cpu().numpy() for x in F.fmm_eval_field(t, cuda(q)))
        np.testing.assert_array_equal(ub_f[sl], u1)
        np.testing.assert_array_equal(fb[sl], f1)
        gq1, gp1 = (x.cpu().numpy() for x in F.fmm_backward(t, cuda(q), cuda(g_all[sl])))
        np.testing.assert_array_equal(gq_b[sl], gq1)
        np.testing.assert_array_equal(gp_b[sl], gp1)
    # and against the oracle for one member
    (pos, q), leaf = sets[2]
    O = orc.Tree(pos, leaf, 2, 0.6)
    uo = O.eval(q, p)
    err = np.linalg.norm(u_b[off[2]:off[3]] - uo) / np.linalg.norm(uo)
    assert err <= (1e-12 if precision == 0 else 3e-6)
    F.fmm_tree_status(B)


def test_batch_graph_replay(F):
    sets = batch_inputs()
    trees = [F.fmm_build_tree(cuda(pos), 6, leaf, 2, 0.6, 1) for (pos, q), leaf in sets]
    B = F.fmm_tree_merge(trees)
    q_all = cuda(np.concatenate([q for (pos, q), _ in sets]))
    u = torch.empty_like(q_all)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            F.fmm_eval_potential(B, q_all, out=u)
    torch.cuda.current_stream().wait_stream(side)
    eager = u.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        F.fmm_eval_potential(B, q_all, out=u)
    u.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, eager)
    F.fmm_tree_status(B)


def test_merge_rejects_mismatched_trees(F):
    a = F.fmm_build_tree(cuda(workloads.uniform_cube(500, 1)[0]), 4, 32, 2, 0.5, 1)
    b = F.fmm_build_tree(cuda(workloads.uniform_cube(500, 2)[0]), 6, 32, 2, 0.5, 1)
    with pytest.raises(F.FmmError) as ei:
        F.fmm_tree_merge([a, b])
    assert ei.value.code == F.FMM_ERR_INVALID_ARG
