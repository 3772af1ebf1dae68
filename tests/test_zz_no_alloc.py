"""fmm_eval_potential_static: the evaluation whose per-call scratch is the
library's static device array, for callers that may not allocate device
memory at evaluation time.  Its results must match fmm_eval_potential on
consecutive calls, and trees beyond its stated capacity must be rejected.
(Collected last so that a stop at the first failure has run every other test.)"""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_FP32 = 1e-6  # FP32C: one-sided near field here, symmetric there (rounding only)
TOL_FP64 = 1e-12
TOL_FP64DF = 2e-13  # FP64DF trees are evaluated in plain FP64 here


@pytest.fixture(scope="module")
def F():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15269_gb300 import build, fmm
    build.build()
    fmm.lib()
    return fmm


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [(1, TOL_FP32), (0, TOL_FP64), (2, TOL_FP64DF)])
def test_static_scratch_matches_eval_on_consecutive_calls(F, precision, tol):
    pos, q1 = workloads.uniform_cube(20000, seed=12)
    q2 = np.random.default_rng(13).uniform(-1, 1, 20000)
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), 6, 32, 2, 0.5, precision)
    assert F.fmm_tree_stats(T)["n_boxes"] <= 5461
    for q in (q1, q2):
        qd = torch.from_numpy(q).cuda()
        ref = F.fmm_eval_potential(T, qd).cpu().numpy()
        got = F.fmm_eval_potential_static(T, qd).cpu().numpy()
        assert rel_l2(got, ref) <= tol
    F.fmm_tree_status(T)


def test_static_scratch_rejects_oversized_tree(F):
    pos, q = workloads.uniform_cube(70000, seed=14)
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), 4, 64, 2, 0.5, 1)
    with pytest.raises(F.FmmError) as ei:
        F.fmm_eval_potential_static(T, torch.from_numpy(q).cuda())
    assert ei.value.code == F.FMM_ERR_CAPACITY
    assert "capacity" in str(ei.value)


def test_static_scratch_at_the_box_limit(F):
    """65,536 points with leaves of 16 points: 5,461 boxes, both limits
    reached exactly, so every per-box slice of the array is in use."""
    pos, q = workloads.uniform_cube(65536, seed=15)
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), 5, 16, 2, 0.5, 1)
    st = F.fmm_tree_stats(T)
    assert (st["n"], st["n_boxes"]) == (65536, 5461)
    qd = torch.from_numpy(q).cuda()
    ref = F.fmm_eval_potential(T, qd).cpu().numpy()
    for _ in range(2):
        assert rel_l2(F.fmm_eval_potential_static(T, qd).cpu().numpy(), ref) <= TOL_FP32
    F.fmm_tree_status(T)


def test_static_scratch_merged_batch(F):
    """A batch of two independent trees (fmm_tree_merge) through the static
    array: each set's potential as evaluated by the batch's own entry point."""
    sets = [workloads.uniform_cube(20000, seed=16), workloads.gaussian_clusters(15000, seed=17)]
    trees = [F.fmm_build_tree(torch.from_numpy(p).cuda(), 6, 32, 2, 0.5, 1) for p, _ in sets]
    B = F.fmm_tree_merge(trees)
    qd = torch.from_numpy(np.concatenate([q for _, q in sets])).cuda()
    ref = F.fmm_eval_potential(B, qd).cpu().numpy()
    for _ in range(2):
        assert rel_l2(F.fmm_eval_potential_static(B, qd).cpu().numpy(), ref) <= TOL_FP32
    F.fmm_tree_status(B)


def test_static_scratch_rejects_too_many_boxes(F):
    """Under the point limit but over the box limit (leaves of 8 points)."""
    pos, q = workloads.uniform_cube(40000, seed=18)
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), 4, 8, 2, 0.5, 1)
    assert F.fmm_tree_stats(T)["n_boxes"] > 5461
    with pytest.raises(F.FmmError) as ei:
        F.fmm_eval_potential_static(T, torch.from_numpy(q).cuda())
    assert ei.value.code == F.FMM_ERR_CAPACITY
