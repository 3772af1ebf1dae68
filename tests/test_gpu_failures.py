"""Failure paths, made on purpose without any GPU fault.

* Timeout: the near-field warps wait for their staged source tiles with a
  bounded wait; a cycle limit of 0 makes every such wait give up before its
  first poll.  The kernels then latch FMM_ERR_TIMEOUT, let their copies in
  flight land and return, the host reads the status, and the context stays
  usable: the next evaluation with the default limit matches the oracle.
* Out of memory: a device-memory cap below the first allocation of a build
  makes that allocation fail as a refused cudaMalloc would; the build returns
  FMM_ERR_OOM, leaves no tree and holds no memory, and works once the cap is
  lifted.
"""
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,field", [(1, False), (1, True), (0, False), (2, False)])
def test_wait_timeout_is_reported_and_recovered(F, orc, precision, field):
    pos, q = workloads.uniform_cube(20000, seed=21)
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), 6, 64, 2, 0.5, precision)
    qd = torch.from_numpy(q).cuda()
    F.fmm_tree_set_wait_limit(T, 0)
    if field:
        F.fmm_eval_field(T, qd)
    else:
        F.fmm_eval_potential(T, qd)
    with pytest.raises(F.FmmError) as ei:
        F.fmm_tree_status(T)
    assert ei.value.code == F.FMM_ERR_TIMEOUT
    F.fmm_tree_status(T)  # the status was cleared by the read
    F.fmm_tree_set_wait_limit(T, 2000000000)
    u = F.fmm_eval_potential(T, qd).cpu().numpy()
    F.fmm_tree_status(T)
    uo = orc.Tree(pos, 64, 2, 0.5).eval(q, 6)
    assert rel_l2(u, uo) <= (1e-6 if precision == 1 else 1e-12)


def test_wait_timeout_in_the_backward_sweep(F, orc):
    # the symmetric backward sweep's tile waits: timeout reported, the tree
    # stays usable and the next backward pass is correct
    pos, q = workloads.uniform_cube(20000, seed=24)
    g = np.random.default_rng(5).normal(size=len(q))
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), 6, 64, 2, 0.5, 1)
    qd, gd = torch.from_numpy(q).cuda(), torch.from_numpy(g).cuda()
    F.fmm_tree_set_wait_limit(T, 0)
    F.fmm_backward(T, qd, gd)
    with pytest.raises(F.FmmError) as ei:
        F.fmm_tree_status(T)
    assert ei.value.code == F.FMM_ERR_TIMEOUT
    F.fmm_tree_set_wait_limit(T, 2000000000)
    gq, gp = (x.cpu().numpy() for x in F.fmm_backward(T, qd, gd))
    F.fmm_tree_status(T)
    O = orc.Tree(pos, 64, 2, 0.5)
    _, fq = O.eval(q, 6, field=True)
    v, fg = O.eval(g, 6, field=True)
    assert rel_l2(gq, v) <= 1e-6
    assert rel_l2(gp, -(g[:, None] * fq + q[:, None] * fg)) <= 3e-5


def test_wait_limit_rejects_negative(F):
    pos, _ = workloads.uniform_cube(1000, seed=22)
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), 4, 32, 2, 0.5, 1)
    with pytest.raises(F.FmmError) as ei:
        F.fmm_tree_set_wait_limit(T, -1)
    assert ei.value.code == F.FMM_ERR_INVALID_ARG


def test_memory_cap_gives_oom_and_recovers(F, orc):
    pos, q = workloads.uniform_cube(50000, seed=23)
    pd = torch.from_numpy(pos).cuda()
    before = F.fmm_device_memory_in_use()
    F.fmm_set_device_memory_limit(before + 1024)
    try:
        with pytest.raises(F.FmmError) as ei:
            F.fmm_build_tree(pd, 6, 64, 2, 0.5, 1)
        assert ei.value.code == F.FMM_ERR_OOM
        assert "limit" in str(ei.value)
        assert F.fmm_device_memory_in_use() == before
    finally:
        F.fmm_set_device_memory_limit(0)
    T = F.fmm_build_tree(pd, 6, 64, 2, 0.5, 1)
    assert F.fmm_device_memory_in_use() >= before + F.fmm_tree_stats(T)["device_bytes"]
    u = F.fmm_eval_potential(T, torch.from_numpy(q).cuda()).cpu().numpy()
    F.fmm_tree_status(T)
    assert rel_l2(u, orc.Tree(pos, 64, 2, 0.5).eval(q, 6)) <= 1e-6
    T.free()
    assert F.fmm_device_memory_in_use() == before
