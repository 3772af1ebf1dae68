"""Thin-film differentiation workload: surface charges of a 256 x 256 x 2
face grid (N = 131072), loss L = 1/2 sum_i q_i u_i, gradients with respect to
charges and positions through FMMPotential (fmm_backward), p = 8.

Checks: central finite differences of the FP64 FMM loss (h = 1e-6) at sampled
coordinates, the direct-sum gradient on sampled points (dL/dq = u and
dL/dr_k = q_k grad u(r_k) = -q_k E_k for this loss), and FP32C against FP64."""
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
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def film_loss_and_grads(F, pos, q, precision):
    c = workloads.CONFIGS["film131k_p8"]
    T = F.fmm_build_tree(torch.from_numpy(pos).cuda(), c["p"], c["leaf_size"], c["s"], c["theta"], precision)
    P = torch.from_numpy(pos).cuda().requires_grad_(True)
    Q = torch.from_numpy(q).cuda().requires_grad_(True)
    u = F.FMMPotential.apply(P, Q, T)
    L = 0.5 * (Q * u).sum()
    L.backward()
    F.fmm_tree_status(T)
    return T, float(L), Q.grad.cpu().numpy(), P.grad.cpu().numpy(), u.detach().cpu().numpy()


def test_film_gradients(F, orc):
    pos, q = workloads.thin_film(256, 0)
    n = len(q)
    assert n == 131072
    T, L64, gq64, gp64, u64 = film_loss_and_grads(F, pos, q, F.FMM_FP64)
    _, L32, gq32, gp32, _ = film_loss_and_grads(F, pos, q, F.FMM_FP32C)
    # direct-sum gradient on sampled points
    tg = workloads.sample_targets(n, 1024, seed=5)
    ud, fd = orc.direct(pos, q, targets=tg, field=True)
    print("film: dq vs direct %.3e, dpos vs direct %.3e, fp32c dq vs fp64 %.3e, dpos %.3e" % (
        rel_l2(gq64[tg], ud), rel_l2(gp64[tg], -q[tg, None] * fd),
        rel_l2(gq32, gq64), rel_l2(gp32, gp64)))
    assert rel_l2(gq64[tg], ud) < 1e-4
    assert rel_l2(gp64[tg], -q[tg, None] * fd) < 1e-3
    assert rel_l2(gq32, gq64) < 3e-6
    assert rel_l2(gp32, gp64) < 3e-5
    # central finite differences (h = 1e-6, FP64) of the direct-sum loss.  r_i
    # and q_i enter L = 1/2 sum_ij q_i q_j K_ij only through row and column i,
    # so L(x + h) - L(x - h) reduces to the row energy E_i = q_i sum_j q_j K_ij.
    def row_energy(r, i):
        d = np.linalg.norm(pos - r, axis=1)
        d[i] = np.inf
        return -q[i] * np.sum(q / d) / (4 * np.pi)

    h = 1e-6
    rms = np.sqrt(np.mean(gp64 ** 2))
    rng = np.random.default_rng(6)
    for i in rng.choice(n, 6, replace=False):
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fdg = (row_energy(pos[i] + e, i) - row_energy(pos[i] - e, i)) / (2 * h)
            assert abs(gp64[i, a] - fdg) <= 2e-3 * max(abs(fdg), rms), (i, a, gp64[i, a], fdg)
        # dL/dq_i: the loss is quadratic in q, the central difference is u_i
        d = np.linalg.norm(pos - pos[i], axis=1)
        d[i] = np.inf
        fdq = -np.sum(q / d) / (4 * np.pi)
        assert abs(gq64[i] - fdq) <= 2e-4 * max(abs(fdq), np.sqrt(np.mean(gq64 ** 2)))
