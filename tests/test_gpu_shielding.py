"""Active-shielding inverse design (Sec. III.B) through the GPU FMM with
separate source/target trees and charge gradients, against the oracle's
closed-form optimum of the same quadratic loss (direct sums)."""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15269_gb300 import build, shielding
    build.build()
    return shielding


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32c"])
def test_shielding_descent_reaches_the_optimum(S, orc, precision):
    geo = workloads.active_shielding(seed=0)
    prob = S.ShieldingProblem(geo, p=8, leaf_size=16, theta=0.5, precision=precision)
    # potentials at a random shield state against the oracle's two-tree FMM
    # (parity) and the direct sum (the FMM truncation error)
    qr = np.random.default_rng(5).uniform(-0.05, 0.05, 128)
    phi_in, phi_out = (x.detach().cpu().numpy() for x in prob.potentials(torch.from_numpy(qr).cuda()))
    src_in = np.concatenate([geo["ext"], geo["shield"]])
    q_all = np.concatenate([geo["q_ext"], qr])
    o_in = orc.Tree2(src_in, geo["inside"], 16, 2, 0.5).eval(q_all, 8)
    o_out = orc.Tree2(geo["shield"], geo["outside"], 16, 2, 0.5).eval(qr, 8)
    tol = 1e-12 if precision == 0 else 3e-6
    for a, b in ((phi_in, o_in), (phi_out, o_out)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= tol
    q0 = torch.zeros(128, dtype=torch.float64, device="cuda")
    f_ref = orc.shielding_loss(geo, np.zeros(128))
    assert abs(float(prob.loss(q0)[0]) - f_ref[0]) <= 1e-3 * f_ref[0]
    q, hist = prob.optimise(100)
    assert all(b <= a * (1 + 1e-7) for a, b in zip(hist, hist[1:]))
    q_opt = orc.shielding_optimum(geo)
    f_opt = orc.shielding_loss(geo, q_opt)[0]
    qn = q.cpu().numpy()
    f_end = orc.shielding_loss(geo, qn)
    print("loss %.6e -> %.6e (optimum %.6e), L_in %.3e -> %.3e, q err %.2e" % (
        hist[0], hist[-1], f_opt, f_ref[1], f_end[1], np.linalg.norm(qn - q_opt) / np.linalg.norm(q_opt)))
    assert (f_end[0] - f_opt) <= 1e-3 * f_opt
    assert np.linalg.norm(qn - q_opt) / np.linalg.norm(q_opt) < 0.03
    assert f_end[1] < 0.05 * f_ref[1]
    prob.free()
