"""Pins of the oracle's active-shielding reference (Sec. III.B): the
closed-form minimiser is a stationary point of the loss (central finite
differences of the direct-sum loss), a minimum (random perturbations raise
the loss), and the optimised shield flattens the inner potential."""
import numpy as np

from paper_2511_15269_gb300 import workloads


def test_shielding_optimum_is_the_minimum(orc):
    geo = workloads.active_shielding(seed=0, n_sh=48, n_ext=64, n_in=256, n_out=256)
    q = orc.shielding_optimum(geo)
    f0 = orc.shielding_loss(geo, q)[0]
    h = 1e-4

    def fd(x, j):
        e = np.zeros(48)
        e[j] = h
        return (orc.shielding_loss(geo, x + e)[0] - orc.shielding_loss(geo, x - e)[0]) / (2 * h)

    scale = max(abs(fd(np.zeros(48), j)) for j in range(0, 48, 7))
    assert scale > 0
    for j in range(0, 48, 7):
        assert abs(fd(q, j)) < 1e-6 * scale
    rng = np.random.default_rng(1)
    for _ in range(5):
        assert orc.shielding_loss(geo, q + 1e-2 * rng.normal(size=48))[0] > f0


def test_shielding_flattens_the_inner_potential(orc):
    geo = workloads.active_shielding(seed=0)
    q = orc.shielding_optimum(geo)
    _, l_in0, l_out0, _ = orc.shielding_loss(geo, np.zeros(128))
    _, l_in, l_out, _ = orc.shielding_loss(geo, q)
    assert l_out0 == 0.0
    assert l_in < 0.05 * l_in0
    # the shield's outer potential stays comparable to the inner variance it removes
    assert 0.2 * l_out < l_in0
