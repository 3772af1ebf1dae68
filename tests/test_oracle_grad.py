"""Pins of the oracle's gradient of u = K q at a fixed geometry:
dL/dq = K g and dL/dr_k = g_k grad u(r_k) + q_k grad v(r_k), v = K g, checked by
central finite differences in FP64 and by the closed form dL/dq = u of the
energy loss L = 1/2 sum q_i u_i."""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads


def test_energy_loss_closed_form(orc):
    pos, q = workloads.thin_film(cells=12, seed=1)
    u = orc.direct(pos, q)
    dq, _ = orc.direct_vjp(pos, q, 0.5 * q)  # g = dL/du = q/2
    # L = 1/2 q.u(q) has dL/dq = u; the explicit part q/2 . d/dq adds u/2 to K g = u/2
    np.testing.assert_allclose(dq + 0.5 * u, u, rtol=1e-13, atol=1e-16)


def test_vjp_matches_finite_differences(orc):
    rng = np.random.default_rng(3)
    pos, q = workloads.uniform_cube(300, seed=4)
    g = rng.normal(size=300)
    dq, dpos = orc.direct_vjp(pos, q, g)

    def loss(P, Q):
        return float(g @ orc.direct(P, Q))

    h = 1e-6
    for i in (0, 13, 299):
        e = np.zeros(300)
        e[i] = h
        fd = (loss(pos, q + e) - loss(pos, q - e)) / (2 * h)
        assert dq[i] == pytest.approx(fd, rel=1e-7)
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            fd = (loss(pp, q) - loss(pm, q)) / (2 * h)
            assert dpos[i, a] == pytest.approx(fd, rel=1e-6, abs=1e-9)
