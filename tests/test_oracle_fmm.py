"""End-to-end pins of the oracle FMM against the direct sum of Eq. 1-3:
geometric error decay in p under the Eq. 5 bound form, the config tolerance,
a single charge, the energy sum, fields, and the sampled-target path."""
import numpy as np
import pytest

from paper_2511_15269_gb300 import workloads


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cube2k():
    return workloads.uniform_cube(2000, seed=0)


def test_error_decays_geometrically_with_p(orc, cube2k):
    pos, q = cube2k
    ud = orc.direct(pos, q)
    theta = 0.6
    T = orc.Tree(pos, 32, 2, theta)
    errs = {p: rel_l2(T.eval(q, p), ud) for p in (2, 4, 6, 8, 10)}
    ps = sorted(errs)
    for a, b in zip(ps, ps[1:]):
        assert errs[b] < errs[a] * 0.5, errs
    # below the bound form theta^(p+1)/(1-theta)^2 up to one constant
    ratio = [errs[p] * (1 - theta) ** 2 / theta ** (p + 1) for p in ps]
    assert max(ratio[1:]) <= ratio[0] * 1.5
    assert errs[10] < 1e-6


def test_effective_theta_below_theta(orc, cube2k):
    """Sec. III.A: solving Eq. 4 for theta per interaction gives an effective
    value below the bound theta."""
    pos, _ = cube2k
    theta = 0.7
    T = orc.Tree(pos, 32, 2, theta)
    d = np.linalg.norm(T.center[T.m2l_src] - T.center[T.m2l_trg], axis=1)
    R = np.maximum(T.radius[T.m2l_src], T.radius[T.m2l_trg])
    r = np.minimum(T.radius[T.m2l_src], T.radius[T.m2l_trg])
    th_eff = R / (d - r)
    assert np.all(th_eff <= theta * (1 + 1e-12))
    assert th_eff.mean() < theta


def test_config_cube4k_p4_tolerance(orc):
    c = workloads.CONFIGS["cube4k_p4"]
    pos, q = workloads.uniform_cube(c["n"], seed=0)
    T = orc.Tree(pos, c["leaf_size"], c["s"], c["theta"])
    assert rel_l2(T.eval(q, c["p"]), orc.direct(pos, q)) < 1e-4


def test_single_charge(orc):
    pos, _ = workloads.uniform_cube(1500, seed=2)
    q = np.zeros(1500)
    q[123] = 2.5
    T = orc.Tree(pos, 16, 2, 0.5)
    u = T.eval(q, 10)
    r = np.linalg.norm(pos - pos[123], axis=1)
    want = np.where(r > 0, -2.5 / (4 * np.pi * np.where(r > 0, r, 1)), 0.0)
    assert u[123] == 0.0
    assert rel_l2(u, want) < 1e-7


def test_energy_and_field(orc, cube2k):
    pos, q = cube2k
    T = orc.Tree(pos, 32, 2, 0.5)
    u, f = T.eval(q, 10, field=True)
    ud, fd = orc.direct(pos, q, field=True)
    assert float(q @ u) == pytest.approx(float(q @ ud), rel=1e-6)
    assert rel_l2(f, fd) < 1e-6
    # field of the direct sum against central differences of the direct potential
    h = 1e-6
    for i in (0, 77, 1999):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            up = orc.direct(pp, q, targets=[i])[0]
            um = orc.direct(pm, q, targets=[i])[0]
            assert fd[i, a] == pytest.approx(-(up - um) / (2 * h), rel=1e-6, abs=1e-8)


def test_sampled_targets_match_full(orc):
    pos, q = workloads.plummer_sphere(3000, seed=5)
    T = orc.Tree(pos, 16, 2, 0.5)
    u, f = T.eval(q, 6, field=True)
    tg = workloads.sample_targets(3000, 100, seed=3)
    us, fs = T.eval(q, 6, targets=tg, field=True)
    np.testing.assert_array_equal(us, u[tg])
    np.testing.assert_array_equal(fs, f[tg])


def test_ties_input_runs(orc):
    pos, q = workloads.thin_film(cells=24, seed=0)
    T = orc.Tree(pos, 32, 2, 0.5)
    assert rel_l2(T.eval(q, 8), orc.direct(pos, q)) < 1e-4
