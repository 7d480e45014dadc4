"""Pins of the oracle's 4th-order Hermite variant (Makino & Aarseth 1992):
predictor through jerk, corrector, cubic interpolation of the acceleration,
Aarseth's time-step criterion, and whole-run behaviour (Kepler closed form
and convergence order 4, conservation, the block-step run).

Paper: Sec. 2 (the code derives from HiGPUs, whose Hermite family this is
the 4th-order member of).  Formulas: Makino & Aarseth 1992, PASJ 44, 141.
"""
import math

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from paper_1812_00367_gb300 import ic


def _derivs(coef, t, kmax):
    out = []
    c = np.array(coef, dtype=np.float64)
    for _ in range(kmax + 1):
        out.append(P.polyval(t, c))
        c = P.polyder(c) if c.size > 1 else np.zeros(1)
    return out


def test_predictor4_exact_for_cubics(oracle):
    rng = np.random.default_rng(41)
    n = 6
    t0 = rng.uniform(0, 1, n)
    t1 = 1.5
    coefs = rng.normal(size=(n, 3, 4))
    f = {k: np.zeros((n, 3)) for k in "xvaj"}
    ref = {k: np.zeros((n, 3)) for k in "xv"}
    for i in range(n):
        for d in range(3):
            dv = _derivs(coefs[i, d], t0[i], 3)
            for k, name in enumerate("xvaj"):
                f[name][i, d] = dv[k]
            dv1 = _derivs(coefs[i, d], t1, 1)
            ref["x"][i, d], ref["v"][i, d] = dv1
    xp, vp = oracle.predict4(f["x"], f["v"], f["a"], f["j"], t0, t1)
    np.testing.assert_allclose(xp, ref["x"], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(vp, ref["v"], rtol=1e-13, atol=1e-13)


def test_predictor4_ignores_snap_terms(oracle):
    """A quartic trajectory is not predicted exactly: the truncation error is
    the dropped snap term, s d^4/24 in x and s d^3/6 in v."""
    coef = np.array([0.3, -0.2, 0.1, 0.4, 1.0])   # x(t), snap = 24
    t0, t1 = 0.0, 0.5
    dv = _derivs(coef, t0, 3)
    f = [np.array([[q, 0.0, 0.0]]) for q in dv]
    xp, vp = oracle.predict4(*f, np.array([t0]), t1)
    x1, v1 = _derivs(coef, t1, 1)
    assert x1 - xp[0, 0] == pytest.approx(24 * 0.5 ** 4 / 24, rel=1e-12)
    assert v1 - vp[0, 0] == pytest.approx(24 * 0.5 ** 3 / 6, rel=1e-12)


def test_corrector4_exact_for_degree4(oracle):
    rng = np.random.default_rng(42)
    for _ in range(5):
        t0, h = rng.uniform(-1, 1), 2.0 ** -rng.integers(0, 6)
        t1 = t0 + h
        coef = rng.normal(size=(3, 5))   # x(t) of degree 4
        q = lambda t, k: np.array([_derivs(coef[d], t, 3)[k] for d in range(3)])
        x1, v1 = oracle.correct4(h, q(t0, 0), q(t0, 1), q(t0, 2), q(t0, 3),
                                 q(t1, 2), q(t1, 3))
        np.testing.assert_allclose(x1, q(t1, 0), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(v1, q(t1, 1), rtol=1e-12, atol=1e-12)


def test_corrector4_velocity_exact_for_degree5(oracle):
    """The velocity rule integrates a cubic acceleration exactly (x of degree
    5); the position rule is then no longer exact (order check)."""
    rng = np.random.default_rng(43)
    t0, h = 0.2, 0.5
    t1 = t0 + h
    coef = rng.normal(size=(3, 6))
    coef[:, 5] = 1.0
    q = lambda t, k: np.array([_derivs(coef[d], t, 3)[k] for d in range(3)])
    x1, v1 = oracle.correct4(h, q(t0, 0), q(t0, 1), q(t0, 2), q(t0, 3), q(t1, 2), q(t1, 3))
    np.testing.assert_allclose(v1, q(t1, 1), rtol=1e-12, atol=1e-12)
    assert np.abs(x1 - q(t1, 0)).max() > 1e-6


def test_interp4_recovers_cubic(oracle):
    rng = np.random.default_rng(44)
    for _ in range(5):
        t0, h = rng.uniform(-1, 1), 2.0 ** -rng.integers(1, 8)
        t1 = t0 + h
        coef = rng.normal(size=(3, 4))   # a(t) cubic
        at = lambda t, k: np.array([_derivs(coef[d], t, 3)[k] for d in range(3)])
        s1, c1 = oracle.interp4(h, at(t0, 0), at(t0, 1), at(t1, 0), at(t1, 1))
        scale = 1e3 * np.finfo(float).eps / h ** 3
        np.testing.assert_allclose(s1, at(t1, 2), rtol=1e-9, atol=scale)
        np.testing.assert_allclose(c1, 6 * coef[:, 3], rtol=1e-9, atol=scale)


def test_aarseth_exponential_ladder(oracle):
    """a^(k) = lam^k u: (2 lam^2 |u|^2) / (2 lam^4 |u|^2) -> dt = sqrt(eta) / lam."""
    rng = np.random.default_rng(45)
    for _ in range(10):
        lam = 10 ** rng.uniform(-3, 3)
        u = rng.normal(size=3)
        ladder = [lam ** k * u for k in range(4)]
        eta = rng.uniform(0.005, 0.05)
        assert oracle.dt_aarseth(*ladder, eta) == pytest.approx(math.sqrt(eta) / lam, rel=1e-12)
        # the start-up rule without snap: eta_init |a| / |j|
        assert oracle.dt_initial(ladder[0], ladder[1], np.zeros(3), eta) == \
            pytest.approx(eta / lam, rel=1e-12)


def test_aarseth_pairs_the_right_norms(oracle):
    """Distinct norms |a|=1, |j|=2, |s|=3, |c|=4 in orthogonal directions:
    (1*3 + 2^2) / (2*4 + 3^2) = 7/17.  Swapping any two derivatives changes it."""
    a, j, s, c = np.eye(3)[0], 2 * np.eye(3)[1], 3 * np.eye(3)[2], 4 * np.eye(3)[0]
    assert oracle.dt_aarseth(a, j, s, c, 0.02) == pytest.approx(math.sqrt(0.02 * 7 / 17), rel=1e-14)
    assert oracle.dt_aarseth(a, s, j, c, 0.02) != pytest.approx(math.sqrt(0.02 * 7 / 17))
    z = np.zeros(3)
    assert oracle.dt_aarseth(z, z, z, z, 0.02) == math.inf


def test_aarseth_time_rescaling(oracle):
    rng = np.random.default_rng(46)
    ladder = [rng.normal(size=3) * 10 ** rng.uniform(-1, 1) for _ in range(4)]
    base = oracle.dt_aarseth(*ladder, 0.02)
    for kappa in (0.01, 0.5, 3.0, 1e3):
        scaled = [q * kappa ** -k for k, q in enumerate(ladder)]
        assert oracle.dt_aarseth(*scaled, 0.02) == pytest.approx(kappa * base, rel=1e-12)


def _kepler_state(t, a=1.0, e=0.5, mu=1.0):
    n_mean = math.sqrt(mu / a ** 3)
    M = n_mean * t
    E = M
    for _ in range(100):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    den = 1 - e * math.cos(E)
    r = np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])
    v = np.array([-a * n_mean * math.sin(E) / den,
                  a * n_mean * math.sqrt(1 - e * e) * math.cos(E) / den, 0.0])
    return r, v


def _kepler_run4(oracle, h, orbits=4):
    m = np.array([0.5, 0.5])
    r0, v0 = _kepler_state(0.0)
    x = np.stack([-0.5 * r0, 0.5 * r0]); v = np.stack([-0.5 * v0, 0.5 * v0])
    sim = oracle.Sim(m, x, v, eps=0.0, eta=0.02, dt_min=h, dt_max=h, order=4).init()
    t_end = math.floor(orbits * 2 * math.pi / h) * h
    sim.run(t_end)
    assert np.all(sim.t == t_end)
    r_ref, _ = _kepler_state(t_end)
    return np.linalg.norm((sim.x[1] - sim.x[0]) - r_ref)


def test_kepler4_closed_form_and_order(oracle):
    """e = 0.5, eps = 0, shared steps: close to Kepler's equation solution,
    and the global error falls ~2^4 per halving of dt."""
    e1 = _kepler_run4(oracle, 2.0 ** -7)
    e2 = _kepler_run4(oracle, 2.0 ** -8)
    assert e1 < 1e-3
    order = math.log2(e1 / e2)
    assert 3.5 < order < 4.6, order


def test_order4_momentum_and_energy(oracle):
    m, x, v = ic.plummer(128, seed=47)
    sim = oracle.Sim(m, x, v, eps=1e-2, eta=0.02, order=4).init()
    ek0, ep0, P0, L0 = sim.energy(0.0)
    sim.run(0.25)
    ek1, ep1, P1, L1 = sim.energy(0.25)
    assert np.all(sim.t == 0.25)
    assert sim.underflows == 0
    assert abs((ek1 + ep1) - (ek0 + ep0)) / abs(ek0 + ep0) < 1e-7
    assert np.linalg.norm(P1 - P0) < 1e-6
    # one start-up pass, then every block step evaluates its active set
    assert sim.interactions >= 128 * 127 * (1 + sim.block_steps) / 128


def test_order_argument_checked(oracle):
    m, x, v = ic.plummer(8, seed=48)
    with pytest.raises(ValueError):
        oracle.Sim(m, x, v, eps=1e-2, order=5)
