"""Pins of the oracle's integrator: predictor, corrector, quintic interpolation,
time-step criterion, power-of-two quantisation, block scheduler, and whole-run
behaviour (Kepler closed form and convergence order, conservation laws,
finite differences along a trajectory).

Paper: Sec. 2 (Hermite 6th order time integrator, derived from HiGPUs).
Formulas: Nitadori & Makino 2008; block steps: Makino 1991 / Aarseth 2003.
"""
import math

import numpy as np
import numpy.polynomial.polynomial as P
import pytest

from paper_1812_00367_gb300 import ic


def _derivs(coef, t, kmax):
    """Values of d^k/dt^k of the polynomial (ascending coef) at t, k=0..kmax."""
    out = []
    c = np.array(coef, dtype=np.float64)
    for _ in range(kmax + 1):
        out.append(P.polyval(t, c) if c.size else 0.0)
        c = P.polyder(c) if c.size > 1 else np.zeros(1)
    return out


# ------------------------------------------------------------------ predictor
def test_predictor_exact_for_quintics(oracle):
    rng = np.random.default_rng(1)
    n = 5
    t0 = rng.uniform(0, 1, n)
    t1 = 1.25
    coefs = rng.normal(size=(n, 3, 6))
    fields = {k: np.zeros((n, 3)) for k in "xvajsc"}
    ref = {k: np.zeros((n, 3)) for k in "xva"}
    for i in range(n):
        for d in range(3):
            dv = _derivs(coefs[i, d], t0[i], 5)
            for k, name in enumerate("xvajsc"):
                fields[name][i, d] = dv[k]
            dv1 = _derivs(coefs[i, d], t1, 2)
            for k, name in enumerate("xva"):
                ref[name][i, d] = dv1[k]
    xp, vp, ap = oracle.predict(*(fields[k] for k in "xvajsc"), t0, t1)
    np.testing.assert_allclose(xp, ref["x"], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(vp, ref["v"], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(ap, ref["a"], rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------- interpolation
def test_interpolation_recovers_quintic(oracle):
    rng = np.random.default_rng(2)
    for trial in range(5):
        t0, h = rng.uniform(-1, 1), 2.0 ** -rng.integers(1, 8)
        t1 = t0 + h
        coef = rng.normal(size=(3, 6))
        at = lambda t, k: np.array([_derivs(coef[d], t, 5)[k] for d in range(3)])
        d3, d4, d5 = oracle.interp_derivs(h, at(t0, 0), at(t0, 1), at(t0, 2),
                                          at(t1, 0), at(t1, 1), at(t1, 2))
        # round-off bound: data of size D(T) = max(|a|, |j| T, |s| T^2) fixes
        # the k-th derivative only to ~ u D(T) / T^k (T = h/2)
        T = h / 2
        D = max(np.abs(at(t, 0)).max() + np.abs(at(t, 1)).max() * T + np.abs(at(t, 2)).max() * T * T
                for t in (t0, t1))
        for got, k in ((d3, 3), (d4, 4), (d5, 5)):
            ref = at(t1, k)
            tol = 1e3 * np.finfo(float).eps * D / T ** k
            assert np.abs(got - ref).max() <= tol, (k, got, ref, tol)


def test_interpolation_matches_6x6_solve(oracle):
    """Arbitrary end data: derivatives equal those of the Hermite quintic from
    a direct 6x6 linear solve in powers of (t - t1)."""
    rng = np.random.default_rng(3)
    h = 0.37
    data = rng.normal(size=(6, 3))
    d3, d4, d5 = oracle.interp_derivs(h, *data)
    # unknowns b_k: a(t) = sum b_k u^k, u = t - t1 in {-h, 0}
    M = np.zeros((6, 6))
    for row, (u, order) in enumerate([(-h, 0), (-h, 1), (-h, 2), (0.0, 0), (0.0, 1), (0.0, 2)]):
        for k in range(6):
            if k >= order:
                M[row, k] = math.factorial(k) / math.factorial(k - order) * u ** (k - order)
    b = np.linalg.solve(M, data)
    np.testing.assert_allclose(d3, 6 * b[3], rtol=1e-10)
    np.testing.assert_allclose(d4, 24 * b[4], rtol=1e-10)
    np.testing.assert_allclose(d5, 120 * b[5], rtol=1e-10)


# ----------------------------------------------------------------- corrector
def test_corrector_exact_for_degree6(oracle):
    rng = np.random.default_rng(4)
    for trial in range(5):
        t0, h = rng.uniform(-1, 1), 2.0 ** -rng.integers(0, 6)
        t1 = t0 + h
        coef = rng.normal(size=(3, 7))   # x(t) of degree 6
        q = lambda t, k: np.array([_derivs(coef[d], t, 4)[k] for d in range(3)])
        x1, v1 = oracle.correct(h, q(t0, 0), q(t0, 1), q(t0, 2), q(t0, 3), q(t0, 4),
                                q(t1, 2), q(t1, 3), q(t1, 4))
        np.testing.assert_allclose(x1, q(t1, 0), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(v1, q(t1, 1), rtol=1e-12, atol=1e-12)


def test_corrector_velocity_exact_for_degree7(oracle):
    """The velocity rule integrates a quintic acceleration exactly (x of
    degree 7); the position rule then is no longer exact (order check)."""
    rng = np.random.default_rng(5)
    t0, h = 0.1, 0.5
    t1 = t0 + h
    coef = rng.normal(size=(3, 8))
    coef[:, 7] = 1.0
    q = lambda t, k: np.array([_derivs(coef[d], t, 4)[k] for d in range(3)])
    x1, v1 = oracle.correct(h, q(t0, 0), q(t0, 1), q(t0, 2), q(t0, 3), q(t0, 4),
                            q(t1, 2), q(t1, 3), q(t1, 4))
    np.testing.assert_allclose(v1, q(t1, 1), rtol=1e-12, atol=1e-12)
    assert np.abs(x1 - q(t1, 0)).max() > 1e-8


# ----------------------------------------------------------------- time step
def test_criterion_exponential_ladder(oracle):
    """a^(k) = lam^k u (an exponential): dt = eta / lam exactly."""
    rng = np.random.default_rng(6)
    for _ in range(10):
        lam = 10 ** rng.uniform(-3, 3)
        u = rng.normal(size=3)
        ladder = [lam ** k * u for k in range(6)]
        eta = rng.uniform(0.05, 1.0)
        assert oracle.dt_criterion(*ladder, eta) == pytest.approx(eta / lam, rel=1e-12)
        assert oracle.dt_initial(*ladder[:3], eta) == pytest.approx(eta / lam, rel=1e-12)


def test_criterion_time_rescaling(oracle):
    """t -> kappa t scales a^(k) by kappa^-k and dt by kappa."""
    rng = np.random.default_rng(7)
    ladder = [rng.normal(size=3) * 10 ** rng.uniform(-1, 1) for _ in range(6)]
    base = oracle.dt_criterion(*ladder, 0.4)
    for kappa in (0.01, 0.5, 3.0, 1e3):
        scaled = [q * kappa ** -k for k, q in enumerate(ladder)]
        assert oracle.dt_criterion(*scaled, 0.4) == pytest.approx(kappa * base, rel=1e-12)
        sc0 = oracle.dt_initial(*scaled[:3], 0.01)
        assert sc0 == pytest.approx(kappa * oracle.dt_initial(*ladder[:3], 0.01), rel=1e-12)


def test_criterion_degenerate(oracle):
    z = np.zeros(3)
    assert oracle.dt_criterion(z, z, z, z, z, z, 0.4) == math.inf


def test_quantize_properties(oracle):
    rng = np.random.default_rng(8)
    dt_min, dt_max = 2.0 ** -20, 2.0 ** -3
    for _ in range(2000):
        k_old = int(rng.integers(3, 21))
        dt_old = 2.0 ** -k_old
        t1 = dt_old * int(rng.integers(1, 1 << 12))
        dt_crit = 10 ** rng.uniform(-7, 0)
        dt, uf = oracle.dt_quantize(dt_crit, dt_old, t1, dt_min, dt_max)
        assert dt_min <= dt <= dt_max
        assert math.frexp(dt)[0] == 0.5                  # power of two
        assert math.fmod(t1, dt) == 0.0                  # commensurable
        assert dt <= 2 * dt_old                          # at most one doubling
        assert uf == (dt_crit < dt_min)
        if dt_crit < dt_old and dt_crit >= dt_min:
            assert dt <= dt_crit < 2 * dt                # 2^floor(log2 dt_crit)
        if dt > dt_old:
            assert dt_crit >= dt and math.fmod(t1, dt) == 0.0


def test_quantize_initial(oracle):
    assert oracle.dt_quantize_initial(0.3, 2.0 ** -20, 2.0 ** -3) == 0.125
    assert oracle.dt_quantize_initial(0.01, 2.0 ** -20, 2.0 ** -3) == 2.0 ** -7
    assert oracle.dt_quantize_initial(math.inf, 2.0 ** -20, 2.0 ** -3) == 0.125
    assert oracle.dt_quantize_initial(1e-9, 2.0 ** -20, 2.0 ** -3) == 2.0 ** -20


# ----------------------------------------------------------------- scheduler
def test_select_brute_force(oracle):
    rng = np.random.default_rng(9)
    m, x, v = ic.plummer(300, seed=2)
    sim = oracle.Sim(m, x, v, eps=1e-2)
    for _ in range(20):
        k = rng.integers(3, 12, sim.n)
        sim.dt[:] = 2.0 ** -k.astype(np.float64)
        sim.t[:] = sim.dt * rng.integers(0, 50, sim.n)
        tn, act = sim.select()
        ref_tn = np.min(sim.t + sim.dt)
        assert tn == ref_tn
        np.testing.assert_array_equal(act, np.nonzero(sim.t + sim.dt == ref_tn)[0])


# ------------------------------------------------------------------- Kepler
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


def _kepler_run(oracle, h, orbits=10):
    m = np.array([0.5, 0.5])
    r0, v0 = _kepler_state(0.0)
    x = np.stack([-0.5 * r0, 0.5 * r0]); v = np.stack([-0.5 * v0, 0.5 * v0])
    sim = oracle.Sim(m, x, v, eps=0.0, eta=0.4, dt_min=h, dt_max=h).init()
    t_end = math.floor(orbits * 2 * math.pi / h) * h
    sim.run(t_end)
    assert np.all(sim.t == t_end)
    r_ref, v_ref = _kepler_state(t_end)
    return (np.linalg.norm((sim.x[1] - sim.x[0]) - r_ref),
            np.linalg.norm((sim.v[1] - sim.v[0]) - v_ref))


def test_kepler_closed_form_and_order(oracle):
    """e = 0.5, eps = 0, 10 orbits with shared steps: close to Kepler's
    equation solution, and the global error falls ~2^6 per halving of dt."""
    e1, _ = _kepler_run(oracle, 2.0 ** -6)
    e2, _ = _kepler_run(oracle, 2.0 ** -7)
    assert e1 < 1e-5
    order = math.log2(e1 / e2)
    assert 5.0 < order < 7.0, order


# ------------------------------------------------- conservation and trajectory
def test_momentum_exact_with_shared_steps(oracle):
    m, x, v = ic.plummer(64, seed=3)
    h = 2.0 ** -9
    sim = oracle.Sim(m, x, v, eps=1e-2, dt_min=h, dt_max=h).init()
    _, _, P0, L0 = sim.energy(0.0)
    sim.run(16 * h)
    _, _, P1, L1 = sim.energy(16 * h)
    assert np.linalg.norm(P1 - P0) < 1e-15
    assert np.linalg.norm(L1 - L0) < 1e-12


def test_energy_block_steps_plummer(oracle):
    m, x, v = ic.plummer(128, seed=4)
    sim = oracle.Sim(m, x, v, eps=1e-2, eta=0.4).init()
    ek0, ep0, _, _ = sim.energy(0.0)
    sim.run(0.5)
    ek1, ep1, _, _ = sim.energy(0.5)
    e0, e1 = ek0 + ep0, ek1 + ep1
    assert np.all(sim.t == 0.5)
    assert abs(e1 - e0) / abs(e0) < 1e-7
    assert sim.underflows == 0
    # Henon units: E close to -1/4 for a Plummer sample
    assert -0.32 < e0 < -0.19


def test_block_run_deterministic(oracle):
    m, x, v = ic.plummer(64, seed=5)
    runs = []
    for _ in range(2):
        sim = oracle.Sim(m, x, v, eps=1e-2).init()
        sim.run(0.25)
        runs.append((sim.x.copy(), sim.dt.copy(), sim.block_steps))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]


def test_jerk_snap_crackle_vs_finite_differences(oracle):
    """Along an integrated trajectory (shared steps h) the stored jerk, snap
    and interpolated crackle match 5-point differences of the acceleration."""
    m, x, v = ic.plummer(16, seed=6)
    h = 2.0 ** -10
    sim = oracle.Sim(m, x, v, eps=5e-2, dt_min=h, dt_max=h).init()
    A, J, S, Cr = [], [], [], []
    for _ in range(9):
        A.append(sim.a.copy()); J.append(sim.j.copy()); S.append(sim.s.copy()); Cr.append(sim.c.copy())
        sim.step()
    A = np.array(A)
    for k in range(3, 6):
        fd_j = (-A[k + 2] + 8 * A[k + 1] - 8 * A[k - 1] + A[k - 2]) / (12 * h)
        fd_s = (-A[k + 2] + 16 * A[k + 1] - 30 * A[k] + 16 * A[k - 1] - A[k - 2]) / (12 * h * h)
        fd_c = (A[k + 2] - 2 * A[k + 1] + 2 * A[k - 1] - A[k - 2]) / (2 * h ** 3)
        for got, fd, tol in ((J[k], fd_j, 1e-8), (S[k], fd_s, 1e-5), (Cr[k], fd_c, 1e-3)):
            err = np.linalg.norm(got - fd, axis=1) / np.linalg.norm(fd, axis=1)
            assert err.max() < tol, (tol, err.max())


def _kepler_block_energy(oracle, eta, order=6, orbits=10):
    m = np.array([0.5, 0.5])
    r0, v0 = _kepler_state(0.0)
    x = np.stack([-0.5 * r0, 0.5 * r0]); v = np.stack([-0.5 * v0, 0.5 * v0])
    sim = oracle.Sim(m, x, v, eps=0.0, eta=eta, order=order).init()
    t_end = math.floor(orbits * 2 * math.pi / 0.125) * 0.125
    e0 = sum(sim.energy(0.0)[:2])
    sim.run(t_end)
    assert np.all(sim.t == t_end)
    return abs(sum(sim.energy(t_end)[:2]) - e0) / abs(e0), sim.block_steps


def test_kepler_block_steps_energy_and_eta_scaling(oracle):
    """e = 0.5, eps = 0, block steps on the criterion (eta 0.4 then 0.2):
    energy error below 1e-6 per orbit, and falling by more than 2^5 when eta
    halves (the step is proportional to eta; 6th order)."""
    e1, n1 = _kepler_block_energy(oracle, 0.4)
    e2, n2 = _kepler_block_energy(oracle, 0.2)
    assert e1 / 10 < 1e-6, e1
    assert e1 / e2 > 32.0, (e1, e2)
    assert 1.5 < n2 / n1 < 2.5, (n1, n2)


def test_kepler4_block_steps_eta_scaling(oracle):
    """The 4th-order scheme's Aarseth step is proportional to sqrt(eta): halving
    eta shortens steps by sqrt(2) and cuts the energy error by about 4."""
    e1, n1 = _kepler_block_energy(oracle, 0.02, order=4)
    e2, n2 = _kepler_block_energy(oracle, 0.01, order=4)
    assert e1 / 10 < 1e-5, e1
    assert e1 / e2 > 2.5, (e1, e2)
    assert 1.2 < n2 / n1 < 1.7, (n1, n2)
