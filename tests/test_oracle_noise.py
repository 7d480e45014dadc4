"""The oracle's evaluation-perturbation hook, and what it shows about the
accuracy the time-step criteria need from the pair arithmetic.

The paper (Sec. 2) states that the Hermite 6th-order code needs double
precision (or the EX pair-of-singles type) in the inter-particle distances and
accelerations.  Perturbing the oracle's own evaluations term by term makes
that quantitative: the 6th-order scheme's step criterion divides differences
of the accelerations at both step ends by up to h^5 (the quintic
interpolation of a^(3), a^(4), a^(5)), so relative acceleration errors of
1e-6 — the size single-precision force arithmetic leaves (unit roundoff
2^-24 ~ 6e-8 per operation) — collapse the steps to the minimum, while
jerk and snap errors of 1e-5 change nothing.  The 4th-order scheme's
criterion (cubic interpolation, h^3) tolerates 1e-6.
"""
import numpy as np
import pytest

from paper_1812_00367_gb300 import ic

N, EPS, T_END = 1024, 1e-4, 1.0 / 64


@pytest.fixture(scope="module")
def plummer1024():
    return ic.plummer(N, seed=1)


def test_noise_off_changes_nothing(oracle, plummer1024):
    m, x, v = plummer1024
    a = oracle.Sim(m, x, v, eps=EPS).init()
    a.run(T_END)
    b = oracle.Sim(m, x, v, eps=EPS).set_noise(0.0, 0.0, 0.0, 7).init()
    b.run(T_END)
    for f in ("x", "v", "a", "j", "s", "c", "t", "dt", "pot"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f), err_msg=f)


@pytest.mark.parametrize("term", ["a", "j"])
def test_noise_size_per_component(oracle, plummer1024, term):
    """After the start-up, a and jerk are the second pass's sums (they do not
    depend on the first pass), so each component is the unperturbed one times
    (1 + e u) with |u| <= 1, and the draws fill the interval."""
    m, x, v = plummer1024
    e = 1e-6
    ref = oracle.Sim(m, x, v, eps=EPS).init()
    kw = {"a": (e, 0.0, 0.0), "j": (0.0, e, 0.0)}[term]
    got = oracle.Sim(m, x, v, eps=EPS).set_noise(*kw, 3).init()
    r = getattr(got, term) / getattr(ref, term) - 1.0
    assert np.abs(r).max() <= e * (1 + 1e-9)
    assert np.abs(r).max() >= 0.99 * e and abs(r.mean()) < 0.05 * e
    other = "j" if term == "a" else "a"
    np.testing.assert_array_equal(getattr(got, other), getattr(ref, other))


def test_noise_is_reproducible_and_seeded(oracle, plummer1024):
    m, x, v = plummer1024
    a = oracle.Sim(m, x, v, eps=EPS).set_noise(1e-9, 1e-9, 1e-9, 5).init()
    b = oracle.Sim(m, x, v, eps=EPS).set_noise(1e-9, 1e-9, 1e-9, 5).init()
    c = oracle.Sim(m, x, v, eps=EPS).set_noise(1e-9, 1e-9, 1e-9, 6).init()
    np.testing.assert_array_equal(a.a, b.a)
    assert np.any(a.a != c.a)


def _steps(oracle, m, x, v, order, noise, cap=-1):
    eta = 0.4 if order == 6 else 0.02
    s = oracle.Sim(m, x, v, eps=EPS, eta=eta, order=order).set_noise(*noise, 1).init()
    k = s.run(T_END, cap)
    return k, s.underflows


def test_sixth_order_criterion_needs_accurate_accelerations(oracle, plummer1024):
    m, x, v = plummer1024
    base, uf0 = _steps(oracle, m, x, v, 6, (0.0, 0.0, 0.0))
    assert uf0 == 0
    cap = 20 * base
    # single-precision-sized acceleration errors: the steps collapse
    k, uf = _steps(oracle, m, x, v, 6, (1e-6, 0.0, 0.0), cap)
    assert k >= 10 * base and uf > 0, (k, uf, base)
    # the same and larger errors in jerk or snap alone leave them as they were
    for noise in ((0.0, 1e-5, 0.0), (0.0, 0.0, 1e-5)):
        k, uf = _steps(oracle, m, x, v, 6, noise, cap)
        assert k <= 1.1 * base + 1 and uf == 0, (noise, k, base)
    # errors at the double-precision scale change nothing
    k, uf = _steps(oracle, m, x, v, 6, (1e-12, 1e-12, 1e-12), cap)
    assert k == base and uf == 0


def test_fourth_order_criterion_tolerates_single_precision_accelerations(oracle, plummer1024):
    m, x, v = plummer1024
    base, _ = _steps(oracle, m, x, v, 4, (0.0, 0.0, 0.0))
    k, uf = _steps(oracle, m, x, v, 4, (1e-6, 1e-6, 0.0), 20 * base)
    assert k <= 1.1 * base + 1 and uf == 0, (k, base)
    # far larger errors do collapse it too
    k, _ = _steps(oracle, m, x, v, 4, (1e-4, 0.0, 0.0), 20 * base)
    assert k >= 5 * base, (k, base)


def test_trajectory_response_grows_with_the_perturbation(oracle, trajectory_envelope, plummer1024):
    """The envelope used as the trajectory tolerance of the GPU shared-step
    tests: larger evaluation perturbations move the trajectory further, and
    well-conditioned particles move by about the perturbation's size times
    the step's small factors."""
    m, x, v = plummer1024
    h = 1.0 / 256
    _, _, ex1, ev1 = trajectory_envelope(m, x, v, EPS, h, 16, 1e-12)
    _, _, ex2, ev2 = trajectory_envelope(m, x, v, EPS, h, 16, 1e-10)
    assert np.median(ex2) > 30 * np.median(ex1) and np.median(ev2) > 30 * np.median(ev1)
    assert np.median(ex1) < 1e-14 and ex1.max() < 1e-11
