"""Pins of the oracle's pairwise evaluation (acceleration, jerk, snap, potential).

The evaluation is the paper's O(N^2) kernel (Sec. 4); its formulas are the
6th-order Hermite scheme's (Nitadori & Makino 2008).  These tests check the
oracle against facts that do not depend on those formulas being retyped:

* Taylor-jet arithmetic: along quadratic trajectories x_k(t) = x + v t + a t^2/2
  the exact force F(t) is expanded as a power series with a generic series
  power recurrence; acceleration, jerk and snap must equal F(0), F'(0), F''(0).
  (At 40 digits with mpmath for tiny N, in float64 for larger N.)
* the two-body closed form of the acceleration and potential;
* Newton's third law for all three derivatives;
* permutation invariance.
"""
import math

import numpy as np
import pytest


# --------------------------------------------------------------------------- jets
class Jet:
    """Truncated power series c0 + c1 t + ... + cK t^K over a scalar field."""

    def __init__(self, c):
        self.c = list(c)

    @property
    def K(self):
        return len(self.c) - 1

    def __add__(self, o):
        if not isinstance(o, Jet):
            o = Jet([o] + [0 * self.c[0]] * self.K)
        return Jet([a + b for a, b in zip(self.c, o.c)])

    __radd__ = __add__

    def __sub__(self, o):
        if not isinstance(o, Jet):
            o = Jet([o] + [0 * self.c[0]] * self.K)
        return Jet([a - b for a, b in zip(self.c, o.c)])

    def __mul__(self, o):
        if not isinstance(o, Jet):
            return Jet([a * o for a in self.c])
        K = self.K
        out = []
        for k in range(K + 1):
            acc = 0 * self.c[0]
            for i in range(k + 1):
                acc = acc + self.c[i] * o.c[k - i]
            out.append(acc)
        return Jet(out)

    __rmul__ = __mul__

    def power(self, p):
        """s^p by the recurrence k s0 f_k = sum_{i=1..k} (p i - k + i) s_i f_{k-i}."""
        s = self.c
        f = [s[0] ** p]
        for k in range(1, self.K + 1):
            acc = 0 * s[0]
            for i in range(1, k + 1):
                acc = acc + (p * i - k + i) * s[i] * f[k - i]
            f.append(acc / (k * s[0]))
        return Jet(f)


def jet_force(m, x, v, a, eps2, i, K=2, conv=float):
    """Force on particle i along x_k(t) = x_k + v_k t + a_k t^2 / 2 as jets.

    Returns (F, pot) with F a list of three Jets (Taylor coefficients)."""
    n = len(m)
    half = conv(1) / conv(2)
    pos = [[Jet([conv(x[k][d]), conv(v[k][d]), conv(a[k][d]) * half] + [conv(0)] * (K - 2))
            for d in range(3)] for k in range(n)]
    F = [Jet([conv(0)] * (K + 1)) for _ in range(3)]
    P = Jet([conv(0)] * (K + 1))
    for j in range(n):
        if j == i:
            continue
        r = [pos[j][d] - pos[i][d] for d in range(3)]
        s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + conv(eps2)
        w = s2.power(conv(-3) / conv(2))
        for d in range(3):
            F[d] = F[d] + (r[d] * w) * conv(m[j])
        P = P - s2.power(conv(-1) / conv(2)) * conv(m[j])
    return F, P


def _system(rng, n):
    m = rng.uniform(0.5, 2.0, n) / n
    x = rng.normal(size=(n, 3))
    v = rng.normal(size=(n, 3)) * 0.5
    a = rng.normal(size=(n, 3)) * 0.3
    return m, x, v, a


@pytest.mark.parametrize("eps", [0.0, 1e-2, 0.3])
def test_jets_mpmath_tiny(oracle, eps):
    """Brute force at 40 digits, N = 7: acc/jerk/snap/pot = F, F', F'' (mp)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(11)
    n = 7
    m, x, v, a = _system(rng, n)
    acc, jrk, snp, pot = oracle.force(m, x, v, a, eps)
    for i in range(n):
        F, P = jet_force(m, x, v, a, eps * eps, i, K=2, conv=mpmath.mpf)
        ref_a = np.array([float(F[d].c[0]) for d in range(3)])
        ref_j = np.array([float(F[d].c[1]) for d in range(3)])
        ref_s = np.array([float(2 * F[d].c[2]) for d in range(3)])
        for got, ref in ((acc[i], ref_a), (jrk[i], ref_j), (snp[i], ref_s)):
            assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref) + 1e-300
        assert abs(pot[i] - float(P.c[0])) <= 1e-14 * abs(float(P.c[0]))


def test_jets_float64_n64(oracle):
    """Float64 jets, N = 64, all particles active: same identity, rtol 1e-11."""
    rng = np.random.default_rng(5)
    n = 64
    m, x, v, a = _system(rng, n)
    eps = 1e-3
    acc, jrk, snp, pot = oracle.force(m, x, v, a, eps)
    for i in range(0, n, 7):
        F, P = jet_force(m, x, v, a, eps * eps, i, K=2)
        ref_a = np.array([F[d].c[0] for d in range(3)])
        ref_j = np.array([F[d].c[1] for d in range(3)])
        ref_s = np.array([2 * F[d].c[2] for d in range(3)])
        assert np.linalg.norm(acc[i] - ref_a) <= 1e-11 * np.linalg.norm(ref_a)
        assert np.linalg.norm(jrk[i] - ref_j) <= 1e-11 * np.linalg.norm(ref_j)
        assert np.linalg.norm(snp[i] - ref_s) <= 1e-11 * np.linalg.norm(ref_s)
        assert abs(pot[i] - P.c[0]) <= 1e-12 * abs(P.c[0])


def test_subset_active_matches_full(oracle):
    rng = np.random.default_rng(2)
    m, x, v, a = _system(rng, 50)
    full = oracle.force(m, x, v, a, 1e-2)
    act = np.array([3, 17, 49, 0])
    sub = oracle.force(m, x, v, a, 1e-2, active=act)
    for q_full, q_sub in zip(full, sub):
        np.testing.assert_array_equal(q_full[act], q_sub)


def test_two_body_closed_form(oracle):
    """a_1 = m_2 r / (r^2 + eps^2)^{3/2}, pot_1 = -m_2 / sqrt(r^2 + eps^2)."""
    m = np.array([0.3, 0.7])
    x = np.array([[0.1, -0.2, 0.3], [1.1, 0.4, -0.5]])
    v = np.zeros((2, 3)); a = np.zeros((2, 3))
    for eps in (0.0, 0.05):
        acc, jrk, snp, pot = oracle.force(m, x, v, a, eps)
        r = x[1] - x[0]
        s2 = r @ r + eps * eps
        np.testing.assert_allclose(acc[0], m[1] * r / s2 ** 1.5, rtol=1e-15, atol=0)
        np.testing.assert_allclose(acc[1], -m[0] * r / s2 ** 1.5, rtol=1e-15, atol=0)
        np.testing.assert_allclose(pot, [-m[1] / math.sqrt(s2), -m[0] / math.sqrt(s2)],
                                   rtol=1e-15)
        assert np.all(jrk == 0) and np.all(snp == 0)


def test_newton_third_law(oracle):
    """sum_i m_i (a_i, j_i, s_i) = 0 up to round-off x sum |terms|."""
    rng = np.random.default_rng(3)
    n = 200
    m, x, v, a = _system(rng, n)
    acc, jrk, snp, pot = oracle.force(m, x, v, a, 1e-2)
    for q in (acc, jrk, snp):
        tot = (m[:, None] * q).sum(axis=0)
        scale = (m[:, None] * np.abs(q)).sum()
        assert np.linalg.norm(tot) <= 1e-13 * scale


def test_permutation_invariance(oracle):
    rng = np.random.default_rng(4)
    n = 40
    m, x, v, a = _system(rng, n)
    perm = rng.permutation(n)
    ref = oracle.force(m, x, v, a, 1e-2)
    got = oracle.force(m[perm], x[perm], v[perm], a[perm], 1e-2)
    for r, g in zip(ref, got):
        np.testing.assert_allclose(g, r[perm], rtol=1e-12, atol=1e-14 * np.abs(r).max())


def test_self_excluded_by_index(oracle):
    """eps = 0 with every particle active: no division by zero from i == j."""
    rng = np.random.default_rng(6)
    m, x, v, a = _system(rng, 10)
    out = oracle.force(m, x, v, a, 0.0)
    assert all(np.all(np.isfinite(q)) for q in out)


def test_single_particle_and_empty(oracle):
    m = np.array([1.0]); x = np.zeros((1, 3))
    acc, jrk, snp, pot = oracle.force(m, x, x, x, 0.1)
    assert np.all(acc == 0) and pot[0] == 0
    acc, jrk, snp, pot = oracle.force(m, x, x, x, 0.1, active=np.zeros(0, dtype=np.int64))
    assert acc.shape == (0, 3)
