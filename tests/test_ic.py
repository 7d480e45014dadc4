"""Pins of the seeded synthetic input generators (no method arithmetic)."""
import math

import numpy as np
import pytest

from paper_1812_00367_gb300 import ic

scipy_stats = pytest.importorskip("scipy.stats")


def _potential_energy(m, x):
    """Unsoftened W = -sum_{i<j} m_i m_j / r_ij (direct, numpy)."""
    W = 0.0
    for i in range(len(m) - 1):
        d = np.linalg.norm(x[i + 1:] - x[i], axis=1)
        W -= m[i] * np.sum(m[i + 1:] / d)
    return W


def test_plummer_henon_units_and_virial():
    m, x, v = ic.plummer(3000, seed=1)
    assert m.sum() == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose((m[:, None] * x).sum(0), 0, atol=1e-14)
    np.testing.assert_allclose((m[:, None] * v).sum(0), 0, atol=1e-14)
    K = 0.5 * np.sum(m * np.sum(v * v, axis=1))
    W = _potential_energy(m, x)
    assert abs(2 * K / abs(W) - 1.0) < 4 * 3 / math.sqrt(len(m))
    assert K + W == pytest.approx(-0.25, abs=0.03)


def test_plummer_mass_profile_ks():
    m, x, v = ic.plummer(20000, seed=2)
    a = ic.HENON_PLUMMER_SCALE
    r = np.linalg.norm(x, axis=1) / a
    cut = 0.999
    cdf = lambda rr: (rr ** 3 / (1 + rr * rr) ** 1.5) / cut
    # centre-of-mass shift is O(1/sqrt(N)) and does not spoil the KS test
    assert scipy_stats.kstest(r, cdf).pvalue > 1e-3


def test_plummer_seeded_and_distinct():
    a = ic.plummer(100, seed=7)
    b = ic.plummer(100, seed=7)
    c = ic.plummer(100, seed=8)
    for p, q in zip(a, b):
        np.testing.assert_array_equal(p, q)
    assert not np.array_equal(a[1], c[1])


def test_kroupa_masses():
    m = ic.kroupa_masses(200000, seed=3)
    assert m.sum() == pytest.approx(1.0, rel=1e-12)
    ratio = m.max() / m.min()
    assert 100 < ratio <= 1000 * (1 + 1e-12)
    # slope of the upper segment: log-log histogram
    raw = m / m.min() * 0.1
    hi = raw[raw > 1.0]
    bins = np.logspace(0, 1.8, 10)
    h, e = np.histogram(hi, bins=bins)
    centres = np.sqrt(e[1:] * e[:-1])
    dens = h / np.diff(e)
    slope = np.polyfit(np.log(centres), np.log(dens), 1)[0]
    assert slope == pytest.approx(-2.3, abs=0.15)


def test_hernquist_profile_and_virial():
    m, x, v = ic.hernquist(20000, seed=4)
    r = np.linalg.norm(x, axis=1)
    cut = 0.99
    cdf = lambda rr: (rr * rr / (rr + 1) ** 2) / cut
    assert scipy_stats.kstest(r, cdf).pvalue > 1e-3
    sub = slice(0, 3000)
    ms = m[sub] * (len(m) / 3000)
    K = 0.5 * np.sum(ms * np.sum(v[sub] ** 2, axis=1))
    W = _potential_energy(ms, x[sub])
    assert abs(2 * K / abs(W) - 1.0) < 0.15


def test_hernquist_df_positive_and_small_q():
    E = -np.linspace(1e-4, 0.999, 200)
    f = ic.hernquist_df(E)
    assert np.all(f > 0)
    # weakly bound limit: f ~ |E|^{5/2}
    E2 = np.array([-1e-3, -2e-3])
    f2 = ic.hernquist_df(E2)
    assert math.log(f2[1] / f2[0]) / math.log(2) == pytest.approx(2.5, abs=0.05)


def test_parabolic_pair_energy_zero():
    dx1, dv1, dx2, dv2 = ic.parabolic_pair(1.0, 1.0, 20.0, 1.0)
    r = dx2 - dx1
    vrel = dv2 - dv1
    eps_orb = 0.5 * vrel @ vrel - 2.0 / np.linalg.norm(r)
    assert abs(eps_orb) < 1e-14
    assert np.linalg.norm(r) == pytest.approx(20.0)
    h = np.linalg.norm(np.cross(r, vrel))
    assert h * h / (2 * 2.0) == pytest.approx(1.0)    # pericentre
    assert r @ vrel < 0                                # approaching
    np.testing.assert_allclose(dx1 + dx2, 0, atol=1e-14)


def test_batch_sizes():
    b = ic.plummer_batch(64, seed=5)
    s = b.sizes
    assert len(s) == 64 and s.min() >= 256 and s.max() <= 16384
    assert b.offsets[-1] == len(b.m)
    for k in range(3):
        sl = slice(b.offsets[k], b.offsets[k + 1])
        assert b.m[sl].sum() == pytest.approx(1.0)
