"""GPU parity of the 4th-order Hermite variant (Makino & Aarseth 1992)
against the oracle's 4th-order scheme, through the C ABI.

Same tolerances as the 6th-order path (per particle ||q_gpu - q_ref|| /
||q_ref|| for a and jerk, |d pot / pot|): FP64 1e-12, EX 1e-10, FP32 2e-5.
"""
import math

import numpy as np
import pytest

from paper_1812_00367_gb300 import ic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ex": 1e-10, "fp32": 2e-5}
ETA4 = 0.02


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00367_gb300 import build as nbbuild
    nbbuild.build()
    from paper_1812_00367_gb300 import nb as nbmod
    nbmod.load()
    return nbmod


def rel_rows(got, ref):
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.linalg.norm(ref, axis=-1)
    return np.where(den > 0, num / np.where(den > 0, den, 1), num)


def _sim4(nb, st, eps, precision="fp64", **kw):
    n = len(st["m"])
    sim = nb.Simulation(st["m"], st["x"], st["v"], eps=eps, eta=ETA4, precision=precision,
                        keep_state=True, order=4, **kw)
    full = {"a": np.zeros((n, 3)), "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
            "c": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, 2.0 ** -6),
            "pot": np.zeros(n)}
    full.update(st)
    sim.set_state_numpy(full)
    return sim


@pytest.mark.parametrize("precision", ["fp64", "ex", "fp32"])
@pytest.mark.parametrize("n", [3, 65, 1000, 4097])
def test_evaluate4_parity(nb, oracle, precision, n):
    """a, jerk, pot of the 4th-order pair terms; the stored accelerations are
    not read (random here) and the snap rows are exactly zero."""
    eps = 1e-4
    m, x, v = ic.plummer(n, seed=100 + n)
    rng = np.random.default_rng(n)
    sim = _sim4(nb, {"m": m, "x": x, "v": v, "a": rng.normal(size=(n, 3))}, eps, precision)
    sim.predict(0.0, out=False)
    for A in sorted({1, min(100, n), n}):
        act = np.sort(rng.choice(n, size=A, replace=False)).astype(np.int32)
        got = sim.evaluate(torch.as_tensor(act, device="cuda")).cpu().numpy()
        acc, jrk, _, pot = oracle.force(m, x, v, np.zeros_like(x), eps, active=act)
        assert rel_rows(got[0:3].T, acc).max() <= TOL[precision]
        assert rel_rows(got[3:6].T, jrk).max() <= TOL[precision]
        assert (np.abs(got[9] - pot) / np.abs(pot)).max() <= TOL[precision]
        assert np.all(got[6:9] == 0.0)
    sim.close()


def test_predict4_parity(nb, oracle):
    rng = np.random.default_rng(3)
    n = 777
    m = rng.uniform(0.5, 1.5, n) / n
    f = {k: rng.normal(size=(n, 3)) * s for k, s in zip("xvajsc", (1, 1, 1, 3, 10, 30))}
    dt = 2.0 ** -rng.integers(3, 12, n).astype(float)
    t = dt * rng.integers(0, 4, n)
    sim = _sim4(nb, {"m": m, **f, "t": t, "dt": dt}, 1e-2)
    tn = float(t.max() + 2.0 ** -3)
    out = sim.predict(tn).cpu().numpy()
    xp, vp = oracle.predict4(f["x"], f["v"], f["a"], f["j"], t, tn)
    np.testing.assert_allclose(out[0:3].T, xp, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(out[3:6].T, vp, rtol=1e-13, atol=1e-13)
    d = (tn - t)[:, None]
    np.testing.assert_allclose(out[6:9].T, f["a"] + f["j"] * d, rtol=1e-13, atol=1e-13)
    sim.close()


def test_correct4_parity(nb, oracle):
    """The oracle's evaluation feeds the GPU corrector: x, v, the cubic's
    derivatives (s, c), new steps and times agree with the oracle's step."""
    n, eps = 512, 1e-2
    m, x, v = ic.plummer(n, seed=15)
    ref = oracle.Sim(m, x, v, eps=eps, eta=ETA4, order=4).init()
    ref.run(2.0 ** -5)
    fields = ("m", "x", "v", "a", "j", "s", "c", "t", "dt", "pot")
    pre = {f: getattr(ref, f).copy() for f in fields}
    tn, act = ref.select()
    xp, vp = oracle.predict4(ref.x, ref.v, ref.a, ref.j, ref.t, tn)
    acc, jrk, _, pot = oracle.force(m, xp, vp, np.zeros_like(xp), eps, active=act)
    ajs = np.concatenate([acc.T, jrk.T, np.zeros((3, len(act))), pot[None, :]], axis=0)
    ref.step()
    sim = _sim4(nb, pre, eps)
    sim.correct(torch.as_tensor(act.astype(np.int32), device="cuda"), tn,
                torch.as_tensor(ajs, device="cuda"))
    sim.sync()
    got = sim.state_numpy()
    np.testing.assert_allclose(got["x"][act], ref.x[act], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(got["v"][act], ref.v[act], rtol=1e-13, atol=1e-14)
    for f in ("a", "j", "pot"):
        np.testing.assert_array_equal(got[f][act], getattr(ref, f)[act])
    assert rel_rows(got["s"][act], ref.s[act]).max() < 1e-9
    assert rel_rows(got["c"][act], ref.c[act]).max() < 1e-8
    np.testing.assert_array_equal(got["t"], ref.t)
    mism = np.nonzero(got["dt"] != ref.dt)[0]
    assert len(mism) <= max(1, len(act) // 1000), mism
    untouched = np.setdiff1d(np.arange(n), act)
    np.testing.assert_array_equal(got["x"][untouched], pre["x"][untouched])
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "ex", "fp32"])
def test_init4_parity(nb, oracle, precision):
    """One start-up pass: a, jerk, pot; s = c = 0; dt0 = eta_init |a|/|j|."""
    n, eps = 1024, 1e-4
    m, x, v = ic.plummer(n, seed=2)
    ref = oracle.Sim(m, x, v, eps=eps, eta=ETA4, order=4).init()
    sim = nb.Simulation(m, x, v, eps=eps, eta=ETA4, precision=precision, order=4)
    got = sim.state_numpy()
    tol = TOL[precision]
    for f in ("a", "j"):
        assert rel_rows(got[f], getattr(ref, f)).max() < tol, f
    assert (np.abs(got["pot"] - ref.pot) / np.abs(ref.pot)).max() < tol
    assert np.all(got["s"] == 0) and np.all(got["c"] == 0) and np.all(got["t"] == 0)
    assert np.mean(got["dt"] == ref.dt) > 0.99
    sim.close()


def test_shared_steps4_plummer_1024(nb, oracle):
    n, eps, h = 1024, 1e-4, 1.0 / 512
    m, x, v = ic.plummer(n, seed=4)
    ref = oracle.Sim(m, x, v, eps=eps, eta=ETA4, dt_min=h, dt_max=h, order=4).init()
    sim = nb.Simulation(m, x, v, eps=eps, eta=ETA4, dt_min=h, dt_max=h, order=4)
    for _ in range(16):
        _, na = sim.step()
        assert na == n
    ref.run(16 * h)
    got = sim.state_numpy()
    assert np.all(got["t"] == 16 * h)
    ex = rel_rows(got["x"], ref.x)
    ev = rel_rows(got["v"], ref.v)
    assert np.median(ex) < 1e-12 and ex.max() < 1e-8, (np.median(ex), ex.max())
    assert np.median(ev) < 1e-12 and ev.max() < 1e-7, (np.median(ev), ev.max())
    sim.close()


def test_block_steps4_energy_and_determinism(nb, oracle):
    n, eps, t_end = 512, 1e-2, 0.125
    m, x, v = ic.plummer(n, seed=17)
    ref = oracle.Sim(m, x, v, eps=eps, eta=ETA4, order=4).init()
    e0 = sum(ref.energy(0.0)[:2])
    ref.run(t_end)
    e1 = sum(ref.energy(t_end)[:2])
    states = []
    for _ in range(2):
        sim = nb.Simulation(m, x, v, eps=eps, eta=ETA4, order=4)
        g0 = sum(sim.energy(0.0)[:2])
        steps, inter = sim.run(t_end)
        g1 = sum(sim.energy(t_end)[:2])
        st = sim.state_numpy()
        states.append(st)
        assert np.all(st["t"] == t_end)
        assert abs(g1 - g0) / abs(g0) < 1e-7
        assert steps == pytest.approx(ref.block_steps, rel=0.2)
        assert inter == pytest.approx(ref.interactions - n * (n - 1), rel=0.2)
        sim.close()
    for f in ("x", "v", "dt"):
        np.testing.assert_array_equal(states[0][f], states[1][f])
    assert abs(e1 - e0) / abs(e0) < 1e-7


def _kepler(t, e=0.5):
    M = t
    E = M
    for _ in range(100):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    den = 1 - e * math.cos(E)
    r = np.array([math.cos(E) - e, math.sqrt(1 - e * e) * math.sin(E), 0.0])
    v = np.array([-math.sin(E) / den, math.sqrt(1 - e * e) * math.cos(E) / den, 0.0])
    return r, v


def test_kepler4_order_on_gpu(nb):
    """Two bodies (total mass 1, a = 1, e = 0.5), eps = 0, shared steps: the
    GPU path alone follows Kepler's equation with global error ~h^4."""
    errs = []
    for h in (2.0 ** -7, 2.0 ** -8):
        r0, v0 = _kepler(0.0)
        m = np.array([0.5, 0.5])
        x = np.stack([-0.5 * r0, 0.5 * r0]); v = np.stack([-0.5 * v0, 0.5 * v0])
        sim = nb.Simulation(m, x, v, eps=0.0, eta=ETA4, dt_min=h, dt_max=h, order=4)
        t_end = math.floor(4 * 2 * math.pi / h) * h
        sim.run(t_end)
        st = sim.state_numpy()
        assert np.all(st["t"] == t_end)
        errs.append(np.linalg.norm((st["x"][1] - st["x"][0]) - _kepler(t_end)[0]))
        sim.close()
    assert errs[0] < 1e-3
    assert 3.5 < math.log2(errs[0] / errs[1]) < 4.6, errs
