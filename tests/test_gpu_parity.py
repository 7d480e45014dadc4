"""GPU parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Tolerances (per particle, ||q_gpu - q_ref|| / ||q_ref|| for q in a, jerk,
snap; |d pot / pot|): FP64 1e-12, EX 1e-10, FP32 2e-5.
"""
import math

import numpy as np
import pytest

from paper_1812_00367_gb300 import ic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ex": 1e-10, "fp32": 2e-5}


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


def _plummer_state(oracle, n, seed, eps):
    """Plummer positions/velocities with their true accelerations as the 'a'
    field (realistic a_j - a_i for the snap terms)."""
    m, x, v = ic.plummer(n, seed=seed)
    a = oracle.force(m, x, v, np.zeros_like(x), eps)[0] if n > 1 else np.zeros((n, 3))
    return m, x, v, a


def _sim_with_state(nb, m, x, v, a, eps, precision, offsets=None, t=None, dt=None):
    n = len(m)
    sim = nb.Simulation(m, x, v, eps=eps, precision=precision, offsets=offsets, keep_state=True)
    st = {"m": m, "x": x, "v": v, "a": a, "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
          "c": np.zeros((n, 3)), "t": np.zeros(n) if t is None else t,
          "dt": np.full(n, 2.0 ** -6) if dt is None else dt, "pot": np.zeros(n)}
    sim.set_state_numpy(st)
    return sim


def _check_eval(out, ref, tol, label):
    acc, jrk, snp, pot = ref
    got = out.cpu().numpy()
    errs = {"a": rel_rows(got[0:3].T, acc), "j": rel_rows(got[3:6].T, jrk),
            "s": rel_rows(got[6:9].T, snp),
            "pot": np.abs(got[9] - pot) / np.maximum(np.abs(pot), 1e-300)}
    for k, e in errs.items():
        assert e.max() <= tol, f"{label} {k}: max rel err {e.max():.3e} > {tol:.1e}"
    return {k: float(e.max()) for k, e in errs.items()}


# ------------------------------------------------------------------ probes
def test_fma_probes(nb):
    f64, _ = nb.nb_probe_fma_peak(nb.NB_FP64, 2048)
    f32, _ = nb.nb_probe_fma_peak(nb.NB_FP32, 8192)
    print(f"\nFP64 FMA peak {f64 / 1e12:.3f} TFLOP/s, FP32 {f32 / 1e12:.2f} TFLOP/s")
    assert f64 > 1e11 and f32 > 1e12


# --------------------------------------------------------------- predictor
def test_predict_parity(nb, oracle):
    rng = np.random.default_rng(1)
    n = 777
    m = rng.uniform(0.5, 1.5, n) / n
    f = {k: rng.normal(size=(n, 3)) * s for k, s in zip("xvajsc", (1, 1, 1, 3, 10, 30))}
    dt = 2.0 ** -rng.integers(3, 12, n).astype(float)
    t = dt * rng.integers(0, 4, n)
    sim = _sim_with_state(nb, m, f["x"], f["v"], f["a"], 1e-2, "fp64", t=t, dt=dt)
    st = {"m": m, **f, "t": t, "dt": dt, "pot": np.zeros(n)}
    sim.set_state_numpy(st)
    tn = float(t.max() + 2.0 ** -3)
    out = sim.predict(tn).cpu().numpy()
    xp, vp, ap = oracle.predict(f["x"], f["v"], f["a"], f["j"], f["s"], f["c"], t, tn)
    np.testing.assert_allclose(out[0:3].T, xp, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(out[3:6].T, vp, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(out[6:9].T, ap, rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(out[9], m)
    sim.close()


# -------------------------------------------------------------- evaluation
@pytest.mark.parametrize("precision", ["fp64", "ex", "fp32"])
@pytest.mark.parametrize("n", [2, 3, 63, 64, 65, 1000, 4097])
def test_evaluate_parity(nb, oracle, precision, n):
    eps = 1e-4
    m, x, v, a = _plummer_state(oracle, n, seed=n, eps=eps)
    sim = _sim_with_state(nb, m, x, v, a, eps, precision)
    sim.predict(0.0, out=False)
    rng = np.random.default_rng(n)
    for A in sorted({1, min(5, n), min(100, n), n}):
        act = np.sort(rng.choice(n, size=A, replace=False)).astype(np.int32)
        out = sim.evaluate(torch.as_tensor(act, device="cuda"))
        ref = oracle.force(m, x, v, a, eps, active=act)
        _check_eval(out, ref, TOL[precision], f"{precision} n={n} A={A}")
    sim.sync()
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "ex", "fp32"])
@pytest.mark.parametrize("n", [8192, 10007])
def test_evaluate_streamk_parity(nb, oracle, precision, n):
    """Large one-cluster evaluations run as stream-K ranges (each CTA an equal
    share of i-tile x j-tile units, pieces summed in CTA order): oracle parity,
    agreement with the split-item plan to rounding, bit-for-bit repeats."""
    eps = 1e-4
    m, x, v, a = _plummer_state(oracle, n, seed=n, eps=eps)
    rng = np.random.default_rng(n)
    acts = [np.arange(n, dtype=np.int32),
            np.sort(rng.choice(n, size=n - 37, replace=False)).astype(np.int32)]
    got = {}
    for sk in (True, False):
        sim = nb.Simulation(m, x, v, eps=eps, precision=precision, keep_state=True, streamk=sk)
        st = {"m": m, "x": x, "v": v, "a": a, "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
              "c": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, 2.0 ** -6),
              "pot": np.zeros(n)}
        sim.set_state_numpy(st)
        sim.predict(0.0, out=False)
        for k, act in enumerate(acts):
            at = torch.as_tensor(act, device="cuda")
            o1 = sim.evaluate(at).cpu().numpy()
            o2 = sim.evaluate(at).cpu().numpy()
            np.testing.assert_array_equal(o1, o2)
            got[(sk, k)] = o1
            if sk and k == 1:
                _check_eval(torch.as_tensor(o1), oracle.force(m, x, v, a, eps, active=act),
                            TOL[precision], f"stream-K {precision} n={n}")
        sim.close()
    for k in range(2):
        e = rel_rows(got[(True, k)][0:3].T, got[(False, k)][0:3].T)
        assert e.max() <= TOL[precision], e.max()


def test_evaluate_single_particle(nb, oracle):
    m = np.array([1.0]); x = np.zeros((1, 3)); v = np.zeros((1, 3))
    sim = _sim_with_state(nb, m, x, v, np.zeros((1, 3)), 1e-2, "fp64")
    sim.predict(0.0, out=False)
    out = sim.evaluate(torch.tensor([0], dtype=torch.int32, device="cuda")).cpu().numpy()
    assert np.all(out == 0)
    sim.close()


def test_evaluate_duplicates_and_order(nb, oracle):
    n, eps = 500, 1e-3
    m, x, v, a = _plummer_state(oracle, n, seed=9, eps=eps)
    sim = _sim_with_state(nb, m, x, v, a, eps, "fp64")
    sim.predict(0.0, out=False)
    act = np.array([7, 3, 7, 499, 0, 3], dtype=np.int32)
    out = sim.evaluate(torch.as_tensor(act, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(out[:, 0], out[:, 2])
    np.testing.assert_array_equal(out[:, 1], out[:, 5])
    _check_eval(torch.as_tensor(out), oracle.force(m, x, v, a, eps, active=act), 1e-12, "dup")
    sim.close()


def test_evaluate_rejects_index_outside_cluster(nb, oracle):
    n = 100
    m, x, v, a = _plummer_state(oracle, n, seed=2, eps=1e-2)
    sim = _sim_with_state(nb, m, x, v, a, 1e-2, "fp64", offsets=[0, 40, 100])
    sim.predict(0.0, out=False)
    # index 50 belongs to cluster 1, not cluster 0: skipped and reported
    sim.evaluate(torch.tensor([3, 50], dtype=torch.int32, device="cuda"), cluster=0)
    with pytest.raises(nb.NbError) as ei:
        sim.sync()
    assert ei.value.status == 1
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "ex", "fp32"])
def test_evaluate_clusters_are_independent(nb, oracle, precision):
    """Clusters of odd and even sizes: each cluster's j-range starts on a
    whole tile, and the two-particle records of the EX and FP32 arrays hold
    the last particle of an odd cluster beside padding."""
    eps = 1e-3
    sizes = (70, 300, 129, 1, 2, 65)
    parts = [ic.plummer(k, seed=k) for k in sizes]
    m = np.concatenate([p[0] for p in parts]); x = np.concatenate([p[1] for p in parts])
    v = np.concatenate([p[2] for p in parts])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(3)
    a = rng.normal(size=x.shape) * 0.3
    sim = _sim_with_state(nb, m, x, v, a, eps, precision, offsets=offs)
    sim.predict(0.0, out=False)
    for c in range(len(sizes)):
        lo, hi = offs[c], offs[c + 1]
        act = np.arange(lo, hi, dtype=np.int32)
        out = sim.evaluate(torch.as_tensor(act, device="cuda"), cluster=c)
        if hi - lo == 1:
            assert np.all(out.cpu().numpy() == 0)
            continue
        ref = oracle.force(m[lo:hi], x[lo:hi], v[lo:hi], a[lo:hi], eps)
        _check_eval(out, ref, TOL[precision], f"{precision} cluster {c}")
    sim.close()


# ------------------------------------------------------------- corrector
def test_correct_parity(nb, oracle):
    """Same inputs on both sides (the oracle's evaluation feeds the GPU
    corrector): positions, velocities, crackle, new steps and times agree."""
    n, eps = 512, 1e-2
    m, x, v = ic.plummer(n, seed=5)
    ref = oracle.Sim(m, x, v, eps=eps).init()
    ref.run(2.0 ** -5)                       # a few block steps: mixed t, dt, c
    pre = {f: getattr(ref, f).copy() for f in ("m", "x", "v", "a", "j", "s", "c", "t", "dt", "pot")}
    tn, act = ref.select()
    xp, vp, ap = oracle.predict(ref.x, ref.v, ref.a, ref.j, ref.s, ref.c, ref.t, tn)
    acc, jrk, snp, pot = oracle.force(m, xp, vp, ap, eps, active=act)
    ajs = np.concatenate([acc.T, jrk.T, snp.T, pot[None, :]], axis=0)
    ref.step()
    sim = _sim_with_state(nb, m, x, v, pre["a"], eps, "fp64")
    sim.set_state_numpy(pre)
    sim.correct(torch.as_tensor(act.astype(np.int32), device="cuda"), tn,
                torch.as_tensor(ajs, device="cuda"))
    sim.sync()
    got = sim.state_numpy()
    np.testing.assert_allclose(got["x"][act], ref.x[act], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(got["v"][act], ref.v[act], rtol=1e-13, atol=1e-14)
    for f in ("a", "j", "s", "pot"):
        np.testing.assert_array_equal(got[f][act], getattr(ref, f)[act])
    crel = rel_rows(got["c"][act], ref.c[act])
    assert crel.max() < 1e-8, crel.max()
    np.testing.assert_array_equal(got["t"], ref.t)
    mism = np.nonzero(got["dt"] != ref.dt)[0]
    assert len(mism) <= max(1, len(act) // 1000), mism
    untouched = np.setdiff1d(np.arange(n), act)
    np.testing.assert_array_equal(got["x"][untouched], pre["x"][untouched])
    sim.close()


# ----------------------------------------------------------------- start-up
@pytest.mark.parametrize("precision", ["fp64", "ex"])
def test_init_parity(nb, oracle, precision):
    n, eps = 1024, 1e-4
    m, x, v = ic.plummer(n, seed=1)
    ref = oracle.Sim(m, x, v, eps=eps).init()
    sim = nb.Simulation(m, x, v, eps=eps, precision=precision)
    got = sim.state_numpy()
    tol = TOL[precision]
    for f in ("a", "j", "s"):
        e = rel_rows(got[f], getattr(ref, f))
        assert e.max() < tol, (f, e.max())
    assert (np.abs(got["pot"] - ref.pot) / np.abs(ref.pot)).max() < tol
    assert np.all(got["t"] == 0) and np.all(got["c"] == 0)
    assert np.mean(got["dt"] == ref.dt) > 0.99
    sim.close()


# -------------------------------------------------- shared-step trajectory
def test_shared_steps_plummer_1024(nb, oracle, trajectory_envelope):
    """Plummer N=1024, eps=1e-4, shared dt=1/256, 16 steps: per-particle
    trajectory parity plus energy / momentum bookkeeping.

    Tolerance per particle: 2e-14 (a few ulps per step of the corrector's
    rounding) plus 4 times the oracle's own deviation when each of its
    evaluations carries relative errors up to 1e-12 (the FP64 evaluation
    bound).  Close pairs that a 1/256 step resolves poorly amplify any such
    difference (here particles 643 and 187, to about 1e-13)."""
    n, eps, h = 1024, 1e-4, 1.0 / 256
    m, x, v = ic.plummer(n, seed=1)
    xr, vr, env_x, env_v = trajectory_envelope(m, x, v, eps, h, 16, 1e-12)
    ref = oracle.Sim(m, x, v, eps=eps, dt_min=h, dt_max=h).init()
    e0 = ref.energy(0.0)
    sim = nb.Simulation(m, x, v, eps=eps, precision="fp64", dt_min=h, dt_max=h)
    g0 = sim.energy(0.0)
    for _ in range(16):
        tn, na = sim.step()
        assert na == n
    ref.run(16 * h)
    np.testing.assert_array_equal(ref.x, xr)
    got = sim.state_numpy()
    assert np.all(got["t"] == 16 * h)
    ex = rel_rows(got["x"], ref.x)
    ev = rel_rows(got["v"], ref.v)
    wx, wv = np.argsort(-ex)[:5], np.argsort(-ev)[:5]
    print(f"\nconfig-1 trajectory: x max {ex.max():.3e} (particles {wx.tolist()}: {ex[wx]}, "
          f"envelope {env_x[wx]}), v max {ev.max():.3e} (particles {wv.tolist()}: {ev[wv]}, "
          f"envelope {env_v[wv]})")
    bad_x = np.nonzero(ex > 2e-14 + 4 * env_x)[0]
    bad_v = np.nonzero(ev > 2e-14 + 4 * env_v)[0]
    assert bad_x.size == 0, (bad_x[:8], ex[bad_x[:8]], env_x[bad_x[:8]])
    assert bad_v.size == 0, (bad_v[:8], ev[bad_v[:8]], env_v[bad_v[:8]])
    assert np.median(ex) < 1e-15 and np.median(ev) < 1e-14
    g1 = sim.energy(16 * h)
    e1 = ref.energy(16 * h)
    E0, E1 = g0[0] + g0[1], g1[0] + g1[1]
    assert abs(E0 - (e0[0] + e0[1])) < 1e-13 * abs(E0)
    assert abs((E1 - E0) - ((e1[0] + e1[1]) - (e0[0] + e0[1]))) < 1e-10 * abs(E0)
    assert np.linalg.norm(g1[2] - g0[2]) < 1e-14
    sim.close()


# ---------------------------------------------------- block time steps
def test_block_steps_statistics_and_determinism(nb, oracle):
    n, eps, t_end = 512, 1e-2, 0.125
    m, x, v = ic.plummer(n, seed=7)
    ref = oracle.Sim(m, x, v, eps=eps).init()
    e_ref0 = sum(ref.energy(0.0)[:2])
    ref.run(t_end)
    e_ref1 = sum(ref.energy(t_end)[:2])
    states = []
    for _ in range(2):
        sim = nb.Simulation(m, x, v, eps=eps, precision="fp64")
        g0 = sum(sim.energy(0.0)[:2])
        steps, inter = sim.run(t_end)
        g1 = sum(sim.energy(t_end)[:2])
        st = sim.state_numpy()
        states.append(st)
        assert np.all(st["t"] == t_end)
        assert abs(g1 - g0) / abs(g0) < 1e-7
        assert steps == pytest.approx(ref.block_steps, rel=0.2)
        assert inter == pytest.approx(ref.interactions - 2 * n * (n - 1), rel=0.2)
        sim.close()
    for f in ("x", "v", "dt"):
        np.testing.assert_array_equal(states[0][f], states[1][f])
    assert abs(e_ref1 - e_ref0) / abs(e_ref0) < 1e-7
