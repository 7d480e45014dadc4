"""GPU tests of the batched (many-cluster) path, checkpoint/resume, the
autotuner, energy diagnostics and error paths, through the C ABI."""
import os

import numpy as np
import pytest

from paper_1812_00367_gb300 import ic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00367_gb300 import build as nbbuild
    nbbuild.build()
    from paper_1812_00367_gb300 import nb as nbmod
    nbmod.load()
    return nbmod


def _write_table(path, precision, gl_of_bucket, target):
    with open(path, "w") as f:
        f.write(f"nbtune {precision} 0\n")
        for b in range(32):
            f.write(f"{gl_of_bucket(b)} {target}\n")


@pytest.mark.parametrize("precision", ["fp64", "ex", "fp32x"])
def test_batched_equals_single_bit_for_bit(nb, tmp_path, precision):
    """Each cluster of a batch ends bit-identical to the same cluster run alone
    (same plan table; deterministic reductions)."""
    sizes = [256, 700, 1500, 333]
    batch = ic.plummer_batch(sizes=sizes, seed=4)
    table = str(tmp_path / "table.txt")
    _write_table(table, nb.PRECISIONS[precision], lambda b: 32 if b < 6 else (8 if b < 10 else 1), 64)
    t_end = 0.0625
    # one start-up state for everybody, then every context loads the same table
    full = nb.Simulation(batch.m, batch.x, batch.v, eps=1e-3, precision=precision,
                         offsets=batch.offsets)
    st0 = full.state_numpy()
    full.close()
    bsim = nb.Simulation(batch.m, batch.x, batch.v, eps=1e-3, precision=precision,
                         offsets=batch.offsets, keep_state=True)
    bsim.autotune(table)
    bsim.set_state_numpy(st0)
    bsteps, _ = bsim.run(t_end)
    bstate = bsim.state_numpy()
    for c, n_c in enumerate(sizes):
        lo, hi = batch.offsets[c], batch.offsets[c + 1]
        s1 = nb.Simulation(batch.m[lo:hi], batch.x[lo:hi], batch.v[lo:hi], eps=1e-3,
                           precision=precision, keep_state=True, streamk=False)
        s1.autotune(table)
        s1.set_state_numpy({f: st0[f][lo:hi] for f in st0})
        s1.run(t_end)
        one = s1.state_numpy()
        for f in ("x", "v", "a", "j", "s", "c", "t", "dt", "pot"):
            np.testing.assert_array_equal(bstate[f][lo:hi], one[f], err_msg=f"cluster {c} {f}")
        s1.close()
    assert np.all(bstate["t"] <= t_end) and np.all(bstate["t"] + bstate["dt"] > t_end)
    bsim.close()


def test_batched_energy_per_cluster(nb, oracle):
    sizes = [300, 500]
    batch = ic.plummer_batch(sizes=sizes, seed=8)
    sim = nb.Simulation(batch.m, batch.x, batch.v, eps=1e-2, offsets=batch.offsets)
    tot = sim.energy(0.0, -1)
    parts = [sim.energy(0.0, c) for c in range(2)]
    assert tot[0] == pytest.approx(parts[0][0] + parts[1][0], rel=1e-14)
    assert tot[1] == pytest.approx(parts[0][1] + parts[1][1], rel=1e-14)
    for c in range(2):
        lo, hi = batch.offsets[c], batch.offsets[c + 1]
        ref = oracle.Sim(batch.m[lo:hi], batch.x[lo:hi], batch.v[lo:hi], eps=1e-2).init()
        ek, ep, P, L = ref.energy(0.0)
        assert parts[c][0] == pytest.approx(ek, rel=1e-13)
        assert parts[c][1] == pytest.approx(ep, rel=1e-12)
        np.testing.assert_allclose(parts[c][2], P, atol=1e-15)
        np.testing.assert_allclose(parts[c][3], L, atol=1e-14)
    sim.close()


def test_checkpoint_resume_bit_equal(nb):
    n = 2048
    m, x, v = ic.plummer(n, seed=12)
    a = nb.Simulation(m, x, v, eps=1e-3)
    a.run(1.0 / 32)
    ckpt = a.state_numpy()
    a.run(1.0 / 16)
    ref = a.state_numpy()
    a.close()
    b = nb.Simulation(m, x, v, eps=1e-3, keep_state=True)
    b.set_state_numpy(ckpt)
    b.run(1.0 / 16)
    got = b.state_numpy()
    for f in ("x", "v", "a", "j", "s", "c", "t", "dt", "pot"):
        np.testing.assert_array_equal(got[f], ref[f], err_msg=f)
    b.close()


def test_step_outputs_and_counters(nb, oracle):
    n = 400
    m, x, v = ic.plummer(n, seed=13)
    sim = nb.Simulation(m, x, v, eps=1e-2)
    ref = oracle.Sim(m, x, v, eps=1e-2).init()
    for _ in range(5):
        tn, na = sim.step()
        tr, nr = ref.step()
        assert tn == tr and na == nr
    c = sim.counters()
    assert c["block_steps"] == 5 and c["device_errors"] == 0
    assert c["interactions"] == pytest.approx(ref.interactions - 2 * n * (n - 1))
    assert c["kernel_launches"] == 25
    sim.close()


def test_time_eval_counts_launches(nb):
    m, x, v = ic.plummer(1000, seed=14)
    sim = nb.Simulation(m, x, v, eps=1e-2, time_eval=True)
    steps, inter = sim.run(1.0 / 64)
    c = sim.counters()
    assert c["eval_launches"] >= steps and c["eval_ms"] > 0
    sim.close()


def test_autotune_keeps_results_correct(nb, oracle, tmp_path):
    n, eps = 3000, 1e-3
    m, x, v = ic.plummer(n, seed=15)
    sim = nb.Simulation(m, x, v, eps=eps)
    path = str(tmp_path / "tune.txt")
    sim.autotune(path)
    assert os.path.exists(path)
    sim.autotune(path)                       # cached table loads
    sim.predict(0.0, out=False)
    st = sim.state_numpy()
    for A in (1, 7, 300, n):
        act = np.arange(0, n, max(1, n // A))[:A].astype(np.int32)
        out = sim.evaluate(torch.as_tensor(act, device="cuda")).cpu().numpy()
        acc, jrk, snp, pot = oracle.force(m, st["x"], st["v"], st["a"], eps, active=act)
        for got, ref in ((out[0:3].T, acc), (out[3:6].T, jrk), (out[6:9].T, snp)):
            err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
            assert err.max() < 1e-12
    sim.close()


def test_argument_errors(nb):
    m, x, v = ic.plummer(100, seed=16)
    sim = nb.Simulation(m, x, v, eps=1e-2)
    act = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros((10, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(nb.NbError) as e:
        nb.nb_evaluate(sim.ctx, 1, act, 4, out)       # no cluster 1
    assert e.value.status == 1
    with pytest.raises(nb.NbError):
        nb.nb_evaluate(sim.ctx, 0, act, 101, out)     # more than the cluster
    with pytest.raises(nb.NbError):
        nb.nb_correct_and_timestep(sim.ctx, 0, act, 4, float("nan"), out)
    nb.nb_evaluate(sim.ctx, 0, act, 0, out)           # empty: no-op
    sim.sync()
    sim.close()


def test_energy_all_matches_per_cluster(nb):
    sizes = [200, 900, 411]
    batch = ic.plummer_batch(sizes=sizes, seed=9)
    sim = nb.Simulation(batch.m, batch.x, batch.v, eps=1e-2, offsets=batch.offsets)
    sim.run(1.0 / 64)
    allc = sim.energy_all(1.0 / 64)
    for c in range(len(sizes)):
        ek, ep, P, L = sim.energy(1.0 / 64, c)
        np.testing.assert_allclose(allc[c], [ek, ep, *P, *L], rtol=1e-13, atol=1e-16)
    sim.close()
