"""GPU parity of nb_evaluate_range, the evaluation over one tile-aligned part
of a cluster's j-particles (the unit of a j-split of the O(N^2) sums,
paper Sec. 2 and Sec. 4), through the C ABI.

The oracle's sums restricted to a j-range are its full sums with every mass
outside the range set to zero (those pair terms vanish exactly; a particle's
own mass never enters its own sums).  Tolerances as for nb_evaluate: FP64
1e-12, EX 1e-10, FP32 2e-5 (per particle, relative).
"""
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
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def check(out, ref, tol, label):
    acc, jrk, snp, pot = ref
    for name, got, r in (("a", out[0:3].T, acc), ("j", out[3:6].T, jrk), ("s", out[6:9].T, snp)):
        e = rel_rows(got, r)
        assert e.max() <= tol, f"{label} {name}: {e.max():.3e}"
    e = np.abs(out[9] - pot) / np.where(pot != 0, np.abs(pot), 1.0)
    assert e.max() <= tol, f"{label} pot: {e.max():.3e}"


def make_sim(nb, n, precision, seed, eps):
    m, x, v = ic.plummer(n, seed=seed)
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(n, 3)) * 0.3
    sim = nb.Simulation(m, x, v, eps=eps, precision=precision, keep_state=True)
    st = {"m": m, "x": x, "v": v, "a": a, "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
          "c": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, 2.0 ** -6), "pot": np.zeros(n)}
    sim.set_state_numpy(st)
    sim.predict(0.0, out=False)
    return sim, m, x, v, a


@pytest.mark.parametrize("precision", ["fp64", "ex", "fp32"])
@pytest.mark.parametrize("n", [1000, 4097])
def test_partition_sums_to_full_and_matches_oracle(nb, oracle, precision, n):
    eps = 1e-4
    sim, m, x, v, a = make_sim(nb, n, precision, n + 7, eps)
    rng = np.random.default_rng(n)
    for A in (1, 77, n):
        act = np.sort(rng.choice(n, A, replace=False)).astype(np.int32)
        at = torch.as_tensor(act, device="cuda")
        full = sim.evaluate(at).cpu().numpy()
        bounds = [0, 256, 640, n]
        total = np.zeros_like(full)
        for lo, hi in zip(bounds[:-1], bounds[1:]):
            part = sim.evaluate_range(at, lo, hi).cpu().numpy()
            total += part
            mm = m.copy()
            mm[:lo] = 0.0
            mm[hi:] = 0.0
            check(part, oracle.force(mm, x, v, a, eps, active=act), TOL[precision],
                  f"{precision} n={n} A={A} j=[{lo},{hi})")
        check(total, (full[0:3].T, full[3:6].T, full[6:9].T, full[9]), TOL[precision],
              f"{precision} n={n} A={A} sum of parts")
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "ex"])
def test_range_with_stream_k_ranges(nb, oracle, precision):
    """Enough work for stream-K ranges (i-tiles x j-tiles of the range spread
    evenly over the CTAs), a range in the middle of the cluster."""
    n, eps = 10007, 1e-4
    sim, m, x, v, a = make_sim(nb, n, precision, 5, eps)
    rng = np.random.default_rng(5)
    act = np.sort(rng.choice(n, n - 37, replace=False)).astype(np.int32)
    at = torch.as_tensor(act, device="cuda")
    lo, hi = 1024, 8192
    part = sim.evaluate_range(at, lo, hi).cpu().numpy()
    again = sim.evaluate_range(at, lo, hi).cpu().numpy()
    np.testing.assert_array_equal(part, again)
    pick = np.sort(rng.choice(len(act), 256, replace=False))
    mm = m.copy()
    mm[:lo] = 0.0
    mm[hi:] = 0.0
    check(part[:, pick], oracle.force(mm, x, v, a, eps, active=act[pick]), TOL[precision],
          f"{precision} stream-K range")
    sim.close()


def test_empty_and_invalid_ranges(nb):
    n = 300
    sim, m, x, v, a = make_sim(nb, n, "fp64", 3, 1e-3)
    at = torch.tensor([0, 5, 299], dtype=torch.int32, device="cuda")
    out = sim.evaluate_range(at, 128, 128).cpu().numpy()
    assert np.all(out == 0)
    for lo, hi in ((1, 64), (0, 100), (64, 0), (0, 301), (-64, 64)):
        with pytest.raises(nb.NbError) as e:
            sim.evaluate_range(at, lo, hi)
        assert e.value.status == 1, (lo, hi)
    # the whole cluster as one range is nb_evaluate
    np.testing.assert_allclose(sim.evaluate_range(at, 0, n).cpu().numpy(),
                               sim.evaluate(at).cpu().numpy(), rtol=1e-13, atol=0)
    sim.sync()
    sim.close()
