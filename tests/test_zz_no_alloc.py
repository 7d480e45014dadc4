"""GPU test of nb_evaluate_noalloc, the evaluation entry for callers that
cannot allocate device memory (their framework's pool owns the memory, or
their loop must not allocate).  It must give what nb_evaluate gives on the
same predicted particles, call after call, although all calls share one
fixed working array inside the library.

Kept in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_1812_00367_gb300 import ic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import nb
    nbbuild.build()
    L = nb.load()
    f = L.nb_evaluate_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return nb, L


def _rel_rows(got, ref):
    return np.linalg.norm(got - ref, axis=-1) / np.linalg.norm(ref, axis=-1)


def test_noalloc_matches_nb_evaluate_on_two_calls(lib):
    nb, L = lib
    n, eps = 5000, 1e-3
    m, x, v = ic.plummer(n, seed=21)
    rng = np.random.default_rng(21)
    sim = nb.Simulation(m, x, v, eps=eps, keep_state=True)
    st = {"m": m, "x": x, "v": v, "a": rng.normal(size=(n, 3)) * 0.3, "j": np.zeros((n, 3)),
          "s": np.zeros((n, 3)), "c": np.zeros((n, 3)), "t": np.zeros(n),
          "dt": np.full(n, 2.0 ** -6), "pot": np.zeros(n)}
    sim.set_state_numpy(st)
    pred = sim.predict(0.0)                      # device [10][n]
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row, different active sets (different split plans)
    for A in (777, 64):
        act = torch.as_tensor(np.sort(rng.choice(n, A, replace=False)).astype(np.int32),
                              device="cuda")
        ref = sim.evaluate(act).cpu().numpy()
        out = torch.full((10, A), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.nb_evaluate_noalloc(pred.data_ptr(), n, eps, act.data_ptr(), A, out.data_ptr(),
                                   stream)
        assert rc == 0, L.nb_last_error(None)
        got = out.cpu().numpy()
        for lo, hi in ((0, 3), (3, 6), (6, 9)):
            assert _rel_rows(got[lo:hi].T, ref[lo:hi].T).max() <= 1e-12
        assert (np.abs(got[9] - ref[9]) / np.abs(ref[9])).max() <= 1e-12
    sim.close()


@pytest.fixture(scope="module")
def full_size_case(lib):
    """n at the array's limit (32768) with a realistic predicted state: the
    Plummer accelerations as the 'a' rows (they feed the snap terms)."""
    nb, L = lib
    n, eps = 32768, 1e-4
    m, x, v = ic.plummer(n, seed=22)
    rng = np.random.default_rng(22)
    sim = nb.Simulation(m, x, v, eps=eps, keep_state=True)
    st = {"m": m, "x": x, "v": v, "a": rng.normal(size=(n, 3)), "j": np.zeros((n, 3)),
          "s": np.zeros((n, 3)), "c": np.zeros((n, 3)), "t": np.zeros(n),
          "dt": np.full(n, 2.0 ** -6), "pot": np.zeros(n)}
    sim.set_state_numpy(st)
    pred = sim.predict(0.0)
    yield sim, pred, n, eps, rng
    sim.close()


def _noalloc(L, pred, n, eps, act, stream):
    A = act.numel()
    out = torch.full((10, A), float("nan"), dtype=torch.float64, device="cuda")
    rc = L.nb_evaluate_noalloc(pred.data_ptr(), n, eps, act.data_ptr(), A, out.data_ptr(), stream)
    return rc, out


# every plan of the entry: 32, 8, 2 and 1 lanes per active particle, split
# items capped to the array's partial-sum room (A = 2048, 4096, 32768)
@pytest.mark.parametrize("A", [1, 17, 63, 777, 2048, 4096, 32768])
def test_noalloc_at_the_size_limit_matches_oracle_and_nb_evaluate(lib, oracle, full_size_case, A):
    nb, L = lib
    sim, pred, n, eps, rng = full_size_case
    act_np = (np.arange(n, dtype=np.int32) if A == n
              else np.sort(rng.choice(n, A, replace=False)).astype(np.int32))
    act = torch.as_tensor(act_np, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, out = _noalloc(L, pred, n, eps, act, stream)
    assert rc == 0, L.nb_last_error(None)
    got = out.cpu().numpy()
    ref_gpu = sim.evaluate(act).cpu().numpy()
    for lo, hi in ((0, 3), (3, 6), (6, 9)):
        assert _rel_rows(got[lo:hi].T, ref_gpu[lo:hi].T).max() <= 1e-12
    # the oracle on the same predicted particles (all of them up to 4096
    # active, a sample of 512 beyond)
    p = pred.cpu().numpy()
    pick = np.arange(A) if A <= 4096 else np.sort(rng.choice(A, 512, replace=False))
    acc, jrk, snp, pot = oracle.force(p[9], p[0:3].T, p[3:6].T, p[6:9].T, eps, active=act_np[pick])
    for (lo, hi), r in zip(((0, 3), (3, 6), (6, 9)), (acc, jrk, snp)):
        e = _rel_rows(got[lo:hi, pick].T, r)
        assert e.max() <= 1e-12, (A, lo, e.max())
    assert (np.abs(got[9, pick] - pot) / np.abs(pot)).max() <= 1e-12


def test_noalloc_index_outside_range_is_reported_and_others_evaluated(lib, full_size_case):
    nb, L = lib
    sim, pred, n, eps, rng = full_size_case
    act_np = np.array([5, n, 77, 40000, n - 1], dtype=np.int32)
    act = torch.as_tensor(act_np, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, out = _noalloc(L, pred, n, eps, act, stream)
    assert rc == 1 and b"outside" in L.nb_last_error(None)
    got = out.cpu().numpy()
    assert np.all(got[:, 1] == 0) and np.all(got[:, 3] == 0)
    good = torch.as_tensor(act_np[[0, 2, 4]], device="cuda")
    ref = sim.evaluate(good).cpu().numpy()
    for lo, hi in ((0, 3), (3, 6), (6, 9)):
        assert _rel_rows(got[lo:hi, [0, 2, 4]].T, ref[lo:hi].T).max() <= 1e-12
    # the next call starts clean again (its error word was cleared)
    rc, out = _noalloc(L, pred, n, eps, good, stream)
    assert rc == 0, L.nb_last_error(None)
    again = out.cpu().numpy()
    for lo, hi in ((0, 3), (3, 6), (6, 9)):
        assert _rel_rows(again[lo:hi].T, ref[lo:hi].T).max() <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    nb, L = lib
    rc = L.nb_evaluate_noalloc(None, 40000, 1e-3, None, 1, None, None)
    assert rc == 1 and b"32768" in L.nb_last_error(None)
    rc = L.nb_evaluate_noalloc(None, 100, 1e-3, None, 40000, None, None)
    assert rc == 1 and b"32768" in L.nb_last_error(None)
