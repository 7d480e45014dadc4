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


def test_noalloc_rejects_sizes_beyond_its_array(lib):
    nb, L = lib
    rc = L.nb_evaluate_noalloc(None, 40000, 1e-3, None, 1, None, None)
    assert rc == 1 and b"32768" in L.nb_last_error(None)
