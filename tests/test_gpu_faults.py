"""Failure detection on the GPU without a GPU fault: bounded device-side waits
give up and report, and non-finite state is reported through the device error
word; in both cases the context stays usable."""
import time

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


def test_bounded_wait_gives_up_and_device_stays_usable(nb, oracle):
    t0 = time.perf_counter()
    st = nb.nb_selftest_wait_timeout(0.1)
    dt = time.perf_counter() - t0
    assert st == 6, nb.STATUS.get(st, st)          # NB_ETIMEOUT
    assert dt < 5.0
    # the same process and device keep working
    n = 300
    m, x, v = ic.plummer(n, seed=30)
    sim = nb.Simulation(m, x, v, eps=1e-2)
    sim.predict(0.0, out=False)
    st_ = sim.state_numpy()
    out = sim.evaluate(torch.arange(n, dtype=torch.int32, device="cuda")).cpu().numpy()
    acc = oracle.force(m, st_["x"], st_["v"], st_["a"], 1e-2)[0]
    assert np.abs(out[0:3].T - acc).max() < 1e-12 * np.abs(acc).max()
    sim.close()


def test_nonfinite_state_is_reported(nb):
    n = 500
    m, x, v = ic.plummer(n, seed=31)
    sim = nb.Simulation(m, x, v, eps=1e-2)
    st = sim.state_numpy()
    st["x"][17, 1] = np.nan                        # planted on the host, in the input
    sim.set_state_numpy(st)
    with pytest.raises(nb.NbError) as e:
        sim.run(1.0 / 32)
    assert e.value.status == 4                     # NB_ENONFINITE
    sim.close()
    # a fresh context on the same device is healthy
    sim2 = nb.Simulation(m, x, v, eps=1e-2)
    sim2.run(1.0 / 64)
    assert sim2.counters()["device_errors"] == 0
    sim2.close()
