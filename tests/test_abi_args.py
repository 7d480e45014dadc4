"""CPU checks of the C ABI's argument validation: every entry point that
takes a context rejects a NULL one with NB_EINVAL and a message, and the
allocation-free evaluation rejects out-of-range sizes, a negative or
non-finite softening and NULL buffers, all before any CUDA call (these run
without a GPU)."""
import ctypes

import pytest

from paper_1812_00367_gb300 import build as nbbuild
from paper_1812_00367_gb300 import nb

NB_OK, NB_EINVAL = 0, 1


@pytest.fixture(scope="module")
def L():
    return nb.load(nbbuild.build())


def _msg(L):
    return L.nb_last_error(None).decode()


def test_null_context_is_rejected_by_every_entry_point(L):
    d = ctypes.c_double()
    i32 = ctypes.c_int32()
    i64 = ctypes.c_int64()
    st = nb.nb_state()
    cnt = nb.nb_counters()
    three = (ctypes.c_double * 3)()
    calls = {
        "nb_predict": lambda: L.nb_predict(None, 0.0, None),
        "nb_evaluate": lambda: L.nb_evaluate(None, 0, None, 1, None),
        "nb_evaluate_range": lambda: L.nb_evaluate_range(None, 0, None, 1, 0, 64, None),
        "nb_correct_and_timestep": lambda: L.nb_correct_and_timestep(None, 0, None, 1, 0.0, None),
        "nb_step": lambda: L.nb_step(None, ctypes.byref(d), ctypes.byref(i32)),
        "nb_run": lambda: L.nb_run(None, 1.0, -1, ctypes.byref(i64), ctypes.byref(d)),
        "nb_energy": lambda: L.nb_energy(None, 0, 0.0, ctypes.byref(d), ctypes.byref(d), three, three),
        "nb_energy_all": lambda: L.nb_energy_all(None, 0.0, three),
        "nb_get_state": lambda: L.nb_get_state(None, ctypes.byref(st)),
        "nb_set_state": lambda: L.nb_set_state(None, ctypes.byref(st)),
        "nb_get_counters": lambda: L.nb_get_counters(None, ctypes.byref(cnt)),
        "nb_autotune": lambda: L.nb_autotune(None, None),
        "nb_sync": lambda: L.nb_sync(None),
    }
    for name, call in calls.items():
        assert call() == NB_EINVAL, name
        assert name in _msg(L), (name, _msg(L))
    L.nb_free(None)  # a no-op


@pytest.mark.parametrize("n, n_active, eps, what", [
    (0, 1, 1e-3, "n must be"),
    (32769, 1, 1e-3, "n must be"),
    (-5, 1, 1e-3, "n must be"),
    (100, -1, 1e-3, "n_active must be"),
    (100, 32769, 1e-3, "n_active must be"),
    (100, 1, -1e-3, "eps must be"),
    (100, 1, float("inf"), "eps must be"),
    (100, 1, float("nan"), "eps must be"),
    (100, 1, 1e-3, "NULL pointer"),
])
def test_noalloc_rejects_bad_arguments_before_any_cuda_call(L, n, n_active, eps, what):
    assert L.nb_evaluate_noalloc(None, n, eps, None, n_active, None, None) == NB_EINVAL
    assert what in _msg(L)


def test_noalloc_empty_active_set_is_a_no_op(L):
    # n_active == 0 returns before the buffers or the device are looked at
    assert L.nb_evaluate_noalloc(None, 100, 1e-3, None, 0, None, None) == NB_OK
    assert L.nb_evaluate_noalloc(None, 32768, 0.0, None, 0, None, None) == NB_OK
