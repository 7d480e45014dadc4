"""CPU checks of the C-ABI boundary: the library builds, loads and exports
every function include/*.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1812_00367_gb300 import build as nbbuild
from paper_1812_00367_gb300 import nb


@pytest.fixture(scope="module")
def libpath():
    return nbbuild.build()


def test_headers_declare_the_hot_path_calls():
    names = nb.declared_symbols()
    for required in ("nb_init", "nb_predict", "nb_evaluate", "nb_correct_and_timestep", "nb_step"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in nb.declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_signatures_cover_declarations(libpath):
    L = nb.load(libpath)
    for s in nb.declared_symbols():
        assert getattr(L, s).restype is not None or s == "nb_free", s


def test_status_strings(libpath):
    L = nb.load(libpath)
    assert L.nb_status_string(0) == b"NB_OK"
    assert L.nb_status_string(6) == b"NB_ETIMEOUT"


def test_init_rejects_bad_arguments_before_touching_the_gpu(libpath):
    """Host-side validation returns NB_EINVAL without any CUDA call."""
    L = nb.load(libpath)
    ctx = ctypes.c_void_p()
    st = nb.nb_state()
    p = nb.nb_params(1e-2, 0.4, 0.01, 2.0 ** -20, 2.0 ** -3, 0, 0)
    # NULL state buffers
    assert L.nb_init(ctypes.byref(ctx), ctypes.byref(p), 10, ctypes.byref(st), 1, None, None) == 1
    assert b"NULL" in L.nb_last_error(None)
    # dt_min not a power of two
    p2 = nb.nb_params(1e-2, 0.4, 0.01, 3e-6, 2.0 ** -3, 0, 0)
    assert L.nb_init(ctypes.byref(ctx), ctypes.byref(p2), 10, ctypes.byref(st), 1, None, None) == 1
    # n = 0
    assert L.nb_init(ctypes.byref(ctx), ctypes.byref(p), 0, ctypes.byref(st), 1, None, None) == 1
    assert ctx.value is None
    # integration order other than 4 / 6, and a non-zero reserved field
    null_free = {f: 8 for f in nb.STATE_FIELDS}  # any non-NULL value: not dereferenced
    st2 = nb.nb_state(**null_free)
    p3 = nb.nb_params(1e-2, 0.4, 0.01, 2.0 ** -20, 2.0 ** -3, 0, 0, 5, 0)
    assert L.nb_init(ctypes.byref(ctx), ctypes.byref(p3), 10, ctypes.byref(st2), 1, None, None) == 1
    assert b"order" in L.nb_last_error(None)
    p4 = nb.nb_params(1e-2, 0.4, 0.01, 2.0 ** -20, 2.0 ** -3, 0, 0, 4, 1)
    assert L.nb_init(ctypes.byref(ctx), ctypes.byref(p4), 10, ctypes.byref(st2), 1, None, None) == 1
    assert b"reserved" in L.nb_last_error(None)


def test_params_layout_matches_header():
    """nb_params: five doubles, then precision, flags, order, reserved."""
    assert ctypes.sizeof(nb.nb_params) == 56
    assert nb.nb_params.order.offset == 48


def test_no_cpu_fallback_in_package():
    """The product path never imports the oracle."""
    pkg = os.path.dirname(nb.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(".py"):
                text = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", text, re.M), f
