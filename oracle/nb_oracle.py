"""ctypes binding of the FP64 CPU oracle (``nb_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``; the
product path never imports it.  It shares nothing with the CUDA library.

Arrays follow the oracle's own layout: vectors ``(n, 3)`` float64 C-contiguous,
scalars ``(n,)``.  The method is the 6th-order Hermite scheme with block time
steps (paper Sec. 2 and Sec. 4; formulas after Nitadori & Makino 2008).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libnb_oracle.so")
_lock = threading.Lock()
_lib = None

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over active i, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            L.orc_force.argtypes = [C.c_int64, _D, _D, _D, _D, C.c_double, C.c_int64,
                                    _I64, _D, _D, _D, _D]
            L.orc_predict.argtypes = [C.c_int64, _D, _D, _D, _D, _D, _D, _D, C.c_double,
                                      _D, _D, _D]
            L.orc_interp_derivs.argtypes = [C.c_double] + [_D] * 9
            L.orc_correct.argtypes = [C.c_double] + [_D] * 10
            L.orc_dt_criterion.argtypes = [_D] * 6 + [C.c_double]
            L.orc_dt_criterion.restype = C.c_double
            L.orc_dt_initial.argtypes = [_D, _D, _D, C.c_double]
            L.orc_dt_initial.restype = C.c_double
            L.orc_dt_quantize.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_int)]
            L.orc_dt_quantize.restype = C.c_double
            L.orc_dt_quantize_initial.argtypes = [C.c_double] * 3
            L.orc_dt_quantize_initial.restype = C.c_double
            L.orc_sim_sizeof.restype = C.c_size_t
            L.orc_bind.argtypes = [C.c_void_p, C.c_int64] + [C.c_double] * 5 + [_D] * 10
            L.orc_bind.restype = C.c_int
            L.orc_free.argtypes = [C.c_void_p]
            L.orc_init.argtypes = [C.c_void_p]
            L.orc_select.argtypes = [C.c_void_p, _D, _I64]
            L.orc_select.restype = C.c_int64
            L.orc_block_step.argtypes = [C.c_void_p, _D]
            L.orc_block_step.restype = C.c_int64
            L.orc_run.argtypes = [C.c_void_p, C.c_double, C.c_int64, _D]
            L.orc_run.restype = C.c_int64
            L.orc_energy.argtypes = [C.c_void_p, C.c_double, _D, _D, _D, _D]
            L.orc_underflows.argtypes = [C.c_void_p]
            L.orc_underflows.restype = C.c_int64
            L.orc_num_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = None
            L.orc_predict4.argtypes = [C.c_int64] + [_D] * 5 + [C.c_double, _D, _D]
            L.orc_correct4.argtypes = [C.c_double] + [_D] * 8
            L.orc_interp4.argtypes = [C.c_double] + [_D] * 6
            L.orc_dt_aarseth.argtypes = [_D] * 4 + [C.c_double]
            L.orc_dt_aarseth.restype = C.c_double
            L.orc_set_order.argtypes = [C.c_void_p, C.c_int]
            L.orc_set_order.restype = C.c_int
            L.orc_set_noise.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double,
                                        C.c_uint64]
            L.orc_set_noise.restype = C.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def force(m, xp, vp, ap, eps, active=None):
    """Acceleration, jerk, snap and potential of the active particles (NM08 sums).

    Returns (acc, jerk, snap, pot) with shapes (A, 3), (A, 3), (A, 3), (A,).
    """
    m = _f64(m)
    n = m.shape[0]
    xp, vp, ap = (_f64(q, (n, 3)) for q in (xp, vp, ap))
    act = (np.arange(n, dtype=np.int64) if active is None
           else np.ascontiguousarray(active, dtype=np.int64))
    na = act.shape[0]
    acc = np.zeros((na, 3)); jrk = np.zeros((na, 3)); snp = np.zeros((na, 3))
    pot = np.zeros(na)
    lib().orc_force(n, _p(m), _p(xp), _p(vp), _p(ap), float(eps) ** 2, na,
                    act.ctypes.data_as(_I64), _p(acc), _p(jrk), _p(snp), _p(pot))
    return acc, jrk, snp, pot


def predict(x, v, a, j, s, c, t, t_next):
    n = np.asarray(t).shape[0]
    x, v, a, j, s, c = (_f64(q, (n, 3)) for q in (x, v, a, j, s, c))
    t = _f64(t)
    xp = np.zeros((n, 3)); vp = np.zeros((n, 3)); ap = np.zeros((n, 3))
    lib().orc_predict(n, _p(x), _p(v), _p(a), _p(j), _p(s), _p(c), _p(t),
                      float(t_next), _p(xp), _p(vp), _p(ap))
    return xp, vp, ap


def interp_derivs(h, a0, j0, s0, a1, j1, s1):
    args = [_f64(q, (3,)) for q in (a0, j0, s0, a1, j1, s1)]
    d3 = np.zeros(3); d4 = np.zeros(3); d5 = np.zeros(3)
    lib().orc_interp_derivs(float(h), *[_p(q) for q in args], _p(d3), _p(d4), _p(d5))
    return d3, d4, d5


def correct(h, x0, v0, a0, j0, s0, a1, j1, s1):
    args = [_f64(q, (3,)) for q in (x0, v0, a0, j0, s0, a1, j1, s1)]
    x1 = np.zeros(3); v1 = np.zeros(3)
    lib().orc_correct(float(h), *[_p(q) for q in args], _p(x1), _p(v1))
    return x1, v1


def dt_criterion(a, j, s, d3, d4, d5, eta):
    args = [_f64(q, (3,)) for q in (a, j, s, d3, d4, d5)]
    return float(lib().orc_dt_criterion(*[_p(q) for q in args], float(eta)))


def dt_initial(a, j, s, eta_init):
    args = [_f64(q, (3,)) for q in (a, j, s)]
    return float(lib().orc_dt_initial(*[_p(q) for q in args], float(eta_init)))


def predict4(x, v, a, j, t, t_next):
    """4th-order predictor (through jerk): (xp, vp)."""
    n = np.asarray(t).shape[0]
    x, v, a, j = (_f64(q, (n, 3)) for q in (x, v, a, j))
    t = _f64(t)
    xp = np.zeros((n, 3)); vp = np.zeros((n, 3))
    lib().orc_predict4(n, _p(x), _p(v), _p(a), _p(j), _p(t), float(t_next), _p(xp), _p(vp))
    return xp, vp


def correct4(h, x0, v0, a0, j0, a1, j1):
    args = [_f64(q, (3,)) for q in (x0, v0, a0, j0, a1, j1)]
    x1 = np.zeros(3); v1 = np.zeros(3)
    lib().orc_correct4(float(h), *[_p(q) for q in args], _p(x1), _p(v1))
    return x1, v1


def interp4(h, a0, j0, a1, j1):
    args = [_f64(q, (3,)) for q in (a0, j0, a1, j1)]
    s1 = np.zeros(3); c1 = np.zeros(3)
    lib().orc_interp4(float(h), *[_p(q) for q in args], _p(s1), _p(c1))
    return s1, c1


def dt_aarseth(a, j, s, c, eta):
    args = [_f64(q, (3,)) for q in (a, j, s, c)]
    return float(lib().orc_dt_aarseth(*[_p(q) for q in args], float(eta)))


def dt_quantize(dt_crit, dt_old, t1, dt_min, dt_max):
    uf = C.c_int(0)
    r = lib().orc_dt_quantize(float(dt_crit), float(dt_old), float(t1), float(dt_min),
                              float(dt_max), C.byref(uf))
    return float(r), bool(uf.value)


def dt_quantize_initial(dt0, dt_min, dt_max):
    return float(lib().orc_dt_quantize_initial(float(dt0), float(dt_min), float(dt_max)))


class Sim:
    """FP64 block-time-step Hermite integrator (oracle), 6th order or 4th order.

    State arrays are numpy attributes in the oracle layout:
    ``m (n,)``, ``x v a j s c (n,3)``, ``t dt pot (n,)``.
    """

    def __init__(self, m, x, v, eps, eta=0.4, eta_init=0.01,
                 dt_min=2.0 ** -20, dt_max=2.0 ** -3, order=6):
        L = lib()
        self.n = n = int(np.asarray(m).shape[0])
        self.m = _f64(m).copy()
        self.x = _f64(x, (n, 3)).copy()
        self.v = _f64(v, (n, 3)).copy()
        for name in ("a", "j", "s", "c"):
            setattr(self, name, np.zeros((n, 3)))
        self.t = np.zeros(n); self.dt = np.zeros(n); self.pot = np.zeros(n)
        self.eps, self.eta, self.eta_init = float(eps), float(eta), float(eta_init)
        self.dt_min, self.dt_max = float(dt_min), float(dt_max)
        self._buf = C.create_string_buffer(int(L.orc_sim_sizeof()))
        rc = L.orc_bind(self._buf, n, self.eps, self.eta, self.eta_init, self.dt_min,
                        self.dt_max, _p(self.m), _p(self.x), _p(self.v), _p(self.a),
                        _p(self.j), _p(self.s), _p(self.c), _p(self.t), _p(self.dt),
                        _p(self.pot))
        if rc != 0:
            raise MemoryError("oracle: allocation failed")
        if L.orc_set_order(self._buf, int(order)) != 0:
            raise ValueError("oracle: order must be 4 or 6")
        self.order = int(order)
        self.block_steps = 0
        self.interactions = 0.0

    def __del__(self):
        try:
            lib().orc_free(self._buf)
        except Exception:
            pass

    def set_noise(self, ea, ej=None, es=None, seed=1):
        """Perturb every later evaluation: each component of a, jerk and snap
        is multiplied by (1 + e u), u uniform in [-1, 1) from a counter-based
        generator keyed by (seed, evaluation, particle, component).  Sizes 0
        (the default) leave the method untouched."""
        ej = ea if ej is None else ej
        es = ea if es is None else es
        if lib().orc_set_noise(self._buf, float(ea), float(ej), float(es), int(seed)) != 0:
            raise ValueError("oracle: noise sizes must be >= 0")
        return self

    def init(self):
        lib().orc_init(self._buf)
        self.interactions += (1.0 if self.order == 4 else 2.0) * self.n * (self.n - 1)
        return self

    def select(self):
        tn = C.c_double(0)
        act = np.zeros(self.n, dtype=np.int64)
        na = lib().orc_select(self._buf, C.byref(tn), act.ctypes.data_as(_I64))
        return tn.value, act[:na]

    def step(self):
        tn = C.c_double(0)
        na = lib().orc_block_step(self._buf, C.byref(tn))
        self.block_steps += 1
        self.interactions += float(na) * (self.n - 1)
        return tn.value, int(na)

    def run(self, t_end, max_steps=-1):
        inter = C.c_double(0.0)
        k = lib().orc_run(self._buf, float(t_end), int(max_steps), C.byref(inter))
        self.block_steps += int(k)
        self.interactions += inter.value
        return int(k)

    def energy(self, t=None):
        """(E_kin, E_pot, P, L) at common time t (default: max particle time)."""
        if t is None:
            t = float(self.t.max()) if self.n else 0.0
        ek = C.c_double(); ep = C.c_double()
        P = np.zeros(3); Lm = np.zeros(3)
        lib().orc_energy(self._buf, float(t), C.byref(ek), C.byref(ep), _p(P), _p(Lm))
        return ek.value, ep.value, P, Lm

    @property
    def underflows(self) -> int:
        return int(lib().orc_underflows(self._buf))


if __name__ == "__main__":  # pragma: no cover - manual build entry
    print(build(force="--force" in sys.argv))
