"""Thin Python binding of libnb (include/nb.h), the GB300 hot path of the
Hermite 6th-order block-time-step N-body integrator.

Functions carry the C names and only marshal arguments: every step of the
method runs in the CUDA library.  Device buffers are torch tensors (torch is
used for device memory and streams only).  There is no CPU fallback: if the
library is not built, or no GPU is present, calls raise.

Layout at the boundary: SoA, vectors [3][n] float64, scalars [n] float64.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libnb.so")
HEADERS = [os.path.join(os.path.dirname(_HERE), "include", h) for h in ("nb.h", "nb_probe.h")]

NB_FP64, NB_EX, NB_FP32, NB_FP32X = 0, 1, 2, 3
PRECISIONS = {"fp64": NB_FP64, "ex": NB_EX, "fp32": NB_FP32, "fp32x": NB_FP32X}
NB_INIT_KEEP_STATE = 1
NB_TIME_EVAL = 2
NB_NO_STREAMK = 4
STATUS = {0: "NB_OK", 1: "NB_EINVAL", 2: "NB_ENOMEM", 3: "NB_ECUDA", 4: "NB_ENONFINITE",
          5: "NB_EDTUNDERFLOW", 6: "NB_ETIMEOUT", 7: "NB_ESTATE"}


class NbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class nb_params(C.Structure):
    _fields_ = [("eps", C.c_double), ("eta", C.c_double), ("eta_init", C.c_double),
                ("dt_min", C.c_double), ("dt_max", C.c_double), ("precision", C.c_int32),
                ("flags", C.c_uint32), ("order", C.c_int32), ("reserved", C.c_int32)]


STATE_FIELDS = ("m", "x", "v", "a", "j", "s", "c", "t", "dt", "pot")
VECTOR_FIELDS = ("x", "v", "a", "j", "s", "c")


class nb_state(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in STATE_FIELDS]


class nb_counters(C.Structure):
    _fields_ = [("block_steps", C.c_int64), ("interactions", C.c_double),
                ("dt_underflows", C.c_int64), ("device_errors", C.c_uint32),
                ("kernel_launches", C.c_int64), ("eval_launches", C.c_int64),
                ("eval_ms", C.c_double)]


_lock = threading.Lock()
_lib = None


def declared_symbols() -> list[str]:
    """Function names declared in include/*.h."""
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(nb_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def load(path: str = LIB_PATH):
    """Load libnb.so and declare its signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libnb.so not built ({path}); run paper_1812_00367_gb300.build.build()")
        L = C.CDLL(path)
        vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        pd = C.POINTER(C.c_double)
        sig = {
            "nb_init": ([C.POINTER(vp), C.POINTER(nb_params), i64, C.POINTER(nb_state), i32,
                         C.POINTER(C.c_int64), vp], C.c_int),
            "nb_predict": ([vp, d, vp], C.c_int),
            "nb_evaluate": ([vp, i32, vp, i32, vp], C.c_int),
            "nb_evaluate_range": ([vp, i32, vp, i32, i64, i64, vp], C.c_int),
            "nb_correct_and_timestep": ([vp, i32, vp, i32, d, vp], C.c_int),
            "nb_step": ([vp, pd, C.POINTER(C.c_int32)], C.c_int),
            "nb_run": ([vp, d, i64, C.POINTER(C.c_int64), pd], C.c_int),
            "nb_energy": ([vp, i32, d, pd, pd, pd, pd], C.c_int),
            "nb_energy_all": ([vp, d, pd], C.c_int),
            "nb_get_state": ([vp, C.POINTER(nb_state)], C.c_int),
            "nb_set_state": ([vp, C.POINTER(nb_state)], C.c_int),
            "nb_get_counters": ([vp, C.POINTER(nb_counters)], C.c_int),
            "nb_autotune": ([vp, C.c_char_p], C.c_int),
            "nb_sync": ([vp], C.c_int),
            "nb_last_error": ([vp], C.c_char_p),
            "nb_status_string": ([C.c_int], C.c_char_p),
            "nb_free": ([vp], None),
            "nb_probe_fma_peak": ([i32, i64, vp, pd, pd], C.c_int),
            "nb_selftest_wait_timeout": ([d, vp], C.c_int),
            "nb_probe_rsqrt": ([i32, vp, vp, i64, vp], C.c_int),
            "nb_evaluate_noalloc": ([vp, i64, d, vp, i32, vp, vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _check(status: int, ctx=None):
    if status != 0:
        msg = load().nb_last_error(ctx).decode(errors="replace")
        raise NbError(status, msg)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def make_state(tensors: dict) -> nb_state:
    return nb_state(*[C.c_void_p(_ptr(tensors[f])) for f in STATE_FIELDS])


def host_state(arrays: dict) -> nb_state:
    """nb_state over host numpy arrays (C-contiguous float64)."""
    return nb_state(*[C.c_void_p(arrays[f].ctypes.data) for f in STATE_FIELDS])


# ------------------------------------------------------------------ raw calls
def nb_init(params: nb_params, n: int, state: nb_state, offsets=None, stream=None) -> int:
    L = load()
    ctx = C.c_void_p()
    if offsets is None:
        nc, offp = 1, None
    else:
        arr = np.ascontiguousarray(offsets, dtype=np.int64)
        nc, offp = len(arr) - 1, arr.ctypes.data_as(C.POINTER(C.c_int64))
    st = L.nb_init(C.byref(ctx), C.byref(params), int(n), C.byref(state), int(nc), offp,
                   _stream_handle(stream))
    _check(st, None)
    return ctx.value


def nb_predict(ctx, t_next: float, out=None):
    _check(load().nb_predict(ctx, float(t_next), _ptr(out)), ctx)


def nb_evaluate(ctx, cluster: int, active, n_active: int, out):
    _check(load().nb_evaluate(ctx, int(cluster), _ptr(active), int(n_active), _ptr(out)), ctx)


def nb_evaluate_range(ctx, cluster: int, active, n_active: int, j_begin: int, j_end: int, out):
    _check(load().nb_evaluate_range(ctx, int(cluster), _ptr(active), int(n_active), int(j_begin),
                                    int(j_end), _ptr(out)), ctx)


def nb_correct_and_timestep(ctx, cluster: int, active, n_active: int, t_next: float, ajs):
    _check(load().nb_correct_and_timestep(ctx, int(cluster), _ptr(active), int(n_active),
                                          float(t_next), _ptr(ajs)), ctx)


def nb_step(ctx, want_outputs: bool = True):
    tn, na = C.c_double(0.0), C.c_int32(0)
    if want_outputs:
        _check(load().nb_step(ctx, C.byref(tn), C.byref(na)), ctx)
        return tn.value, na.value
    _check(load().nb_step(ctx, None, None), ctx)
    return None


def nb_run(ctx, t_end: float, max_block_steps: int = -1):
    bs, inter = C.c_int64(0), C.c_double(0.0)
    _check(load().nb_run(ctx, float(t_end), int(max_block_steps), C.byref(bs), C.byref(inter)), ctx)
    return bs.value, inter.value


def nb_energy(ctx, cluster: int, t: float):
    ek, ep = C.c_double(), C.c_double()
    P = (C.c_double * 3)()
    Lm = (C.c_double * 3)()
    _check(load().nb_energy(ctx, int(cluster), float(t), C.byref(ek), C.byref(ep), P, Lm), ctx)
    return ek.value, ep.value, np.array(P[:]), np.array(Lm[:])


def nb_energy_all(ctx, n_clusters: int, t: float) -> np.ndarray:
    """(n_clusters, 8) array: E_kin, E_pot, P[3], L[3] of every cluster."""
    out = np.zeros((n_clusters, 8))
    _check(load().nb_energy_all(ctx, float(t), out.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return out


def nb_get_state(ctx, dst: nb_state):
    _check(load().nb_get_state(ctx, C.byref(dst)), ctx)


def nb_set_state(ctx, src: nb_state):
    _check(load().nb_set_state(ctx, C.byref(src)), ctx)


def nb_get_counters(ctx) -> dict:
    c = nb_counters()
    _check(load().nb_get_counters(ctx, C.byref(c)), ctx)
    return {f: getattr(c, f) for f, _ in nb_counters._fields_}


def nb_autotune(ctx, cache_path: str | None = None):
    _check(load().nb_autotune(ctx, cache_path.encode() if cache_path else None), ctx)


def nb_sync(ctx):
    _check(load().nb_sync(ctx), ctx)


def nb_free(ctx):
    if ctx:
        load().nb_free(ctx)


def nb_probe_fma_peak(precision: int, iters: int = 4096, stream=None):
    fps, sec = C.c_double(), C.c_double()
    _check(load().nb_probe_fma_peak(int(precision), int(iters), _stream_handle(stream),
                                    C.byref(fps), C.byref(sec)))
    return fps.value, sec.value


# ------------------------------------------------------------- convenience
class Simulation:
    """A context over torch-owned device state.

    ``m (n,)``, ``x v (n,3)`` are taken in the natural row layout and stored
    on the device in the library's [3][n] layout.
    """

    def __init__(self, m, x, v, eps, eta=0.4, eta_init=0.01, dt_min=2.0 ** -20,
                 dt_max=2.0 ** -3, precision="fp64", offsets=None, device="cuda",
                 keep_state=False, stream=None, time_eval=False, order=6, streamk=True):
        import torch
        n = int(np.asarray(m).shape[0])
        self.n = n
        self.device = torch.device(device)
        f64 = dict(dtype=torch.float64, device=self.device)
        self.buf = {"m": torch.as_tensor(np.ascontiguousarray(m, dtype=np.float64)).to(**f64)}
        for f in VECTOR_FIELDS:
            self.buf[f] = torch.zeros((3, n), **f64)
        for f in ("t", "dt", "pot"):
            self.buf[f] = torch.zeros(n, **f64)
        self.buf["x"].copy_(torch.as_tensor(np.asarray(x, dtype=np.float64).T.copy()))
        self.buf["v"].copy_(torch.as_tensor(np.asarray(v, dtype=np.float64).T.copy()))
        self.offsets = None if offsets is None else np.asarray(offsets, dtype=np.int64)
        self.params = nb_params(float(eps), float(eta), float(eta_init), float(dt_min),
                                float(dt_max), PRECISIONS[precision] if isinstance(precision, str)
                                else int(precision),
                                (NB_INIT_KEEP_STATE if keep_state else 0) | (NB_TIME_EVAL if time_eval else 0)
                                | (0 if streamk else NB_NO_STREAMK),
                                int(order), 0)
        self.order = int(order)
        self.stream = stream
        self._state = make_state(self.buf)
        torch.cuda.synchronize(self.device)
        self.ctx = nb_init(self.params, n, self._state, self.offsets, stream)

    def close(self):
        if getattr(self, "ctx", None):
            nb_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- calls
    def predict(self, t_next, out=True):
        import torch
        o = torch.empty((10, self.n), dtype=torch.float64, device=self.device) if out else None
        nb_predict(self.ctx, t_next, o)
        return o

    def evaluate(self, active, cluster=0):
        import torch
        act = torch.as_tensor(active, dtype=torch.int32, device=self.device).contiguous()
        out = torch.empty((10, act.numel()), dtype=torch.float64, device=self.device)
        nb_evaluate(self.ctx, cluster, act, act.numel(), out)
        return out

    def evaluate_range(self, active, j_begin, j_end, cluster=0):
        import torch
        act = torch.as_tensor(active, dtype=torch.int32, device=self.device).contiguous()
        out = torch.empty((10, act.numel()), dtype=torch.float64, device=self.device)
        nb_evaluate_range(self.ctx, cluster, act, act.numel(), j_begin, j_end, out)
        return out

    def correct(self, active, t_next, ajs, cluster=0):
        import torch
        act = torch.as_tensor(active, dtype=torch.int32, device=self.device).contiguous()
        nb_correct_and_timestep(self.ctx, cluster, act, act.numel(), t_next, ajs.contiguous())

    def step(self):
        return nb_step(self.ctx)

    def run(self, t_end, max_block_steps=-1):
        return nb_run(self.ctx, t_end, max_block_steps)

    def energy(self, t, cluster=-1):
        return nb_energy(self.ctx, cluster, t)

    def energy_all(self, t):
        nc = 1 if self.offsets is None else len(self.offsets) - 1
        return nb_energy_all(self.ctx, nc, t)

    def counters(self):
        return nb_get_counters(self.ctx)

    def autotune(self, cache_path=None):
        nb_autotune(self.ctx, cache_path)

    def sync(self):
        nb_sync(self.ctx)

    def state_numpy(self) -> dict:
        """State copied to host in the natural layout: vectors (n, 3)."""
        host = {f: np.zeros((3, self.n)) if f in VECTOR_FIELDS else np.zeros(self.n)
                for f in STATE_FIELDS}
        nb_get_state(self.ctx, host_state(host))
        return {f: (a.T.copy() if f in VECTOR_FIELDS else a) for f, a in host.items()}

    def set_state_numpy(self, st: dict):
        host = {}
        for f in STATE_FIELDS:
            a = np.asarray(st[f], dtype=np.float64)
            host[f] = np.ascontiguousarray(a.T if f in VECTOR_FIELDS else a)
        nb_set_state(self.ctx, host_state(host))


def nb_probe_rsqrt(which: int, x, y, stream=None):
    """y = 1/sqrt(x) elementwise with the evaluation kernel's own reciprocal
    square root (which = 0: FP64, 1: float-float); x, y: device float64 tensors."""
    _check(load().nb_probe_rsqrt(int(which), _ptr(x), _ptr(y), int(x.numel()),
                                 _stream_handle(stream)))


def nb_selftest_wait_timeout(budget_seconds: float, stream=None) -> int:
    """Returns the raw status: NB_ETIMEOUT (6) is the expected answer."""
    return int(load().nb_selftest_wait_timeout(float(budget_seconds), _stream_handle(stream)))
