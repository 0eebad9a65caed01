"""ctypes binding of libsre (include/sre.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts
torch tensors / numpy arrays to pointers, sizes and streams and maps status
codes to exceptions.  It never falls back to a CPU path: if libsre.so is
missing or no CUDA device is present the first call raises.

Names follow the C ABI: ``Plan.m2`` <-> ``sre_m2``, ``Plan.m2_async`` <->
``sre_m2_async``, ``Plan.m2_host`` <-> ``sre_m2_host``, ``Plan.sum4_range`` <->
``sre_sum4_range``, ``Plan.m2_batched`` <-> ``sre_m2_batched``, ``Server`` <->
``sre_server_*``.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "SreError", "Plan", "Server", "m2", "m2_batched", "library_path", "load_library",
    "selftest_wait_timeout",
    "MODES", "DTYPES", "STATUS", "MAX_QUBITS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsre.so")
_lock = threading.Lock()
_lib = None

MAX_QUBITS = 24
DTYPES = {"c64": 0, "c128": 1}
MODES = {"fp32": 0, "bf16_split": 1, "fp16_split": 2, "fp64": 4, "auto": -1}
STATUS = {
    0: "SRE_OK", 1: "SRE_EINVAL", 2: "SRE_EALIGN", 3: "SRE_EZERO", 4: "SRE_ENONFINITE",
    5: "SRE_ENOMEM", 6: "SRE_EBUSY", 7: "SRE_ETIMEDOUT", 8: "SRE_ECUDA", 9: "SRE_ENOTFOUND",
    10: "SRE_EUNSUPPORTED",
}

_vp = ctypes.c_void_p
_i = ctypes.c_int
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)


class SreError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        name = STATUS.get(self.status, str(status))
        msg = _lib.sre_status_str(self.status).decode() if _lib else name
        extra = ""
        if self.status == 8 and _lib is not None:
            extra = " [" + _lib.sre_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {name}: {msg}{extra}")


class Tuning(ctypes.Structure):
    _fields_ = [("x_batch_log", ctypes.c_int), ("ring_slots", ctypes.c_int), ("lag", ctypes.c_int),
                ("pass2_tiles_log", ctypes.c_int), ("pass1_blocks_log", ctypes.c_int),
                ("pass1_staged", ctypes.c_int), ("pass2_staged", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_int),
                ("max_queue", ctypes.c_int), ("max_N", ctypes.c_int), ("mode", ctypes.c_int),
                ("wait_limit_ns", ctypes.c_uint64), ("device", ctypes.c_int),
                ("slot_scratch_bytes", ctypes.c_uint64), ("chunk_terms", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("inflight", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("p50_latency_ms", ctypes.c_double),
                ("p99_latency_ms", ctypes.c_double), ("mean_latency_ms", ctypes.c_double),
                ("states_per_s", ctypes.c_double), ("pauli_terms_per_s", ctypes.c_double),
                ("resident_bytes", ctypes.c_uint64), ("peak_resident_bytes", ctypes.c_uint64)]


def library_path() -> str:
    return _LIB_PATH


def _declare(lib):
    S = ctypes.c_int  # sre_status_t
    sig = {
        "sre_status_str": (ctypes.c_char_p, [_i]),
        "sre_last_cuda_error": (ctypes.c_char_p, []),
        "sre_version": (_i, []),
        "sre_plan_create": (S, [_i, _i, ctypes.POINTER(_vp)]),
        "sre_plan_set_mode": (S, [_vp, _i]),
        "sre_plan_get_mode": (S, [_vp, ctypes.POINTER(_i)]),
        "sre_plan_destroy": (S, [_vp]),
        "sre_plan_set_profiling": (S, [_vp, _i]),
        "sre_plan_last_kernel_ms": (S, [_vp, _dp, ctypes.POINTER(ctypes.c_char_p)]),
        "sre_plan_launch_count": (S, [_vp, ctypes.POINTER(_u64)]),
        "sre_plan_set_tuning": (S, [_vp, ctypes.POINTER(Tuning)]),
        "sre_plan_get_tuning": (S, [_vp, _i, ctypes.POINTER(Tuning)]),
        "sre_plan_autotune": (S, [_vp, _i, _vp, ctypes.POINTER(Tuning), _dp]),
        "sre_m2": (S, [_vp, _vp, _i, _vp, _dp]),
        "sre_m2_async": (S, [_vp, _vp, _i, _vp, _vp]),
        "sre_m2_host": (S, [_vp, _vp, _i, _vp, _dp]),
        "sre_sum4_range": (S, [_vp, _vp, _i, _u64, _u64, _vp, _vp, _vp]),
        "sre_m_alpha": (S, [_vp, _vp, _i, _i, _vp, _dp]),
        "sre_brickwork_m2_series": (S, [_vp, _i, _i, _i, _vp, _vp, _vp, _vp]),
        "sre_tfim_m2_series": (S, [_vp, _i, _i, _i, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _vp, _vp, _vp]),
        "sre_sum_pow_range": (S, [_vp, _vp, _i, _i, _u64, _u64, _vp, _vp, _vp]),
        "sre_m2_batched": (S, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i), _i, _vp, _vp]),
        "sre_selftest_wait_timeout": (S, [_u64, _vp]),
        "sre_m_alpha_from_sums": (S, [_vp, _vp, _i, _i, _vp, _vp]),
        "sre_server_cfg_default": (None, [ctypes.POINTER(ServerCfg)]),
        "sre_server_create": (S, [ctypes.POINTER(ServerCfg), ctypes.POINTER(_vp)]),
        "sre_server_submit": (S, [_vp, _vp, _i, _i, _i, ctypes.POINTER(_u64)]),
        "sre_server_set_tuning": (S, [_vp, _i, ctypes.POINTER(Tuning)]),
        "sre_server_poll": (S, [_vp, _u64, ctypes.POINTER(_i), _dp]),
        "sre_server_wait": (S, [_vp, _u64, ctypes.c_double, _dp]),
        "sre_server_stats": (S, [_vp, ctypes.POINTER(ServerStats)]),
        "sre_server_destroy": (S, [_vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load_library(build_if_missing: bool = True):
    """Load libsre.so (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH) and build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libsre.so not found at {_LIB_PATH}; run "
                               "`python -m paper_2512_24685_gb300.build`")
        _lib = _declare(ctypes.CDLL(_LIB_PATH))
        return _lib


def _check(status: int, where: str):
    if status != 0:
        raise SreError(status, where)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libsre needs a CUDA device; none is available")
    return torch


def _stream_handle(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_of(t) -> str:
    torch = _torch()
    if t.dtype == torch.complex64:
        return "c64"
    if t.dtype == torch.complex128:
        return "c128"
    raise TypeError(f"state must be complex64 or complex128, got {t.dtype}")


def _n_of(numel: int) -> int:
    N = int(numel).bit_length() - 1
    if numel < 2 or (1 << N) != numel:
        raise ValueError(f"state length {numel} is not 2^N with N >= 1")
    return N


def _check_state(t):
    if not t.is_cuda:
        raise ValueError("state must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("state must be contiguous")
    return _n_of(t.numel())


class Plan:
    """sre_plan_t: device workspace for states of up to N qubits of one dtype."""

    def __init__(self, N: int, dtype: str = "c64", mode: str | None = None):
        lib = load_library()
        _torch()
        self.N = int(N)
        self.dtype = dtype
        h = ctypes.c_void_p()
        _check(lib.sre_plan_create(self.N, DTYPES[dtype], ctypes.byref(h)), "sre_plan_create")
        self._h = h
        if mode is not None:
            self.set_mode(mode)

    def set_mode(self, mode: str):
        _check(load_library().sre_plan_set_mode(self._h, MODES[mode]), "sre_plan_set_mode")

    @property
    def mode(self) -> str:
        m = ctypes.c_int()
        _check(load_library().sre_plan_get_mode(self._h, ctypes.byref(m)), "sre_plan_get_mode")
        return {v: k for k, v in MODES.items()}[m.value]

    def set_profiling(self, enable: bool = True):
        _check(load_library().sre_plan_set_profiling(self._h, int(bool(enable))),
               "sre_plan_set_profiling")

    def last_kernel_ms(self):
        """(milliseconds, kernel name) of the last evaluation's main kernel."""
        ms, name = ctypes.c_double(), ctypes.c_char_p()
        _check(load_library().sre_plan_last_kernel_ms(self._h, ctypes.byref(ms), ctypes.byref(name)),
               "sre_plan_last_kernel_ms")
        return ms.value, (name.value or b"").decode()

    def set_tuning(self, x_batch_log=-1, ring_slots=-1, lag=-1, pass2_tiles_log=-1,
                   pass1_blocks_log=-1, pass1_staged=-1, pass2_staged=-1):
        """sre_plan_set_tuning: override two-pass fields (-1 = library choice)."""
        t = Tuning(int(x_batch_log), int(ring_slots), int(lag), int(pass2_tiles_log),
                   int(pass1_blocks_log), int(pass1_staged), int(pass2_staged))
        _check(load_library().sre_plan_set_tuning(self._h, ctypes.byref(t)), "sre_plan_set_tuning")

    def get_tuning(self, N: int) -> dict:
        t = Tuning()
        _check(load_library().sre_plan_get_tuning(self._h, int(N), ctypes.byref(t)), "sre_plan_get_tuning")
        return t.as_dict()

    def autotune(self, N: int | None = None, stream=None):
        """sre_plan_autotune: (best tuning dict, ms on the timing slice)."""
        t, ms = Tuning(), ctypes.c_double()
        _check(load_library().sre_plan_autotune(self._h, int(self.N if N is None else N),
                                                _stream_handle(stream), ctypes.byref(t),
                                                ctypes.byref(ms)), "sre_plan_autotune")
        return t.as_dict(), ms.value

    def launch_count(self) -> int:
        c = ctypes.c_uint64()
        _check(load_library().sre_plan_launch_count(self._h, ctypes.byref(c)), "sre_plan_launch_count")
        return c.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().sre_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _state(self, t):
        N = _check_state(t)
        if _dtype_of(t) != self.dtype:
            raise TypeError(f"plan dtype {self.dtype} != state dtype {_dtype_of(t)}")
        return N

    def m2(self, t, stream=None) -> float:
        """sre_m2: synchronous M2 of a device state."""
        N = self._state(t)
        out = ctypes.c_double()
        _check(load_library().sre_m2(self._h, ctypes.c_void_p(t.data_ptr()), N,
                                     _stream_handle(stream), ctypes.byref(out)), "sre_m2")
        return out.value

    def m2_async(self, t, out, stream=None):
        """sre_m2_async: writes M2 into the 1-element float64 CUDA tensor `out`."""
        N = self._state(t)
        torch = _torch()
        if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 1:
            raise ValueError("out must be a float64 CUDA tensor")
        _check(load_library().sre_m2_async(self._h, ctypes.c_void_p(t.data_ptr()), N,
                                           _stream_handle(stream), ctypes.c_void_p(out.data_ptr())),
               "sre_m2_async")
        return out

    def m2_host(self, h, stream=None) -> float:
        """sre_m2_host: M2 of a HOST buffer (torch CPU tensor, pinned for an
        asynchronous copy, or a numpy array); the copy runs inside the call."""
        import numpy as np
        if isinstance(h, np.ndarray):
            arr = np.ascontiguousarray(h)
            want = np.complex64 if self.dtype == "c64" else np.complex128
            if arr.dtype != want:
                raise TypeError(f"host state must be {want}")
            ptr, n = arr.ctypes.data, arr.size
            keep = arr
        else:
            if h.is_cuda or not h.is_contiguous():
                raise ValueError("host state must be a contiguous CPU tensor")
            if _dtype_of(h) != self.dtype:
                raise TypeError("dtype mismatch")
            ptr, n, keep = h.data_ptr(), h.numel(), h
        N = _n_of(n)
        out = ctypes.c_double()
        _check(load_library().sre_m2_host(self._h, ctypes.c_void_p(ptr), N, _stream_handle(stream),
                                          ctypes.byref(out)), "sre_m2_host")
        del keep
        return out.value

    def sum4_range(self, t, x_begin: int, x_end: int, per_x: bool = False, stream=None):
        """sre_sum4_range: (S over shifts [x_begin, x_end), n2[, per-shift sums])
        as CUDA float64 tensors (asynchronous on `stream`)."""
        torch = _torch()
        N = self._state(t)
        out = torch.empty(2, dtype=torch.float64, device=t.device)
        px = torch.empty(int(x_end) - int(x_begin), dtype=torch.float64, device=t.device) if per_x else None
        _check(load_library().sre_sum4_range(
            self._h, ctypes.c_void_p(t.data_ptr()), N, int(x_begin), int(x_end), _stream_handle(stream),
            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(px.data_ptr()) if per_x else None),
            "sre_sum4_range")
        return (out, px) if per_x else out

    def m_alpha(self, t, alpha: int, stream=None) -> float:
        """sre_m_alpha: stabilizer Renyi entropy of integer order alpha
        (Eq. (sre)) of a device state (synchronous)."""
        N = self._state(t)
        out = ctypes.c_double()
        _check(load_library().sre_m_alpha(self._h, ctypes.c_void_p(t.data_ptr()), N, int(alpha),
                                          _stream_handle(stream), ctypes.byref(out)), "sre_m_alpha")
        return out.value

    def sum_pow_range(self, t, alpha: int, x_begin: int, x_end: int, per_x: bool = False, stream=None):
        """sre_sum_pow_range: (S_alpha over shifts [x_begin, x_end), n2[,
        per-shift sums]) as CUDA float64 tensors (asynchronous on `stream`)."""
        torch = _torch()
        N = self._state(t)
        out = torch.empty(2, dtype=torch.float64, device=t.device)
        px = torch.empty(int(x_end) - int(x_begin), dtype=torch.float64, device=t.device) if per_x else None
        _check(load_library().sre_sum_pow_range(
            self._h, ctypes.c_void_p(t.data_ptr()), N, int(alpha), int(x_begin), int(x_end),
            _stream_handle(stream), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(px.data_ptr()) if per_x else None), "sre_sum_pow_range")
        return (out, px) if per_x else out

    def brickwork_m2_series(self, gates, states=None, stream=None):
        """sre_brickwork_m2_series: M2 after every step of brickwork circuit
        dynamics evolved on the device.  gates: complex128 CUDA tensor of
        shape (T, S, N - 1, 4, 4) (even bonds then odd bonds per step);
        states: optional complex128 CUDA tensor (S, 2^N) that receives the
        final states.  Returns (M2 as a (T, S) float64 CUDA tensor, states)."""
        torch = _torch()
        T, S, nb = int(gates.shape[0]), int(gates.shape[1]), int(gates.shape[2])
        N = nb + 1
        if gates.dtype != torch.complex128 or tuple(gates.shape[3:]) != (4, 4) or not gates.is_contiguous():
            raise ValueError("gates must be a contiguous complex128 tensor of shape (T, S, N-1, 4, 4)")
        if states is None:
            states = torch.empty((S, 1 << N), dtype=torch.complex128, device=gates.device)
        out = torch.empty((T, S), dtype=torch.float64, device=gates.device)
        _check(load_library().sre_brickwork_m2_series(
            self._h, N, S, T, ctypes.c_void_p(gates.data_ptr()), ctypes.c_void_p(states.data_ptr()),
            _stream_handle(stream), ctypes.c_void_p(out.data_ptr())), "sre_brickwork_m2_series")
        return out, states

    def tfim_m2_series(self, states, T: int, dt: float = 0.2, J: float = 1.0, hx: float = 1.5,
                       hz: float = 1.5, stream=None):
        """sre_tfim_m2_series: M2 after each of T steps exp(-i H dt) of the
        TFIM with longitudinal field, evolved on the device.  states: complex128
        CUDA tensor (S, 2^N) of initial states, overwritten by the states at
        time T dt.  Returns M2 as a (T, S) float64 CUDA tensor."""
        torch = _torch()
        if states.dtype != torch.complex128 or states.dim() != 2 or not states.is_contiguous():
            raise ValueError("states must be a contiguous complex128 tensor of shape (S, 2^N)")
        S = int(states.shape[0])
        N = _n_of(int(states.shape[1]))
        out = torch.empty((int(T), S), dtype=torch.float64, device=states.device)
        _check(load_library().sre_tfim_m2_series(
            self._h, N, S, int(T), float(dt), float(J), float(hx), float(hz),
            ctypes.c_void_p(states.data_ptr()), _stream_handle(stream), ctypes.c_void_p(out.data_ptr())),
            "sre_tfim_m2_series")
        return out

    def m2_batched(self, states, out=None, stream=None):
        """sre_m2_batched: M2 of many device states of uneven N (float64 CUDA tensor)."""
        torch = _torch()
        states = list(states)
        n = len(states)
        Ns = (ctypes.c_int * n)(*[self._state(s) for s in states])
        ptrs = (ctypes.c_void_p * n)(*[s.data_ptr() for s in states])
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=states[0].device)
        _check(load_library().sre_m2_batched(self._h, ptrs, Ns, n, _stream_handle(stream),
                                             ctypes.c_void_p(out.data_ptr())), "sre_m2_batched")
        return out


def m_alpha_from_sums(S, n2, N: int, alpha: int = 2, stream=None):
    """sre_m_alpha_from_sums: M_alpha (M2 at alpha = 2) from device scalars
    S_alpha and n2 (CUDA float64 tensors of one element); returns a CUDA
    float64 tensor of one element, computed on `stream` (default: torch's
    current stream)."""
    torch = _torch()
    for t in (S, n2):
        if not (t.is_cuda and t.dtype == torch.float64 and t.numel() == 1):
            raise ValueError("S and n2 must be one-element CUDA float64 tensors")
    out = torch.empty(1, dtype=torch.float64, device=S.device)
    _check(load_library().sre_m_alpha_from_sums(
        ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(n2.data_ptr()), int(N), int(alpha),
        _stream_handle(stream), ctypes.c_void_p(out.data_ptr())), "sre_m_alpha_from_sums")
    return out


def selftest_wait_timeout(wait_ns: int = 200_000_000, stream=None) -> int:
    """sre_selftest_wait_timeout: status of a device wait that nothing satisfies
    (SRE_ETIMEDOUT = 7 when the bound works)."""
    return int(load_library().sre_selftest_wait_timeout(int(wait_ns), _stream_handle(stream)))


_plans: dict = {}


def m2(t, mode: str | None = None) -> float:
    """M2 of one complex64 / complex128 CUDA state (plan cached per N, dtype, mode)."""
    N = _check_state(t)
    key = (N, _dtype_of(t), mode, t.device.index)
    p = _plans.get(key)
    if p is None:
        p = _plans[key] = Plan(N, _dtype_of(t), mode)
    return p.m2(t)


def m2_batched(states, mode: str | None = None):
    states = list(states)
    Nmax = max(_check_state(s) for s in states)
    dt = _dtype_of(states[0])
    with Plan(Nmax, dt, mode) as p:
        out = p.m2_batched(states)
        _torch().cuda.current_stream().synchronize()
        return out


class Server:
    """sre_server_t: continuous-batching M2 requests of mixed N."""

    def __init__(self, hbm_budget_bytes=None, max_inflight=None, max_queue=None, max_N=None,
                 mode: str | None = None, wait_limit_ns=None, device=None, slot_scratch_bytes=None,
                 chunk_terms=None):
        lib = load_library()
        _torch()
        cfg = ServerCfg()
        lib.sre_server_cfg_default(ctypes.byref(cfg))
        for k, v in (("hbm_budget_bytes", hbm_budget_bytes), ("max_inflight", max_inflight),
                     ("max_queue", max_queue), ("max_N", max_N), ("wait_limit_ns", wait_limit_ns),
                     ("device", device), ("slot_scratch_bytes", slot_scratch_bytes),
                     ("chunk_terms", chunk_terms)):
            if v is not None:
                setattr(cfg, k, int(v))
        if mode is not None:
            cfg.mode = MODES[mode]
        self.cfg = cfg
        h = ctypes.c_void_p()
        _check(lib.sre_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sre_server_create")
        self._h = h

    def set_tuning(self, N: int, tuning: dict):
        """sre_server_set_tuning: two-pass tuning (a dict as Plan.autotune
        returns; missing fields = library choice) for requests of N qubits."""
        t = Tuning(*[int(tuning.get(k, -1)) for k, _ in Tuning._fields_])
        _check(load_library().sre_server_set_tuning(self._h, int(N), ctypes.byref(t)), "sre_server_set_tuning")

    def submit(self, state) -> int:
        """Submit a state (CUDA tensor, CPU tensor or numpy array); returns a ticket.
        The server copies the state before returning."""
        import numpy as np
        lib = load_library()
        if isinstance(state, np.ndarray):
            arr = np.ascontiguousarray(state)
            dt = {np.dtype(np.complex64): 0, np.dtype(np.complex128): 1}[arr.dtype]
            ptr, n, on_dev = arr.ctypes.data, arr.size, 0
        else:
            dt = DTYPES[_dtype_of(state)]
            if not state.is_contiguous():
                raise ValueError("state must be contiguous")
            ptr, n, on_dev = state.data_ptr(), state.numel(), int(state.is_cuda)
        t = ctypes.c_uint64()
        _check(lib.sre_server_submit(self._h, ctypes.c_void_p(ptr), on_dev, _n_of(n), dt,
                                     ctypes.byref(t)), "sre_server_submit")
        return t.value

    def poll(self, ticket: int):
        """(done, m2) without blocking."""
        done, m = ctypes.c_int(), ctypes.c_double()
        _check(load_library().sre_server_poll(self._h, int(ticket), ctypes.byref(done), ctypes.byref(m)),
               "sre_server_poll")
        return bool(done.value), m.value

    def wait(self, ticket: int, timeout_ms: float = 60000.0) -> float:
        m = ctypes.c_double()
        _check(load_library().sre_server_wait(self._h, int(ticket), float(timeout_ms), ctypes.byref(m)),
               "sre_server_wait")
        return m.value

    def stats(self) -> dict:
        s = ServerStats()
        _check(load_library().sre_server_stats(self._h, ctypes.byref(s)), "sre_server_stats")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().sre_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
