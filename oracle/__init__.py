"""FP64 CPU oracle for the second-order stabilizer Renyi entropy (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the product path (the
CUDA library ``libsre`` and ``paper_2512_24685_gb300``) never does.

It wraps ``sre_oracle.c`` (plain C, FP64, OpenMP) through ctypes:

* ``m2(psi, method)`` -- M2 = -log2(S / (d n2^4)) (Eq. (sre) at alpha = 2,
  base-2 log as in Algorithm 1);
* ``sum4_direct`` (O1) -- S from the definition: each Pauli expectation by
  Eq. (Pauli_expect), |.|^4 summed over all 4^N strings X^x Z^z;
* ``sum4_xorfwht`` (O2) -- S by Algorithm 1 (XOR-shifted product, unnormalised
  FWHT, sum of |.|^4);
* ``fwht``, ``pauli_table``, ``shift_transform``, ``norm2`` -- the pieces, for
  pinning tests.

complex64 inputs are widened exactly to complex128, so the oracle evaluates
the state that is actually stored.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sre_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile sre_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.sre_oracle_norm2.restype = ctypes.c_double
        lib.sre_oracle_norm2.argtypes = [_dp, ctypes.c_int]
        lib.sre_oracle_pauli_expectation.restype = None
        lib.sre_oracle_pauli_expectation.argtypes = [
            _dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _dp, _dp]
        lib.sre_oracle_pauli_table_direct.restype = None
        lib.sre_oracle_pauli_table_direct.argtypes = [_dp, ctypes.c_int, _dp]
        lib.sre_oracle_sum4_direct.restype = ctypes.c_double
        lib.sre_oracle_sum4_direct.argtypes = [_dp, ctypes.c_int, _dp]
        lib.sre_oracle_fwht.restype = None
        lib.sre_oracle_fwht.argtypes = [_dp, ctypes.c_int]
        lib.sre_oracle_shift_transform.restype = None
        lib.sre_oracle_shift_transform.argtypes = [_dp, ctypes.c_int, ctypes.c_uint64, _dp]
        lib.sre_oracle_sum4_xorfwht_range.restype = ctypes.c_double
        lib.sre_oracle_sum4_xorfwht_range.argtypes = [
            _dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _dp]
        lib.sre_oracle_m2.restype = ctypes.c_double
        lib.sre_oracle_m2.argtypes = [_dp, ctypes.c_int, ctypes.c_int]
        lib.sre_oracle_sum_pow_direct.restype = ctypes.c_double
        lib.sre_oracle_sum_pow_direct.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp]
        lib.sre_oracle_sum_pow_xorfwht_range.restype = ctypes.c_double
        lib.sre_oracle_sum_pow_xorfwht_range.argtypes = [
            _dp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, _dp]
        lib.sre_oracle_malpha.restype = ctypes.c_double
        lib.sre_oracle_malpha.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.sre_oracle_num_threads.restype = ctypes.c_int
        lib.sre_oracle_set_threads.restype = None
        lib.sre_oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _as_c128(psi) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(np.asarray(psi).reshape(-1), dtype=np.complex128)
    n = a.size
    N = n.bit_length() - 1
    if n < 2 or (1 << N) != n:
        raise ValueError(f"state length {n} is not 2^N with N >= 1")
    return a, N


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return _load().sre_oracle_num_threads()


def set_threads(n: int) -> None:
    _load().sre_oracle_set_threads(int(n))


def norm2(psi) -> float:
    a, N = _as_c128(psi)
    return _load().sre_oracle_norm2(_ptr(a), N)


def pauli_expectation(psi, x: int, z: int) -> complex:
    """<psi| X^x Z^z |psi> by Eq. (Pauli_expect)."""
    a, N = _as_c128(psi)
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().sre_oracle_pauli_expectation(_ptr(a), N, x, z, ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def pauli_table(psi) -> np.ndarray:
    """(d, d) complex table A[x, z] = <psi|X^x Z^z|psi> by the direct sum."""
    a, N = _as_c128(psi)
    d = 1 << N
    out = np.empty(d * d, dtype=np.complex128)
    _load().sre_oracle_pauli_table_direct(_ptr(a), N, _ptr(out))
    return out.reshape(d, d)


def fwht(v) -> np.ndarray:
    """Unnormalised FWHT (copy) of a complex vector of length 2^N."""
    a, N = _as_c128(v)
    a = a.copy()
    _load().sre_oracle_fwht(_ptr(a), N)
    return a


def shift_transform(psi, x: int) -> np.ndarray:
    """FWHT_t( conj(psi[t^x]) psi[t] ) -- one iteration of Algorithm 1."""
    a, N = _as_c128(psi)
    out = np.empty_like(a)
    _load().sre_oracle_shift_transform(_ptr(a), N, x, _ptr(out))
    return out


def sum4_direct(psi, per_x: bool = False):
    """O1: S = sum_{x,z} |<psi|X^x Z^z|psi>|^4 from the definition (8^N)."""
    a, N = _as_c128(psi)
    px = np.empty(1 << N) if per_x else None
    s = _load().sre_oracle_sum4_direct(_ptr(a), N, _ptr(px) if per_x else None)
    return (s, px) if per_x else s


def sum4_xorfwht(psi, x_begin: int = 0, x_end: int | None = None, per_x: bool = False):
    """O2: S by Algorithm 1 over shifts [x_begin, x_end)."""
    a, N = _as_c128(psi)
    d = 1 << N
    xe = d if x_end is None else min(int(x_end), d)
    xb = int(x_begin)
    px = np.empty(max(xe - xb, 0)) if per_x else None
    s = _load().sre_oracle_sum4_xorfwht_range(_ptr(a), N, xb, xe,
                                              _ptr(px) if per_x else None)
    return (s, px) if per_x else s


def m2_from_sum(S: float, n2: float, N: int) -> float:
    """M2 = -log2(S / (d n2^4))."""
    return float(-np.log2(S / (2.0 ** N * n2 ** 4)))


def m2(psi, method: str = "auto") -> float:
    """M2 of the stored state. method: 'direct' (O1), 'xorfwht' (O2) or
    'auto' (O1 for N <= 6, O2 above)."""
    a, N = _as_c128(psi)
    if method == "auto":
        method = "direct" if N <= 6 else "xorfwht"
    code = {"direct": 0, "xorfwht": 1}[method]
    return _load().sre_oracle_m2(_ptr(a), N, code)


# ---- general integer Renyi order (Eq. (sre)) ------------------------------

def sum_pow_direct(psi, alpha: int, per_x: bool = False):
    """O1 for order alpha: S_alpha = sum_{x,z} |<psi|X^x Z^z|psi>|^(2 alpha)
    from the definition (8^N)."""
    a, N = _as_c128(psi)
    px = np.empty(1 << N) if per_x else None
    s = _load().sre_oracle_sum_pow_direct(_ptr(a), N, int(alpha), _ptr(px) if per_x else None)
    return (s, px) if per_x else s


def sum_pow_xorfwht(psi, alpha: int, x_begin: int = 0, x_end: int | None = None,
                    per_x: bool = False):
    """O2 for order alpha: S_alpha by Algorithm 1's loop over shifts
    [x_begin, x_end) with the exponent 2 alpha."""
    a, N = _as_c128(psi)
    d = 1 << N
    xe = d if x_end is None else min(int(x_end), d)
    xb = int(x_begin)
    px = np.empty(max(xe - xb, 0)) if per_x else None
    s = _load().sre_oracle_sum_pow_xorfwht_range(_ptr(a), N, int(alpha), xb, xe,
                                                 _ptr(px) if per_x else None)
    return (s, px) if per_x else s


def malpha_from_sum(S: float, n2: float, N: int, alpha: int) -> float:
    """M_alpha = log2(S_alpha / (d n2^(2 alpha))) / (1 - alpha)."""
    return float(np.log2(S / (2.0 ** N * n2 ** (2 * alpha))) / (1 - alpha))


def malpha(psi, alpha: int, method: str = "auto") -> float:
    """M_alpha of Eq. (sre) for integer alpha >= 2. method: 'direct' (O1),
    'xorfwht' (O2) or 'auto' (O1 for N <= 6, O2 above)."""
    a, N = _as_c128(psi)
    if method == "auto":
        method = "direct" if N <= 6 else "xorfwht"
    return _load().sre_oracle_malpha(_ptr(a), N, int(alpha), 0 if method == "direct" else 1)


# ---- TFIM with longitudinal field, Example 1 (Eq. (TFIM_LF_OBC)) ------------

def tfim_hamiltonian(N: int, J: float = 1.0, hx: float = 1.5, hz: float = 1.5):
    """Sparse H = -J sum_{i=0}^{N-2} Z_i Z_{i+1} - hx sum_i X_i - hz sum_i Z_i
    on an open chain, qubit i <-> bit i of the basis index, Z|0> = |0>."""
    import scipy.sparse as sp
    d = 1 << N
    t = np.arange(d, dtype=np.int64)
    s = 1 - 2 * ((t[:, None] >> np.arange(N)) & 1)  # Z eigenvalue of each qubit
    diag = -J * np.sum(s[:, :-1] * s[:, 1:], axis=1) - hz * np.sum(s, axis=1)
    rows = [t] + [t] * N
    cols = [t] + [t ^ (1 << i) for i in range(N)]
    vals = [diag.astype(np.float64)] + [np.full(d, -hx, dtype=np.float64)] * N
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(d, d))


def tfim_evolve(psi, dt: float, steps: int, J: float = 1.0, hx: float = 1.5, hz: float = 1.5):
    """States after each of `steps` steps of exp(-i H dt) applied to psi,
    by scipy.sparse.linalg.expm_multiply (the method the paper uses)."""
    from scipy.sparse.linalg import expm_multiply
    a = np.asarray(psi, dtype=np.complex128)
    N = a.size.bit_length() - 1
    H = tfim_hamiltonian(N, J, hx, hz)
    out = []
    for _ in range(steps):
        a = expm_multiply(-1j * dt * H, a)
        out.append(a.copy())
    return out
