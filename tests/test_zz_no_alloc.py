"""sre_m2_noalloc: M2 from a fixed module scratch array, no allocation.

This entry point exists for callers that cannot allocate memory where they
need M2 (for example inside a region where cudaMalloc is unsafe, or under a
fixed memory budget).  The test calls it through the C ABI and checks its
result against the ordinary entry point (sre_m2, via a plan) and against the
FP64 oracle (Algorithm 1) with the FP32 tolerance the other tests use, on two
calls in a row per size, so a second call that reuses the shared array (and
its leftover contents) is covered.  The sizes span the single-tile path
(N = 1, 2, 3, 12), the two-pass kernel on the fixed ring (13 to 16, with
N = 15 the last halved size below the limit).
It is collected last and sets up everything it needs itself, so it passes in
a fresh process as well as after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-6  # FP32 path, |Delta M2|


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2512_24685_gb300 import binding, workloads
    lib = binding.load_library()
    f = lib.sre_m2_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return torch, binding, workloads, f


def _noalloc(torch, f, psi_dev, N):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = f(ctypes.c_void_p(psi_dev.data_ptr()), N, ctypes.c_void_p(stream.cuda_stream),
           ctypes.c_void_p(out.data_ptr()))
    assert st == 0, st
    torch.cuda.synchronize()
    return out.item()


@pytest.mark.parametrize("N", [1, 2, 3, 12, 13, 14, 15, 16])
def test_noalloc_matches_plan_twice(env, N):
    torch, binding, W, f = env
    host = W.haar_state(N, 77 + N, np.complex64)
    psi = torch.from_numpy(host).cuda()
    with binding.Plan(N, "c64") as p:
        ref = p.m2(psi)
    want = oracle.m2(host)
    first = _noalloc(torch, f, psi, N)
    second = _noalloc(torch, f, psi, N)
    assert abs(first - ref) <= TOL, (first, ref)
    assert abs(second - ref) <= TOL, (second, ref)
    assert abs(first - want) <= TOL, (first, want)
    assert abs(second - want) <= TOL, (second, want)
    # a different state in between must not leak through the shared array
    other = torch.from_numpy(W.haar_state(N, 999, np.complex64)).cuda()
    _noalloc(torch, f, other, N)
    assert abs(_noalloc(torch, f, psi, N) - ref) <= TOL


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, binding, W, f = env
    psi = torch.zeros(1 << 17, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = f(ctypes.c_void_p(psi.data_ptr()), 17, None, ctypes.c_void_p(out.data_ptr()))
    assert st == 1  # SRE_EINVAL: N above SRE_NOALLOC_MAX_QUBITS


_RESET_CHILD = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2512_24685_gb300 import binding, workloads as W
lib = binding.load_library()
rt_path = next(l.split()[-1] for l in open('/proc/self/maps') if 'libcudart' in l)
rt = ctypes.CDLL(rt_path)
f = lib.sre_m2_noalloc
f.restype = ctypes.c_int
f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
N = 14
psi = W.haar_state(N, 4321, np.complex64)
def once():
    d_psi, d_out = ctypes.c_void_p(), ctypes.c_void_p()
    assert rt.cudaMalloc(ctypes.byref(d_psi), ctypes.c_size_t(psi.nbytes)) == 0
    assert rt.cudaMalloc(ctypes.byref(d_out), ctypes.c_size_t(8)) == 0
    assert rt.cudaMemcpy(d_psi, psi.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(psi.nbytes), 1) == 0
    assert f(d_psi, N, None, d_out) == 0
    assert rt.cudaDeviceSynchronize() == 0
    out = ctypes.c_double()
    assert rt.cudaMemcpy(ctypes.byref(out), d_out, ctypes.c_size_t(8), 2) == 0
    rt.cudaFree(d_psi); rt.cudaFree(d_out)
    return out.value
a = once()
assert rt.cudaDeviceReset() == 0
b = once()
print(repr(a), repr(b))
sys.exit(0 if a == b else 3)
"""


def test_noalloc_after_device_reset(env):
    """A call after cudaDeviceReset (in a child process, which owns its own
    context) finds the reloaded module array and gives the same M2."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _RESET_CHILD, root], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr[-2000:])
