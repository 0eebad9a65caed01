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
