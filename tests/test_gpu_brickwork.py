"""Brickwork random-circuit dynamics evolved on the device (Example 2) with
M2 after every step, against the same gates applied by numpy and the FP64
oracle.  Tolerances: |Delta M2| <= 1e-6 (FP32 M2), 1e-10 (FP64 M2); final
states within 1e-12 of the numpy evolution (both FP64)."""
import math

import numpy as np
import pytest

import oracle
from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def sre():
    from paper_2512_24685_gb300 import binding
    binding.load_library()
    return binding


def numpy_series(gates):
    """States after every step by W.apply_2q with the same gates."""
    T, S, nb = gates.shape[:3]
    N = nb + 1
    out = []
    psis = [W.basis_state(N) for _ in range(S)]
    for t in range(T):
        for s in range(S):
            for b in range(nb):
                q = 2 * b if b < N // 2 else 2 * (b - N // 2) + 1
                psis[s] = W.apply_2q(psis[s], N, q, gates[t, s, b])
        out.append([p.copy() for p in psis])
    return out


@pytest.mark.parametrize("N,S,T,mode,tol", [
    (10, 3, 5, "fp32", 1e-6),
    (9, 2, 4, "fp64", 1e-10),
    (14, 3, 3, "fp32", 1e-6),
])
def test_series_matches_numpy_and_oracle(sre, torch_cuda, N, S, T, mode, tol):
    torch = torch_cuda
    gates = W.brickwork_gate_tensor(N, S, T)
    ref_states = numpy_series(gates)
    with sre.Plan(N, "c128", mode) as p:
        m2, states = p.brickwork_m2_series(torch.from_numpy(gates).cuda())
        torch.cuda.synchronize()
    m2 = m2.cpu().numpy()
    states = states.cpu().numpy()
    for s in range(S):
        assert np.max(np.abs(states[s] - ref_states[-1][s])) <= 1e-12
    for t in range(T):
        for s in range(S):
            assert abs(m2[t, s] - oracle.m2(ref_states[t][s])) <= tol, (t, s)


def test_same_gates_as_brickwork_state(sre, torch_cuda):
    """The gate tensor reproduces W.brickwork_state (depth T) exactly."""
    torch = torch_cuda
    N, S, T = 8, 2, 3
    gates = W.brickwork_gate_tensor(N, S, T)
    with sre.Plan(N, "c128") as p:
        _, states = p.brickwork_m2_series(torch.from_numpy(gates).cuda())
    for s in range(S):
        ref = W.brickwork_state(N, T, W.config_seed(4, s))
        assert np.max(np.abs(states[s].cpu().numpy() - ref)) <= 1e-12


def test_approach_to_haar_value(sre, torch_cuda):
    """N = 12: M2 starts near 0 and saturates near log2(2^N + 3) - 2."""
    torch = torch_cuda
    N, S, T = 12, 8, 24
    gates = W.brickwork_gate_tensor(N, S, T)
    with sre.Plan(N, "c128") as p:
        m2, _ = p.brickwork_m2_series(torch.from_numpy(gates).cuda())
    m2 = m2.cpu().numpy()
    haar = math.log2(2 ** N + 3) - 2
    assert np.all(np.isfinite(m2))
    assert m2[0].mean() < haar - 2.0
    assert abs(m2[-1].mean() - haar) < 0.1


def test_rejects_complex64_plan(sre, torch_cuda):
    torch = torch_cuda
    gates = torch.from_numpy(W.brickwork_gate_tensor(6, 1, 1)).cuda()
    with sre.Plan(6, "c64") as p:
        with pytest.raises(sre.SreError) as ei:
            p.brickwork_m2_series(gates)
        assert ei.value.status == 1
