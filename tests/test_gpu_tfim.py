"""Hamiltonian quench dynamics (Example 1) evolved on the device with M2
after every step, against scipy's expm_multiply evolution of the same
initial states and the FP64 oracle.  Tolerances: states within 1e-10 of the
reference (FP64 Chebyshev vs Krylov-type expm_multiply), |Delta M2| <= 1e-6
(FP32 M2) or 1e-9 (FP64 M2, limited by the reference evolution)."""
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


def initial_states(N, S, seed0=500):
    return np.stack([W.product_state(N, seed0 + s)[0] for s in range(S)])


@pytest.mark.parametrize("N,S,T,dt,mode,tol", [
    (8, 3, 4, 0.2, "fp32", 1e-6),
    (7, 2, 3, 0.5, "fp64", 1e-9),
    (13, 2, 2, 0.2, "fp32", 1e-6),
])
def test_series_matches_expm_multiply_and_oracle(sre, torch_cuda, N, S, T, dt, mode, tol):
    torch = torch_cuda
    psi0 = initial_states(N, S)
    refs = [oracle.tfim_evolve(psi0[s], dt, T) for s in range(S)]
    states = torch.from_numpy(psi0.copy()).cuda()
    with sre.Plan(N, "c128", mode) as p:
        m2 = p.tfim_m2_series(states, T, dt).cpu().numpy()
    final = states.cpu().numpy()
    for s in range(S):
        assert np.max(np.abs(final[s] - refs[s][-1])) <= 1e-10
        for t in range(T):
            assert abs(m2[t, s] - oracle.m2(refs[s][t])) <= tol, (t, s)


def test_other_couplings_and_single_qubit(sre, torch_cuda):
    """Non-default J, hx, hz and N = 1 (no bonds) against expm_multiply."""
    torch = torch_cuda
    for N, J, hx, hz in ((6, -0.7, 0.3, 2.1), (1, 1.0, 1.5, 1.5)):
        psi0 = initial_states(N, 2, 77)
        states = torch.from_numpy(psi0.copy()).cuda()
        with sre.Plan(max(N, 1), "c128", "fp64") as p:
            p.tfim_m2_series(states, 3, 0.3, J, hx, hz)
        final = states.cpu().numpy()
        for s in range(2):
            ref = oracle.tfim_evolve(psi0[s], 0.3, 3, J, hx, hz)[-1]
            assert np.max(np.abs(final[s] - ref)) <= 1e-10


def test_norm_and_energy_conserved(sre, torch_cuda):
    """N = 12, 20 steps of dt = 0.2: norm and <H> of every realization stay
    at their initial values; M2 starts below the Haar value and grows."""
    torch = torch_cuda
    N, S, T = 12, 4, 20
    psi0 = initial_states(N, S, 900)
    H = oracle.tfim_hamiltonian(N)
    states = torch.from_numpy(psi0.copy()).cuda()
    with sre.Plan(N, "c128") as p:
        m2 = p.tfim_m2_series(states, T, 0.2).cpu().numpy()
    final = states.cpu().numpy()
    for s in range(S):
        e0 = np.vdot(psi0[s], H @ psi0[s]).real
        assert abs(np.linalg.norm(final[s]) - 1) <= 1e-11
        assert abs(np.vdot(final[s], H @ final[s]).real - e0) <= 1e-9
    haar = np.log2(2.0 ** N + 3) - 2
    assert np.all(np.isfinite(m2))
    assert m2[-1].mean() > m2[0].mean()
    assert m2[-1].mean() < haar + 0.05


def test_rejects_bad_arguments(sre, torch_cuda):
    torch = torch_cuda
    states = torch.from_numpy(initial_states(6, 1)).cuda()
    with sre.Plan(6, "c128") as p:
        for kw in ({"dt": -0.1}, {"dt": 1e6}):
            with pytest.raises(sre.SreError) as ei:
                p.tfim_m2_series(states, 1, **kw)
            assert ei.value.status == 1
    with sre.Plan(6, "c64") as p:
        with pytest.raises(sre.SreError):
            p.tfim_m2_series(states, 1)
