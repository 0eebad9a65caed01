"""Shift-range sharding finished on the device (sre_m_alpha_from_sums).

* m2_sharded at world size 1 (no process group) reproduces the plan's M2 and
  the oracle's;
* shard partials from sre_sum4_range added on the host and finished by
  sre_m_alpha_from_sums equal the oracle's M2 (Eq. (final1)) for several
  world sizes; at alpha = 3 the call matches the oracle's M_alpha (Eq. (sre));
* zero, negative and non-finite sums give NaN; bad arguments SRE_EINVAL.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_24685_gb300 import shard
from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available()
    return torch


@pytest.fixture(scope="module")
def sre():
    from paper_2512_24685_gb300 import binding
    binding.load_library()
    return binding


def test_m2_sharded_single_rank(sre, torch_cuda):
    N = 14
    psi = W.haar_state(N, 31, np.complex64)
    t = torch_cuda.from_numpy(psi).cuda()
    with sre.Plan(N, "c64") as p:
        got = shard.m2_sharded(t, N, p)
        whole = p.m2(t)
    assert abs(got - whole) <= 1e-9
    assert abs(got - oracle.m2(psi)) <= 1e-6


@pytest.mark.parametrize("world", [2, 3, 8])
def test_shard_partials_finished_on_device(sre, torch_cuda, world):
    torch = torch_cuda
    N = 13
    psi = W.brickwork_state(N, 4, 40 + world, np.complex128)
    t = torch.from_numpy(psi).cuda()
    with sre.Plan(N, "c128", "fp64") as p:
        parts = [p.sum4_range(t, *shard.shard_range(1 << N, r, world)) for r in range(world)]
        S = sum(x[0:1] for x in parts)
        m = sre.m_alpha_from_sums(S, parts[0][1:2], N).item()
    assert abs(m - oracle.m2(psi)) <= 1e-10


def test_alpha3_from_sums(sre, torch_cuda):
    torch = torch_cuda
    N = 10
    psi = W.haar_state(N, 8, np.complex128)
    S3 = oracle.sum_pow_xorfwht(psi, 3)
    n2 = oracle.norm2(psi)
    dS = torch.tensor([S3], dtype=torch.float64, device="cuda")
    dn = torch.tensor([n2], dtype=torch.float64, device="cuda")
    got = sre.m_alpha_from_sums(dS, dn, N, 3).item()
    assert abs(got - oracle.malpha_from_sum(S3, n2, N, 3)) <= 1e-12


def test_degenerate_sums_and_errors(sre, torch_cuda):
    torch = torch_cuda
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    for bad in (0.0, -1.0, math.inf, math.nan):
        v = torch.tensor([bad], dtype=torch.float64, device="cuda")
        assert math.isnan(sre.m_alpha_from_sums(v, one, 4).item())
        assert math.isnan(sre.m_alpha_from_sums(one, v, 4).item())
    # a stabilizer-like value: S = d n2^4 gives M2 = 0
    S = torch.tensor([16.0], dtype=torch.float64, device="cuda")
    assert sre.m_alpha_from_sums(S, one, 4).item() == 0.0
    for N, alpha in ((0, 2), (25, 2), (4, 1), (4, 17)):
        with pytest.raises(sre.SreError) as e:
            sre.m_alpha_from_sums(one, one, N, alpha)
        assert e.value.status == 1  # SRE_EINVAL
