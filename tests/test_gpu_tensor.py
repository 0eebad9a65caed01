"""Split-precision tensor-core modes (tcgen05 MMA with exact +-1 H_16 on
BF16 / FP16 hi-lo operands, FP32 accumulation in TMEM) against the FP64
oracle: |Delta M2| <= 1e-6, per-shift sums, and agreement with the FP32
CUDA-core path at the benchmark size."""
import numpy as np
import pytest

import oracle
from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu
MODES = ["bf16_split", "fp16_split"]


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


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("N", [13, 14, 16])
def test_split_modes_match_oracle(sre, torch_cuda, mode, N):
    for psi in (W.haar_state(N, 300 + N, np.complex64),
                W.product_state(N, 310 + N, np.complex64)[0],
                W.brickwork_state(N, 6, 320 + N, np.complex64)):
        with sre.Plan(N, "c64", mode) as p:
            got = p.m2(torch_cuda.from_numpy(psi).cuda())
        ref = oracle.m2(psi)
        assert abs(got - ref) <= 1e-6, (mode, N, got - ref)


@pytest.mark.parametrize("mode", MODES)
def test_split_mode_per_shift_sums(sre, torch_cuda, mode):
    N = 14
    psi = W.haar_state(N, 41, np.complex64)
    _, ref = oracle.sum4_xorfwht(psi, per_x=True)
    with sre.Plan(N, "c64", mode) as p:
        _, px = p.sum4_range(torch_cuda.from_numpy(psi).cuda(), 0, 1 << N, per_x=True)
        torch_cuda.cuda.synchronize()
    np.testing.assert_allclose(px.cpu().numpy(), ref, rtol=0, atol=1e-5 * ref.max())


@pytest.mark.parametrize("mode", MODES)
def test_split_mode_stabilizer_zero(sre, torch_cuda, mode):
    psi = W.stabilizer_state(15, 7).astype(np.complex64)
    with sre.Plan(15, "c64", mode) as p:
        assert abs(p.m2(torch_cuda.from_numpy(psi).cuda())) <= 1e-6


def test_split_modes_agree_with_fp32_at_n20(sre, torch_cuda):
    """Benchmark size: the split-precision forms agree with the FP32 path
    (itself pinned to the oracle on sampled shifts) within 1e-6."""
    N = 20
    psi = torch_cuda.from_numpy(W.haar_state(N, W.config_seed(2, 0), np.complex64)).cuda()
    vals = {}
    for mode in ["fp32"] + MODES:
        with sre.Plan(N, "c64", mode) as p:
            vals[mode] = p.m2(psi)
    for mode in MODES:
        assert abs(vals[mode] - vals["fp32"]) <= 1e-6, vals
        # a different arithmetic ran: the hi/lo MMA does not reproduce the
        # FP32 butterflies bit for bit
        assert vals[mode] != vals["fp32"], vals
