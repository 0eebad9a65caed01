"""Split-precision tensor-core modes (tcgen05 Hadamard MMAs on fixed-point
BF16 / FP16 hi-lo pieces, both passes of the halved shifts for N = 16-20)
against the FP64 oracle: |Delta M2| <= 1e-6, per-shift sums, shift ranges
with partial chunks, and agreement with the FP32 CUDA-core path at the
benchmark size.  Below N = 16 the modes run the FP32 kernels."""
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


_REF = {}


def ref_m2(key, psi):
    """oracle.m2 once per state (the tests share states across modes)."""
    if key not in _REF:
        _REF[key] = oracle.m2(psi)
    return _REF[key]


def families(N, seed):
    """The four state families of the N = 16 workload mix."""
    return {
        "haar": W.haar_state(N, seed, np.complex64),
        "product": W.product_state(N, seed + 1, np.complex64)[0],
        "stabilizer": W.stabilizer_state(N, seed + 2).astype(np.complex64),
        "brickwork": W.brickwork_state(N, 8, seed + 3, np.complex64),
    }


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
def test_split_modes_n16_family_mix(sre, torch_cuda, mode):
    """All four families of the N = 16 workload mix through the tensor-core
    kernel (h2 = 3: pass 2 stacks 16 column blocks along K)."""
    for name, psi in families(16, 1600).items():
        with sre.Plan(16, "c64", mode) as p:
            got = p.m2(torch_cuda.from_numpy(psi).cuda())
        ref = ref_m2(("fam", name), psi)
        assert abs(got - ref) <= 1e-6, (mode, name, got - ref)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scale", [1e-3, 37.0])
def test_split_modes_scale_invariance(sre, torch_cuda, mode, scale):
    """Unnormalised states: the fixed-point scales follow the amplitudes, and
    M2 does not move (S scales as n2^4)."""
    psi = W.haar_state(17, 1717, np.complex64)
    ref = ref_m2(("haar17",), psi)
    t = torch_cuda.from_numpy((psi * np.float32(scale)).astype(np.complex64)).cuda()
    with sre.Plan(17, "c64", mode) as p:
        got = p.m2(t)
    assert abs(got - ref) <= 1e-6, (mode, scale, got - ref)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("N", [17, 18])
def test_split_mode_per_shift_sums_tma_pass2(sre, torch_cuda, mode, N):
    """Per-shift sums of halved shifts at N = 17 and 18 (pass-2 tiles of 2^4
    and 2^5 rows copied by TMA) against the oracle, on a range whose ends
    cut chunks, plus the shift just below the first halved one."""
    psi = W.haar_state(N, 410 + N, np.complex64)
    t = torch_cuda.from_numpy(psi).cuda()
    xb, xe = 4093, 4093 + 203
    _, ref = oracle.sum4_xorfwht(psi, xb, xe, per_x=True)
    with sre.Plan(N, "c64", mode) as p:
        _, px = p.sum4_range(t, xb, xe, per_x=True)
        torch_cuda.cuda.synchronize()
    px = px.cpu().numpy()
    tol = 3e-5 if mode == "bf16_split" else 1e-6
    np.testing.assert_allclose(px, ref, rtol=tol, atol=0)


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
    for N in (15, 17):
        psi = W.stabilizer_state(N, 7).astype(np.complex64)
        with sre.Plan(N, "c64", mode) as p:
            assert abs(p.m2(torch_cuda.from_numpy(psi).cuda())) <= 1e-6


def test_split_modes_agree_with_fp32_at_n20(sre, torch_cuda):
    """Benchmark size: the split-precision forms agree with the FP32 path
    within 1e-6 (each is pinned to the oracle's value in test_gpu_n20.py)."""
    N = 20
    psi = torch_cuda.from_numpy(W.haar_state(N, W.config_seed(2, 0), np.complex64)).cuda()
    vals = {}
    for mode in ["fp32"] + MODES:
        with sre.Plan(N, "c64", mode) as p:
            vals[mode] = p.m2(psi)
    for mode in MODES:
        assert abs(vals[mode] - vals["fp32"]) <= 1e-6, vals
        # a different arithmetic ran: the MMA stages do not reproduce the
        # FP32 butterflies bit for bit
        assert vals[mode] != vals["fp32"], vals
