"""GPU parity at general integer Renyi order alpha (Eq. (sre)): libsre's
sre_m_alpha / sre_sum_pow_range through the C ABI against the FP64 oracle on
the same seeded inputs.

Tolerances: |Delta M_alpha| <= 1e-6 for the FP32 and split-precision paths,
1e-10 for FP64; per-shift sums relative to the largest one, 1e-5 (FP32).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORDERS = (3, 4, 6)


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


def dev(torch, psi):
    return torch.from_numpy(np.ascontiguousarray(psi)).cuda()


@pytest.mark.parametrize("N", [3, 9, 12, 13, 14])
def test_m_alpha_matches_oracle(sre, torch_cuda, N):
    """Single-tile (N <= 12) and two-pass (N > 12) paths, normalised and
    unnormalised Haar states, orders 3, 4, 6."""
    for seed, scale in ((40 + N, 1.0), (41 + N, 0.37)):
        psi = (W.haar_state(N, seed) * scale).astype(np.complex64)
        with sre.Plan(N, "c64") as p:
            t = dev(torch_cuda, psi)
            for a in ORDERS:
                ref = oracle.malpha(psi, a)
                got = p.m_alpha(t, a)
                assert abs(got - ref) <= 1e-6, (N, a, got, ref)


@pytest.mark.parametrize("N", [10, 16])
def test_order_two_is_m2_bitwise(sre, torch_cuda, N):
    """alpha = 2 runs the M2 arithmetic unchanged."""
    psi = W.haar_state(N, 5, np.complex64)
    t = dev(torch_cuda, psi)
    with sre.Plan(N, "c64") as p:
        assert p.m_alpha(t, 2) == p.m2(t)


def test_fp64_mode(sre, torch_cuda):
    """FP64 path at orders 3 and 4 (N = 13, both passes)."""
    N = 13
    psi = W.haar_state(N, 77)
    t = dev(torch_cuda, psi)
    with sre.Plan(N, "c128", "fp64") as p:
        for a in (3, 4):
            assert abs(p.m_alpha(t, a) - oracle.malpha(psi, a)) <= 1e-10


@pytest.mark.parametrize("N", [13, 16])
def test_product_states_closed_form(sre, torch_cuda, N):
    """Random product states: M_alpha = sum_q log2((1 + x^(2a) + y^(2a) +
    z^(2a)) / 2) / (1 - a)."""
    psi, bloch = W.product_state(N, 321, np.complex64)
    t = dev(torch_cuda, psi)
    with sre.Plan(N, "c64") as p:
        for a in ORDERS:
            expect = np.sum(np.log2((1 + np.sum(bloch ** (2 * a), axis=1)) / 2)) / (1 - a)
            assert abs(p.m_alpha(t, a) - expect) <= 1e-6, a


def test_stabilizer_states_zero(sre, torch_cuda):
    psi = W.stabilizer_state(14, 8, dtype=np.complex64)
    t = dev(torch_cuda, psi)
    with sre.Plan(14, "c64") as p:
        for a in ORDERS:
            assert abs(p.m_alpha(t, a)) <= 1e-6


@pytest.mark.parametrize("N,tuning", [(17, (0, 15, 7, 2, 2)), (20, (0, 23, 11, 3, 2))])
def test_per_shift_sums_sampled(sre, torch_cuda, N, tuning):
    """Per-shift order-alpha sums on sampled shifts against the oracle, both
    copy paths, shifts on both sides of 4096 (full and halved transforms);
    S over the range equals the sum of the per-shift sums."""
    torch = torch_cuda
    psi_np = W.haar_state(N, 123, np.complex64)
    psi = dev(torch, psi_np)
    xr = (4096 - 48, 4096 + 464)
    with sre.Plan(N, "c64") as p:
        for a in (3, 4):
            for s12 in ((1, 1), (0, 0)):
                p.set_tuning(*tuning, *s12)
                out, px = p.sum_pow_range(psi, a, xr[0], xr[1], per_x=True)
                torch.cuda.synchronize()
                px = px.cpu().numpy()
                assert out[0].item() == pytest.approx(float(np.sum(px)), rel=1e-12)
                big = float(np.max(px))
                for x in (xr[0], 4095, 4096, 4200, xr[1] - 1):
                    ref = oracle.sum_pow_xorfwht(psi_np, a, x, x + 1)
                    assert abs(px[x - xr[0]] - ref) <= 1e-5 * big, (a, s12, x)


def test_split_precision_mode(sre, torch_cuda):
    """BF16 hi/lo tensor-core mode at order 3 within the FP32 tolerance."""
    N = 14
    psi = W.haar_state(N, 9, np.complex64)
    t = dev(torch_cuda, psi)
    with sre.Plan(N, "c64", "bf16_split") as p:
        assert abs(p.m_alpha(t, 3) - oracle.malpha(psi, 3)) <= 1e-6


def test_invalid_order_rejected(sre, torch_cuda):
    psi = dev(torch_cuda, W.haar_state(8, 1, np.complex64))
    with sre.Plan(8, "c64") as p:
        for a in (0, 1, 17):
            with pytest.raises(sre.SreError) as ei:
                p.m_alpha(psi, a)
            assert ei.value.status == 1  # SRE_EINVAL


def test_haar_order_three_scale(sre, torch_cuda):
    """N = 18 Haar state: for alpha = 3 the identity term dominates
    S_3 / d (the other 4^N - 1 terms add O(1/d)), so M_3 sits just below
    log2(d) / 2, well under M2."""
    N = 18
    psi = W.haar_state(N, 31, np.complex64)
    t = dev(torch_cuda, psi)
    with sre.Plan(N, "c64") as p:
        m3 = p.m_alpha(t, 3)
        m2 = p.m2(t)
    assert m3 < m2
    assert abs(m3 - N / 2) < 1.0
    assert math.isfinite(m3)
