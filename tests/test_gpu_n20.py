"""The N = 20 benchmark state against the FP64 oracle at the metric's
tolerance (Eq. (final1), Algorithm 1's return value).

tests/golden/n20_haar_oracle.json holds S, n2 and M2 of
haar_state(20, config_seed(2, 0)) stored as complex64 and as complex128,
written by tests/golden/make_n20_oracle.py (which calls only the oracle),
with 256 partial sums over consecutive 4096-shift ranges.  The state is
regenerated here and its sha256 checked against the record first.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "n20_haar_oracle.json")
N = 20


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


def record(dtype_name):
    with open(GOLD) as f:
        doc = json.load(f)
    rec = doc.get(dtype_name)
    if rec is None:
        pytest.skip(f"no {dtype_name} record in {GOLD}")
    return rec


def state(dtype):
    psi = W.haar_state(N, W.config_seed(2, 0), dtype)
    rec = record({np.complex64: "complex64", np.complex128: "complex128"}[dtype])
    assert hashlib.sha256(psi.tobytes()).hexdigest() == rec["sha256"], "generator drifted from the record"
    return psi, rec


@pytest.fixture(scope="module")
def c64(torch_cuda):
    psi, rec = state(np.complex64)
    return torch_cuda.from_numpy(psi).cuda(), rec


@pytest.mark.parametrize("mode", ["fp32", "bf16_split", "fp16_split"])
def test_n20_m2_within_tolerance(sre, torch_cuda, c64, mode):
    """|Delta M2| <= 1e-6 against the oracle for the benchmark state, in the
    benchmark's launch configuration (autotuned plan)."""
    t, rec = c64
    with sre.Plan(N, "c64", mode) as p:
        p.autotune(N)
        m2 = p.m2(t)
    assert abs(m2 - rec["m2"]) <= 1e-6, (mode, m2, rec["m2"])


@pytest.mark.parametrize("mode", ["fp32", "fp16_split"])
def test_n20_range_sums(sre, torch_cuda, c64, mode):
    """Partial sums over whole 4096-shift ranges (the shift-0 range takes the
    full 20-bit transform, the others the halved form) against the oracle's:
    a relative error of 1e-6 in S moves M2 by 1.4e-6 at most."""
    t, rec = c64
    step = rec["range_shifts"]
    with sre.Plan(N, "c64", mode) as p:
        for r in (0, 1, 2, 37, 128, 200, 255):
            out = p.sum4_range(t, r * step, (r + 1) * step)
            torch_cuda.cuda.synchronize()
            got = out[0].item()
            ref = rec["range_sums"][r]
            assert abs(got - ref) <= 1e-6 * ref, (mode, r, got, ref)


def test_n20_fp64_complex128(sre, torch_cuda):
    """The FP64 path on the complex128 benchmark state: |Delta M2| <= 1e-10."""
    psi, rec = state(np.complex128)
    with sre.Plan(N, "c128", "fp64") as p:
        m2 = p.m2(torch_cuda.from_numpy(psi).cuda())
    assert abs(m2 - rec["m2"]) <= 1e-10, (m2, rec["m2"])
