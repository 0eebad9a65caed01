"""The 64-state N = 16 mix (16 Haar-random, 16 product, 16 stabilizer, 16
depth-8 brickwork states) as one batch in every arithmetic mode, against the
FP64 oracle's M2 per state (Eq. (final1), Algorithm 1's return value).

tests/golden/n16_mix_oracle.json is written by
tests/golden/make_n16_mix_oracle.py, which calls only the oracle; the states
are regenerated here and checked against the record's fingerprint (norm2 and
eight amplitudes) within a rounding tolerance first: the generators' last bits
differ between platforms, which moves M2 by far less than the tolerances.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2512_24685_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "n16_mix_oracle.json")


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


def mix(dtype):
    name = {np.complex64: "complex64", np.complex128: "complex128"}[dtype]
    if not os.path.exists(GOLD):
        pytest.skip(f"{GOLD} not written yet")
    with open(GOLD) as f:
        doc = json.load(f)
    recs = doc.get(name)
    if not recs or len(recs) != 64:
        pytest.skip(f"no complete {name} record")
    states = [psi for _, psi, _ in W.mixed_n16_batch(1, 16, 16, 8, dtype)]
    for psi, rec in zip(states, recs):
        assert_fingerprint(psi, rec)
    return states, [r["m2"] for r in recs], [r["kind"] for r in recs]


PROBE = [0, 1, 2, 3, 4097, 20000, 32768, 65535]


def assert_fingerprint(psi, rec):
    """The regenerated state equals the recorded one up to rounding."""
    if hashlib.sha256(psi.tobytes()).hexdigest() == rec["sha256"]:
        return
    rtol = 1e-6 if psi.dtype == np.complex64 else 1e-12
    v = psi.astype(np.complex128)
    n2 = float(np.sum(v.real ** 2 + v.imag ** 2))
    assert abs(n2 - rec["norm2"]) <= rtol * rec["norm2"], "generator drifted from the record"
    for i, (re, im) in zip(PROBE, rec["probe"]):
        assert abs(v[i] - complex(re, im)) <= rtol * (1e-3 + abs(complex(re, im))), ("generator drifted", i)


@pytest.mark.parametrize("mode", ["fp32", "fp16_split", "bf16_split"])
def test_mix16_batch_complex64(sre, torch_cuda, mode):
    torch = torch_cuda
    states, want, kinds = mix(np.complex64)
    ts = [torch.from_numpy(v).cuda() for v in states]
    with sre.Plan(16, "c64", mode) as p:
        got = p.m2_batched(ts).cpu().numpy()
    for g, w, k in zip(got, want, kinds):
        assert abs(g - w) <= 1e-6, (mode, k, g, w)


def test_mix16_batch_fp64(sre, torch_cuda):
    torch = torch_cuda
    states, want, kinds = mix(np.complex128)
    ts = [torch.from_numpy(v).cuda() for v in states]
    with sre.Plan(16, "c128", "fp64") as p:
        got = p.m2_batched(ts).cpu().numpy()
    for g, w, k in zip(got, want, kinds):
        assert abs(g - w) <= 1e-10, (k, g, w)
