"""The stored oracle records pinned to what the paper and the mathematics
fix, independently of the oracle that wrote them (no GPU):

* product states of the N = 16 mix: M2 = -sum_q log2((1 + x^4 + y^4 + z^4)/2)
  from their Bloch vectors (additivity and the single-qubit sum);
* stabilizer states: M2 = 0;
* Haar-random states (the N = 16 mix and the N = 20 benchmark state): near
  the Haar value log2(2^N + 3) - 2 quoted with Fig. 1(b);
* every record's buffer hash (or, on another platform, its fingerprint)
  matches the regenerated state.
"""
import hashlib
import json
import math
import os

import numpy as np
import pytest

from paper_2512_24685_gb300 import workloads as W

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    path = os.path.join(HERE, name)
    if not os.path.exists(path):
        pytest.skip(f"{path} not written yet")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("dtype,name", [(np.complex64, "complex64"), (np.complex128, "complex128")])
def test_n16_mix_record(dtype, name):
    doc = load("n16_mix_oracle.json")
    recs = doc.get(name)
    if not recs or len(recs) != 64:
        pytest.skip(f"no complete {name} record")
    haar = math.log2(2 ** 16 + 3) - 2
    for (kind, psi, bloch), rec in zip(W.mixed_n16_batch(1, 16, 16, 8, dtype), recs):
        assert rec["kind"] == kind
        if hashlib.sha256(psi.tobytes()).hexdigest() != rec["sha256"]:
            # another platform: the generator's last bits may differ
            v = psi.astype(np.complex128)
            n2 = float(np.sum(v.real ** 2 + v.imag ** 2))
            assert abs(n2 - rec["norm2"]) <= 1e-6 * rec["norm2"]
        m = rec["m2"]
        if kind == "product":
            b = np.asarray(bloch, dtype=np.float64)
            closed = -float(np.sum(np.log2((1.0 + np.sum(b ** 4, axis=1)) / 2.0)))
            tol = 1e-10 if dtype == np.complex128 else 1e-5  # complex64 rounding of the stored state
            assert abs(m - closed) <= tol, (m, closed)
        elif kind == "stabilizer":
            assert abs(m) <= (1e-10 if dtype == np.complex128 else 1e-5), m
        elif kind == "haar":
            assert abs(m - haar) < 0.01, (m, haar)
        else:
            assert 0.0 < m < haar + 0.01


def test_n20_record():
    doc = load("n20_haar_oracle.json")
    haar = math.log2(2 ** 20 + 3) - 2
    for name in ("complex64", "complex128"):
        rec = doc.get(name)
        if rec is None:
            continue
        assert abs(rec["m2"] - haar) < 0.001, (name, rec["m2"], haar)
        # the range sums add up to S, and S, n2 give M2 (Eq. (final1))
        S = math.fsum(rec["range_sums"])
        assert abs(S - rec["S"]) <= 1e-12 * rec["S"]
        assert abs(-(math.log2(rec["S"]) - 20 - 4 * math.log2(rec["n2"])) - rec["m2"]) <= 1e-12
