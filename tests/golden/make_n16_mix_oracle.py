"""Writes tests/golden/n16_mix_oracle.json: the FP64 oracle's M2 for each of
the 64 states of the N = 16 four-family mix (16 Haar-random, 16 product, 16
stabilizer, 16 depth-8 brickwork states; workloads.mixed_n16_batch), stored
as complex64 and as complex128.

Only ``oracle`` (Algorithm 1 restated in FP64) and the seeded state
generator are called; nothing here touches the CUDA path.  complex64 values
are widened exactly to FP64 by the oracle, so it evaluates the stored state.
Each record carries the sha256 of the stored buffer and a fingerprint (norm2
and eight amplitudes at fixed indices): the product, stabilizer and brickwork
generators call trigonometric and linear-algebra routines whose last bits
differ between platforms, so a consumer on another machine checks the
fingerprint within a rounding tolerance (a change of the state at that level
moves M2 by far less than any test tolerance) instead of the hash.  About
9 s per state on 8 cores; --reuse keeps the M2 of every state whose hash is
unchanged from an existing record and only recomputes the rest.

Run:  python tests/golden/make_n16_mix_oracle.py [--threads T] [--reuse]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_24685_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "n16_mix_oracle.json")
PROBE = [0, 1, 2, 3, 4097, 20000, 32768, 65535]  # amplitude indices of the fingerprint


def fingerprint(psi):
    v = psi.astype(np.complex128)
    return {"norm2": float(np.sum(v.real ** 2 + v.imag ** 2)),
            "probe": [[float(v[i].real), float(v[i].imag)] for i in PROBE]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--reuse", action="store_true")
    args = ap.parse_args()
    old = {}
    if args.reuse and os.path.exists(OUT):
        with open(OUT) as f:
            prev = json.load(f)
        for name in ("complex64", "complex128"):
            for rec in prev.get(name, []):
                old[rec["sha256"]] = rec["m2"]
    if args.threads:
        oracle.set_threads(args.threads)
    doc = {"comment": "FP64 oracle M2 of workloads.mixed_n16_batch(1, 16, 16, 8, dtype); "
                      "written by tests/golden/make_n16_mix_oracle.py (oracle only)",
           "N": 16, "per_kind": 16, "depth": 8}
    t0 = time.time()
    for name, dtype in (("complex64", np.complex64), ("complex128", np.complex128)):
        recs = []
        for k, (kind, psi, _) in enumerate(W.mixed_n16_batch(1, 16, 16, 8, dtype)):
            sha = hashlib.sha256(psi.tobytes()).hexdigest()
            m2 = old[sha] if sha in old else oracle.m2(psi)
            recs.append({"kind": kind, "m2": m2, "sha256": sha, **fingerprint(psi)})
            print(f"[{name}] {k + 1}/64 {kind} M2={recs[-1]['m2']:.12f} ({time.time() - t0:.0f} s)", flush=True)
        doc[name] = recs
        with open(OUT, "w") as f:
            json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
