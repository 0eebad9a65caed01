"""Writes tests/golden/n20_haar_oracle.json: the FP64 oracle's S, n2 and M2
for the N = 20 Haar-random benchmark state, stored as complex64 and as
complex128.

Only ``oracle`` (Algorithm 1 restated in FP64, O2) and the seeded state
generator are called; nothing here touches the CUDA path.  The state is
``workloads.haar_state(20, config_seed(2, 0), dtype)``: re, im i.i.d. N(0, 1),
normalised in FP64, then stored in the given dtype (complex64 values are
widened exactly to FP64 by the oracle, so it evaluates the stored state).

S = sum_{x,z} |<psi|X^x Z^z|psi>|^4 is accumulated as 256 partial sums over
consecutive shift ranges of 4096 (each a Neumaier-compensated FP64 sum inside
the oracle) and combined with math.fsum; M2 = -log2(S / (d n2^4)) (Eq. (sre)
at alpha = 2, base-2 log as in Algorithm 1).  The partial sums are kept, so a
test can compare any shift range on its own.  Each record carries the sha256
of the stored buffer; a consumer must check it before using the values.

The run takes about an hour per dtype on 8 cores.  Progress is checkpointed
in the system temporary directory, so an interrupted run resumes.

Run:  python tests/golden/make_n20_oracle.py [--dtypes c64,c128] [--threads T]
"""
import argparse
import hashlib
import json
import math
import os
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_24685_gb300 import workloads as W  # noqa: E402

N = 20
RANGES = 256
OUT = os.path.join(HERE, "n20_haar_oracle.json")
DTYPES = {"c64": np.complex64, "c128": np.complex128}


def state(tag: str) -> np.ndarray:
    return W.haar_state(N, W.config_seed(2, 0), DTYPES[tag])


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def run(tag: str, ckpt_dir: str) -> dict:
    psi = state(tag)
    digest = sha256(psi)
    ckpt = os.path.join(ckpt_dir, f"sre_n20_{tag}_{digest[:16]}.json")
    parts = {}
    if os.path.exists(ckpt):
        with open(ckpt) as f:
            parts = {int(k): v for k, v in json.load(f).items()}
    d = 1 << N
    step = d // RANGES
    t0 = time.time()
    for r in range(RANGES):
        if r in parts:
            continue
        parts[r] = oracle.sum4_xorfwht(psi, r * step, (r + 1) * step)
        with open(ckpt + ".tmp", "w") as f:
            json.dump({str(k): v for k, v in parts.items()}, f)
        os.replace(ckpt + ".tmp", ckpt)
        done = len(parts)
        el = time.time() - t0
        print(f"[{tag}] range {r + 1}/{RANGES} S_r={parts[r]:.17g} ({el:.0f} s)", flush=True)
    partial = [parts[r] for r in range(RANGES)]
    S = math.fsum(partial)
    n2 = oracle.norm2(psi)
    return {
        "dtype": {"c64": "complex64", "c128": "complex128"}[tag],
        "sha256": digest,
        "N": N,
        "seed": W.config_seed(2, 0),
        "n2": n2,
        "S": S,
        "m2": oracle.m2_from_sum(S, n2, N),
        "range_shifts": step,
        "range_sums": partial,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtypes", default="c64,c128")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--checkpoint-dir", default=tempfile.gettempdir())
    args = ap.parse_args()
    if args.threads > 0:
        oracle.set_threads(args.threads)
    doc = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            doc = json.load(f)
    doc.setdefault("comment", "FP64 oracle (O2, Algorithm 1) on the N = 20 Haar state "
                   "haar_state(20, config_seed(2, 0)); written by make_n20_oracle.py")
    for tag in args.dtypes.split(","):
        rec = run(tag.strip(), args.checkpoint_dir)
        doc[rec["dtype"]] = rec
        with open(OUT + ".tmp", "w") as f:
            json.dump(doc, f, indent=1)
        os.replace(OUT + ".tmp", OUT)
        print(f"[{tag}] S={rec['S']:.17g} n2={rec['n2']:.17g} M2={rec['m2']:.17g}", flush=True)


if __name__ == "__main__":
    main()
