"""Command line front end of libsre.

    python -m paper_2512_24685_gb300.cli m2 --N 20 [--family haar] [--seed S] [--mode fp32]
    python -m paper_2512_24685_gb300.cli range --N 20 --x-begin B --count C [--per-x]

Both take --tuning C_LOG,R,D,G2,B1[,S1,S2] (the two-pass kernel's chunk
size, ring slots, lag, pass-2 tiles and pass-1 blocks per item, logs base 2
where named so, and whether pass 1 / pass 2 take their data by bulk copy
into shared memory; -1 keeps the default) or --autotune
(sre_plan_autotune first).

`m2` evaluates M2 of one generated state; `range` evaluates the partial sum
sum_{x in [B, B+C)} sum_z |<psi|X^x Z^z|psi>|^4 through sre_sum4_range (the
shard of a state's work that one device takes when shifts are split).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def _state(args):
    from . import workloads as W
    dt = np.complex64 if args.dtype == "c64" else np.complex128
    if args.family == "haar":
        return W.haar_state(args.N, args.seed, dt)
    if args.family == "product":
        return W.product_state(args.N, args.seed, dt)[0]
    if args.family == "stabilizer":
        return W.stabilizer_state(args.N, args.seed, dtype=dt)
    if args.family == "brickwork":
        return W.brickwork_state(args.N, args.depth, args.seed, dt)
    raise SystemExit(f"unknown family {args.family}")


def main(argv=None):
    ap = argparse.ArgumentParser(prog="paper_2512_24685_gb300.cli")
    sub = ap.add_subparsers(dest="cmd", required=True)
    for name in ("m2", "range"):
        p = sub.add_parser(name)
        p.add_argument("--N", type=int, required=True)
        p.add_argument("--family", default="haar", choices=["haar", "product", "stabilizer", "brickwork"])
        p.add_argument("--seed", type=int, default=0)
        p.add_argument("--depth", type=int, default=8)
        p.add_argument("--dtype", default="c64", choices=["c64", "c128"])
        p.add_argument("--mode", default=None)
        p.add_argument("--repeat", type=int, default=1)
        p.add_argument("--tuning", default=None, help="C_LOG,R,D,G2,B1[,S1,S2] of the halved-shift launch")
        p.add_argument("--autotune", action="store_true")
        p.add_argument("--alpha", type=int, default=2, help="Renyi order (integer >= 2)")
        if name == "range":
            p.add_argument("--x-begin", type=int, required=True)
            p.add_argument("--count", type=int, required=True)
            p.add_argument("--per-x", action="store_true")
    args = ap.parse_args(argv)

    import torch

    from . import binding
    psi = torch.from_numpy(_state(args)).cuda()
    out = {"cmd": args.cmd, "N": args.N, "family": args.family, "seed": args.seed}
    with binding.Plan(args.N, args.dtype, args.mode) as plan:
        if args.tuning:
            plan.set_tuning(*[int(v) for v in args.tuning.split(",")])
        elif args.autotune:
            plan.autotune(args.N)
        if args.tuning or args.autotune:
            out["tuning"] = plan.get_tuning(args.N)
        t0 = time.perf_counter()
        for _ in range(args.repeat):
            if args.cmd == "m2":
                if args.alpha == 2:
                    out["m2"] = plan.m2(psi)
                else:
                    out["alpha"] = args.alpha
                    out["m_alpha"] = plan.m_alpha(psi, args.alpha)
            else:
                xe = args.x_begin + args.count
                if args.alpha == 2:
                    res = plan.sum4_range(psi, args.x_begin, xe, per_x=args.per_x)
                else:
                    out["alpha"] = args.alpha
                    res = plan.sum_pow_range(psi, args.alpha, args.x_begin, xe, per_x=args.per_x)
                sums = res[0] if args.per_x else res
                torch.cuda.synchronize()
                out["x_range"] = [args.x_begin, xe]
                out["sum4"] = sums[0].item()
                out["n2"] = sums[1].item()
                if args.per_x:
                    out["per_x_first"] = res[1][:8].cpu().tolist()
        torch.cuda.synchronize()
        out["seconds"] = (time.perf_counter() - t0) / args.repeat
        out["mode"] = plan.mode
    print(json.dumps(out))


if __name__ == "__main__":
    main()
