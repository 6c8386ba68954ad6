"""Micro-benchmark of one COCG kernel in isolation, through ``rsn_bench_kernel``.

    python -m paper_1401_0782_gb300.kernel_bench --kind op --slots 256 --reps 3

Builds the 24x24x120 synthetic junction (8th-order FD, 20 atoms x 4 KB
projectors, seed 1), gives every slot a synthetic ACTIVE state and times
``reps`` launches of the chosen kernel with CUDA events on the library's
stream.  Prints one JSON line: milliseconds per launch, the kernel's
algorithmic bytes per launch and their ratio in GB/s.  This is the command the
operator- and update-kernel profiles are taken with (a small case: about 1 GB
on the device for 256 slots).
"""
from __future__ import annotations

import argparse
import json

from . import binding as B
from . import problems as P

KINDS = {"op": 0, "update": 1, "resid": 2}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--kind", choices=sorted(KINDS), default="op")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--slots", type=int, default=256)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tiling", type=int, nargs=3, metavar=("TY", "LZ", "PPT"), default=None,
                    help="fixed operator tiling (default: the library's choice)")
    args = ap.parse_args(argv)
    prec = B.RSN_MIXED if args.precision == "mixed" else B.RSN_FP64
    j = P.molecular_junction(seed=1)
    ctx = B.Context(0).set_junction(j)
    if args.tiling:
        ctx.set_tiling(*args.tiling)
    ms, by = ctx.bench_kernel(prec, KINDS[args.kind], args.slots, args.reps)
    print(json.dumps({"kernel": args.kind, "precision": args.precision, "slots": args.slots,
                      "junction": j.name, "N": j.N, "ms_per_launch": ms, "bytes_per_launch": by,
                      "GB_per_s": by / ms / 1e6}))
    ctx.close()


if __name__ == "__main__":
    main()
