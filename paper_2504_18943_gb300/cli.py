"""Command line: solve a seeded workload, or build its levels up to a size.

  python -m paper_2504_18943_gb300.cli solve  --workload mid --seed 2
  python -m paper_2504_18943_gb300.cli levels --workload mid --seed 2 --up-to 9 --cache-gb 4

Prints one JSON object per level and a summary. Every step runs in the CUDA
library through the C ABI; the traces are labelled on the GPU (lsyn_eval).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

from . import lsyn as L
from . import workloads as W

MAKERS = {"tiny": W.tiny_problem, "mid": W.mid_problem, "large": W.large_problem}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(prog="python -m paper_2504_18943_gb300.cli")
    ap.add_argument("mode", choices=["solve", "levels"])
    ap.add_argument("--workload", default="mid", choices=sorted(MAKERS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--max-size", type=int, default=16)
    ap.add_argument("--up-to", type=int, default=8)
    ap.add_argument("--cache-gb", type=float, default=8.0)
    ap.add_argument("--ops", default="all", choices=["all", "paper"])
    ap.add_argument("--full-levels", action="store_true")
    args = ap.parse_args(argv)

    problem = MAKERS[args.workload](args.seed, L.labeller)
    packed = L.pack_problem(problem)
    cfg = L.make_config(op_mask=L.OPS_ALL if args.ops == "all" else L.OPS_PAPER,
                        cache_bytes=int(args.cache_gb * (1 << 30)), timing=True,
                        full_levels=args.full_levels or args.mode == "levels")
    with L.Synthesizer(packed, cfg) as s:
        t0 = time.perf_counter()
        if args.mode == "solve":
            st, res, formula, levels = s.solve(args.max_size)
            for lv in levels:
                print(json.dumps(lv.as_dict()))
            print(json.dumps({"status": st, "size": res.size, "formula": formula, "unique": res.unique,
                              "constructed": res.constructed, "seconds": time.perf_counter() - t0}))
        else:
            for k in range(1, args.up_to + 1):
                lv = s.level(k)
                print(json.dumps(lv.as_dict()))
                if lv.cache_full:
                    break
            print(json.dumps({"levels": args.up_to, "seconds": time.perf_counter() - t0}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
