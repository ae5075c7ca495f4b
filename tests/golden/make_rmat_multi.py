"""Writes the oracle's counts and checksums of the batched multi-query sample
(tests/golden/rmat24_multi64.json): the 64 mixed queries (the five shapes
and seeded direction/order variants) on R-MAT scale 24, restricted to the
matches whose first attribute lies in [0, 64), which is the sample the
multi-query benchmark times.

Only the CPU oracle computes these values (mode 1: edge seeds, Section 4.1
and Section 4.2), one query per task in independent processes.

    python tests/golden/make_rmat_multi.py [--scale 24] [--procs 3]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

_G = None


def _init(scale, seed):
    global _G
    import oracle
    from paper_1802_03760_b300.inputs import rmat_edges
    s, d = rmat_edges(scale, seed=seed)
    _G = oracle.Graph(1 << scale, s, d)


def _one(args):
    import oracle
    i, k, atoms, order, lo, hi = args
    t0 = time.process_time()
    c, h, st = _G.count(oracle.Query(k, atoms, order), first_range=(lo, hi), stats=True, mode=1)
    return i, c, h, st.as_dict(), time.process_time() - t0


def main():
    from paper_1802_03760_b300.inputs import mixed_queries
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--queries", type=int, default=64)
    ap.add_argument("--query-seed", type=int, default=1)
    ap.add_argument("--first", type=int, default=64, help="first attribute in [0, FIRST)")
    ap.add_argument("--procs", type=int, default=3)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = args.out or os.path.join(HERE, "rmat%d_multi%d.json" % (args.scale, args.queries))
    mq = mixed_queries(args.queries, seed=args.query_seed)
    tasks = [(i, k, atoms, order, 0, args.first) for i, (_, k, atoms, order) in enumerate(mq)]
    res = [None] * len(tasks)
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs, initializer=_init, initargs=(args.scale, args.seed)) as pool:
        for i, c, h, st, cpu in pool.imap_unordered(_one, tasks):
            res[i] = {"name": mq[i][0], "k": mq[i][1], "atoms": mq[i][2], "order": mq[i][3], "count": c,
                      "checksum": "%016x" % h, "stats": st, "oracle_cpu_s": round(cpu, 2)}
            print(i, mq[i][0], c, flush=True)
    result = {"workload": "R-MAT scale %d, seed %d; %d mixed queries (seed %d); first attribute in [0, %d)"
                          % (args.scale, args.seed, args.queries, args.query_seed, args.first),
              "scale": args.scale, "seed": args.seed, "query_seed": args.query_seed, "first": args.first,
              "command": "python tests/golden/make_rmat_multi.py --scale %d" % args.scale, "queries": res}
    with open(out + ".tmp", "w") as f:
        json.dump(result, f, indent=1)
    os.replace(out + ".tmp", out)
    print("wrote", out, flush=True)


if __name__ == "__main__":
    main()
