"""Writes the oracle's per-batch changes of the triangle and 4-clique counts
and checksums for a stream of update batches (tests/golden/rmat22_delta1k.json):
the R-MAT scale-22 base graph and the first 20 batches of 1,000 updates of
its update stream (90% R-MAT inserts, 10% deletes of base edges), the stream
the dynamic-maintenance benchmark applies.

Only the CPU oracle computes these values: each batch is normalised under
R' = R + Delta R (Section 3.3.1), and the change is Delta-GJ's sum of the
delta queries dQ_1..dQ_n over the old and new graphs (Section 3.3.1, Section
4.3), evaluated literally by the oracle.

    python tests/golden/make_rmat_delta.py [--scale 22] [--batches 20] [--size 1000]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import oracle
    from paper_1802_03760_b300.inputs import QUERIES, UpdateStream, rmat_edges
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--batches", type=int, default=20)
    ap.add_argument("--size", type=int, default=1000)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = args.out or os.path.join(HERE, "rmat%d_delta%dk.json" % (args.scale, args.size // 1000))
    n = 1 << args.scale
    s, d = rmat_edges(args.scale, seed=args.seed)
    stream = UpdateStream(s, d, args.scale, seed=args.seed)
    g = oracle.Graph(n, s, d)
    names = ["triangle", "4-clique"]
    qs = [oracle.Query(*QUERIES[nm]) for nm in names]
    batches = []
    for b in range(args.batches):
        t0 = time.time()
        bs, bd, bg = stream.next_batch(args.size)
        (cs, cd, cg), g2 = oracle.apply_batch(g, bs, bd, bg)
        deltas = {}
        for nm, q in zip(names, qs):
            c, h = oracle.delta(g, g2, cs, cd, cg, q)
            deltas[nm] = {"count": c, "checksum": "%016x" % h}
        batches.append({"batch": b, "changes": int(len(cs)), "edges_after": g2.m, "delta": deltas})
        print(b, len(cs), deltas, round(time.time() - t0, 1), flush=True)
        g = g2
    result = {"workload": "R-MAT scale %d base (seed %d), %d batches of %d updates of its update stream (seed %d)"
                          % (args.scale, args.seed, args.batches, args.size, args.seed),
              "scale": args.scale, "seed": args.seed, "size": args.size, "queries": names,
              "command": "python tests/golden/make_rmat_delta.py --scale %d --batches %d --size %d"
                         % (args.scale, args.batches, args.size), "batches": batches}
    with open(out + ".tmp", "w") as f:
        json.dump(result, f, indent=1)
    os.replace(out + ".tmp", out)
    print("wrote", out, flush=True)


if __name__ == "__main__":
    main()
