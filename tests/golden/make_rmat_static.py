"""Writes the oracle's full-graph counts, checksums and work units for the
static R-MAT workload (tests/golden/rmat20_static.json by default).

Only the CPU oracle computes these values. Counts and checksums are additive
over disjoint ranges of the first attribute of the order (every match has
one value there), so the vertex range is cut into chunks that independent
single-threaded processes evaluate; the sums are the whole graph's. Each
formulation is evaluated in the oracle mode that follows the method it
stands for: mode 1 (edge seeds, Section 4.1 and Section 4.2) and mode 2
(the same with factorised output, Section 5.4).

    python tests/golden/make_rmat_static.py [--scale 20] [--procs 7]

Finished chunks are appended to <out>.partial.jsonl, so an interrupted run
resumes where it stopped; the file is removed once the totals are written.
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

M64 = (1 << 64) - 1

# name -> (shape whose matches it counts, query spec, oracle mode)
FORMULATIONS = {
    "triangle": ("triangle", "triangle", 1),
    "diamond-f": ("diamond", "diamond-f", 2),
    "4-clique-tr": ("4-clique", "4-clique-tr", 1),
}

_G = None


def _spec(name):
    from paper_1802_03760_b300.inputs import QUERIES, SPECIALISED
    if name in SPECIALISED:
        return dict(SPECIALISED[name])
    k, atoms = QUERIES[name]
    return dict(k=k, atoms=atoms, tri=[], lt=[], order=None)


def _init(scale, seed, need_tri):
    global _G
    import oracle
    from paper_1802_03760_b300.inputs import rmat_edges
    s, d = rmat_edges(scale, seed=seed)
    _G = oracle.Graph(1 << scale, s, d)
    if need_tri:
        _G.num_triangles()


def _chunk(args):
    import oracle
    lo, hi, names = args
    out = {"lo": lo, "hi": hi, "res": {}}
    for nm in names:
        _, spec_name, mode = FORMULATIONS[nm]
        sp = _spec(spec_name)
        q = oracle.Query(sp["k"], sp["atoms"], sp["order"], tri=sp["tri"], lt=sp["lt"])
        t0 = time.process_time()
        c, h, st = _G.count(q, first_range=(lo, hi), stats=True, mode=mode)
        out["res"][nm] = {"count": c, "checksum": h, "stats": st.as_dict(), "cpu_s": time.process_time() - t0}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=20)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--procs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--chunk", type=int, default=1024, help="vertex ids per task")
    ap.add_argument("--queries", default=",".join(FORMULATIONS))
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    names = [x for x in args.queries.split(",") if x]
    out = args.out or os.path.join(HERE, "rmat%d_static.json" % args.scale)
    part = out + ".partial.jsonl"
    n = 1 << args.scale
    tasks = [(lo, min(n, lo + args.chunk)) for lo in range(0, n, args.chunk)]
    done = {}
    if os.path.exists(part):
        for line in open(part):
            r = json.loads(line)
            done[(r["lo"], r["hi"])] = r
    todo = [(lo, hi, names) for lo, hi in tasks if (lo, hi) not in done]
    need_tri = any(_spec(FORMULATIONS[nm][1])["tri"] for nm in names)
    t0 = time.time()
    if todo:
        ctx = mp.get_context("spawn")
        with ctx.Pool(args.procs, initializer=_init, initargs=(args.scale, args.seed, need_tri)) as pool, \
                open(part, "a") as pf:
            for i, r in enumerate(pool.imap_unordered(_chunk, todo)):
                pf.write(json.dumps(r) + "\n")
                pf.flush()
                done[(r["lo"], r["hi"])] = r
                if (i + 1) % 64 == 0:
                    print("%d/%d chunks, %.0f s" % (len(done), len(tasks), time.time() - t0), flush=True)
    import oracle
    from paper_1802_03760_b300.inputs import rmat_edges
    s, d = rmat_edges(args.scale, seed=args.seed)
    m = oracle.Graph(n, s, d).m
    result = {"workload": "R-MAT scale %d, seed %d (2^%d vertices, %d samples, %d distinct edges)"
                          % (args.scale, args.seed, args.scale, len(s), m),
              "scale": args.scale, "seed": args.seed, "edges": m, "chunks": len(tasks),
              "command": "python tests/golden/make_rmat_static.py --scale %d --seed %d" % (args.scale, args.seed),
              "queries": {}}
    for nm in names:
        shape, spec_name, mode = FORMULATIONS[nm]
        tot = {"count": 0, "checksum": 0, "cpu_s": 0.0, "stats": None}
        for key in tasks:
            r = done[key]["res"][nm]
            tot["count"] += r["count"]
            tot["checksum"] = (tot["checksum"] + r["checksum"]) & M64
            tot["cpu_s"] += r["cpu_s"]
            if tot["stats"] is None:
                tot["stats"] = {f: list(v) for f, v in r["stats"].items()}
            else:
                for f, v in r["stats"].items():
                    tot["stats"][f] = [a + b for a, b in zip(tot["stats"][f], v)]
        result["queries"][nm] = {"shape": shape, "spec": _spec(spec_name), "oracle_mode": mode,
                                 "count": tot["count"], "checksum": "%016x" % tot["checksum"],
                                 "stats": tot["stats"], "oracle_cpu_s": round(tot["cpu_s"], 1)}
    with open(out + ".tmp", "w") as f:
        json.dump(result, f, indent=1)
    os.replace(out + ".tmp", out)
    os.remove(part)
    print("wrote", out, flush=True)


if __name__ == "__main__":
    main()
