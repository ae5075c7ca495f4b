"""Benchmark: static subgraph-query throughput on the R-MAT scale-20 graph,
with the dynamic-maintenance and serving metrics as sub-records.

One step is one pass of the whole static hot path over one synthetic input:
build the forward and reverse indices from the device-resident edge list
(sort, dedup, offsets, hash sets), build the triangle index (the ternary
relation of Section 5.4), then count and checksum the triangle, diamond and
4-clique queries in one persistent launch of the fused engine. The diamond
runs in the attribute order a2, a3, a1, a4, whose last two attributes extend
independently (factorised output, Section 5.4: the a1 extensions of each
(a2, a3) pair are counted and their hash factors summed, and the pair is
extended to a4 once); the 4-clique runs over three triangle atoms (triangle
indexing, Section 5.4). ``value`` is matches per second
over the step (device-resident inputs, CUDA events on the library's
stream); ``e2e`` is the same metric through the C ABI with pinned host
inputs, so every step also copies the edge list in and the counts out.

The line also carries: ``delta`` (edge-updates/s and per-batch p50/p99 of
update batches on an R-MAT scale-22 base, inputs copied from the host),
``serve`` (served vs sequential plain p50/p99 under Poisson arrivals),
``plain`` (the level-synchronous engine, one query at a time, plain
formulations) and ``default_orders`` (the fused engine on the plain
formulations), each with its own clock record.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs the full workload on its own GPU (replicas,
weak scaling, no collective on the data path); rank 0 prints one JSON line.
``--impl reference`` times the CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1802_03760_b300.inputs import QUERIES, SPECIALISED, rmat_edges  # noqa: E402

SCALE = 20
BENCH_QUERIES = ["triangle", "diamond", "4-clique"]
# shape -> the formulation the benchmark evaluates (same matches, Section 5.4)
FORMULATIONS = {"triangle": "triangle", "diamond": "diamond-f", "4-clique": "4-clique-tr"}
METRIC = "matches/sec (tri, 4-clique, diamond)"
GOLDEN = os.path.join(ROOT, "tests", "golden")
PROFILE = os.path.join(ROOT, "profiles", "k_fused_static_rmat20.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1802_03760_b300", "csrc", f) for f in ("engine_fused.cu", "gj_internal.cuh")]


def workload_name(scale, queries):
    return "static %s count+checksum, R-MAT scale %d (2^%d vertices, 2^%d samples)" % (
        "+".join(queries), scale, scale, scale + 4)


def formulation(name):
    """(k, atoms, order, tri, lt) of a query shape or a specialised formulation."""
    if name in SPECIALISED:
        sp = SPECIALISED[name]
        return sp["k"], sp["atoms"], sp["order"], sp["tri"], sp["lt"]
    k, atoms = QUERIES[name]
    return k, atoms, None, [], []


def gj_query(gj, ctx, name):
    k, atoms, order, tri, lt = formulation(name)
    return gj.Query(ctx, k, atoms, order, tri=tri, lt=lt)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(w, k: int) -> int:
    """Bytes of the prefix-extension cost model for one query's work units.

    8 per seed edge (vertex and neighbour), and per prefix of length j with
    n_j binding atoms and min count c: 4j (prefix) + 16 n_j (two offsets per
    atom) + 4c (min list) + 4c(n_j - 1) (one probe per proposal per other
    atom), plus 4(j+1) per prefix produced for a non-final level.
    """
    total = 8 * w.seeds
    for j in range(2, k):
        if w.extended[j] == 0:
            continue
        nb = w.nbind[j] // w.extended[j]
        total += 4 * j * w.extended[j] + 16 * w.nbind[j] + 4 * w.proposals[j] + 4 * w.proposals[j] * (nb - 1)
        if j + 1 < k:
            total += 4 * (j + 1) * w.produced[j + 1]
    return total


def golden_static(scale, seed=1):
    """The oracle's full-graph counts, checksums and work units for the
    benchmark's formulations (written by tests/golden/make_rmat_static.py),
    or None when no golden exists for this graph."""
    path = os.path.join(GOLDEN, "rmat%d_static.json" % scale)
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    if g.get("seed") != seed:
        return None
    return g


def oracle_bytes(gold, shape):
    """Cost-model bytes of one formulation from the oracle's work units."""
    q = gold["queries"][FORMULATIONS[shape]]
    st = q["stats"]

    class W:
        seeds = gold["edges"]
        extended = st["extended"]
        nbind = st["nbind_sum"]
        proposals = st["proposals"]
        produced = st["prefixes"]
    return algorithmic_bytes(W, q["spec"]["k"])


def code_only(text: str) -> str:
    """A CUDA source with its comments, blank lines and trailing blanks
    removed: what the compiler turns into the kernel."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_sources_sha():
    """sha256 of the dominant kernel's sources without comments, so that a
    comment edit keeps an ncu capture of the same code valid."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(code_only(open(f).read()).encode())
        h.update(b"\0")
    return h.hexdigest()


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if that summary measured the current kernel sources (else None)."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None, "no ncu summary"
    m_sha = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", text)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    if not m_sha or not m_tr:
        return None, "ncu summary without traffic"
    if m_sha.group(1) != kernel_sources_sha():
        return None, "kernel changed since the ncu capture"
    return int(m_tr.group(1)), "ncu capture (profiles/%s)" % os.path.basename(PROFILE)


def cpu_sample(s, d, n, target_s: float, queries, seed=5):
    """Times the CPU oracle (single thread) on a sample of the same workload:
    the matches whose first attribute lies in a set of 64-vertex ranges at
    seeded random offsets, grown until a pass takes about a third of
    target_s. The oracle evaluates the triangle and the 4-clique with edge
    atoms (mode 1) and the diamond factorised (mode 2); its triangle index is
    not built, as building it for the whole graph would take minutes.
    Returns (matches/s, sample description, seconds, matches)."""
    import oracle

    og = oracle.Graph(n, s, d)
    forms = []
    for nm in queries:
        f = FORMULATIONS.get(nm, nm)
        if formulation(f)[3]:  # tri atoms: the edge formulation of the same shape
            f = nm
        k, atoms, order, tri, lt = formulation(f)
        forms.append((oracle.Query(k, atoms, order, tri=tri, lt=lt), 2 if f in SPECIALISED else 1))
    rng = np.random.default_rng(seed)
    starts = [int(x) * 64 for x in rng.permutation(max(1, n // 64))]
    nr = 1
    while True:
        t0 = time.perf_counter()
        matches = 0
        for q, mode in forms:
            for lo in starts[:nr]:
                matches += og.count(q, first_range=(lo, min(n, lo + 64)), mode=mode)[0]
        el = time.perf_counter() - t0
        if el >= target_s / 3 or nr >= len(starts):
            break
        nr = min(len(starts), nr * 2)
    sample = ("first attribute in %d ranges of 64 vertex ids at seeded random offsets (%.3f%% of %d vertices), "
              "queries %s" % (nr, 100.0 * min(n, 64 * nr) / n, n, "+".join(queries)))
    return matches / el, sample, el, matches


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    n = 1 << args.scale
    s, d = rmat_edges(args.scale, seed=1)
    per = max(3.0, 45.0 / max(1, args.steps + args.warmup))
    vals = []
    sample = ""
    for i in range(args.warmup + args.steps):
        v, sample, el, _ = cpu_sample(s, d, n, per, args.queries)
        if i >= args.warmup:
            vals.append(v)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "matches/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload_name(args.scale, args.queries), "engine": "cpu oracle (single thread)"},
            "cpu_baseline": {"value": v, "unit": "matches/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "matches/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def sub_record(name, fn, *a, **kw):
    """One secondary record of the headline line (delta, serve). A failure
    there is reported in the record and on stderr; the headline, already
    measured and checked against the oracle, is still printed."""
    try:
        return fn(*a, **kw)
    except Exception as e:
        print("bench: the %s record failed: %s: %s" % (name, type(e).__name__, e), file=sys.stderr, flush=True)
        return {"error": "%s: %s" % (type(e).__name__, e)}


def _events(torch, stream):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_ours(args):
    import torch
    from paper_1802_03760_b300 import gj

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    n = 1 << args.scale
    s, d = rmat_edges(args.scale, seed=1)
    stream = torch.cuda.Stream()
    ctx = gj.Context(local, stream=stream.cuda_stream)
    forms = [FORMULATIONS[nm] for nm in args.queries]
    qs = [gj_query(gj, ctx, f) for f in forms]
    ds = torch.from_numpy(s.view(np.int32)).cuda()
    dd = torch.from_numpy(d.view(np.int32)).cuda()
    hs = torch.from_numpy(s.view(np.int32)).pin_memory()
    hd = torch.from_numpy(d.view(np.int32)).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step(src, dst, queries=qs, engine=gj.ENGINE_FUSED, tri=True):
        g = gj.Graph(ctx, src, dst, n)
        if tri:
            g.build_triangles()
        c, h = gj.count_many(g, queries, engine=engine)
        g.free()
        return c, h

    def timed(src, dst, k, **kw):
        times = []
        res = None
        for _ in range(k):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = _events(torch, stream)
            torch.cuda.synchronize()
            e0.record(stream)
            res = step(src, dst, **kw)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, res

    # warm-up (also fixes the expected counts of the timed steps)
    for _ in range(args.warmup):
        ref = step(ds, dd)
    gold = golden_static(args.scale)
    parity = None
    if gold is not None:
        want = ([gold["queries"][f]["count"] for f in forms], [int(gold["queries"][f]["checksum"], 16) for f in forms])
        if tuple(ref) != tuple(want):
            raise RuntimeError("counts differ from the oracle's full-graph golden: %s vs %s" % (ref, want))
        parity = "bit-exact counts and checksums against the oracle's full-graph golden (%s)" % (
            "tests/golden/rmat%d_static.json" % args.scale)
        abytes = sum(oracle_bytes(gold, nm) for nm in args.queries)
        bytes_source = "oracle work units (golden), cost model per formulation"
    else:
        g = gj.Graph(ctx, ds, dd, n)
        g.build_triangles()
        abytes = 0
        for f, q in zip(forms, qs):
            _, _, w = gj.count(g, q, engine=gj.ENGINE_FUSED, stats=True)
            abytes += algorithmic_bytes(w, formulation(f)[0])
        g.free()
        bytes_source = "kernel work counters (no oracle golden at this scale)"
    m_edges = gj.Graph(ctx, ds, dd, n).m

    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local).start()
    ctx.profile(True)
    ctx.profile_read()
    l0 = ctx.launches
    times, res = timed(ds, dd, args.steps)
    launches = ctx.launches - l0
    kern_ms, kern_n = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    torch.cuda.synchronize()
    if res != ref:
        raise RuntimeError("counts changed between steps: %s vs %s" % (res, ref))
    matches = sum(res[0])
    step_ms = sum(times) / len(times)
    if world > 1:
        import torch.distributed as dist
        from paper_1802_03760_b300.shard import max_over_ranks
        step_ms = max_over_ranks(step_ms)
        dist.barrier()

    # end to end through the C ABI with pinned host inputs
    clocks_e2e = ClockSampler(local).start()
    e2e_times, res_e2e = timed(hs, hd, args.steps)
    clk_e2e = clocks_e2e.stop()
    if res_e2e != ref:
        raise RuntimeError("end-to-end counts differ from the device-resident run")
    e2e_ms = sum(e2e_times) / len(e2e_times)
    if world > 1:
        from paper_1802_03760_b300.shard import max_over_ranks
        e2e_ms = max_over_ranks(e2e_ms)

    extra = {}
    plain_q = [gj.Query(ctx, *QUERIES[nm]) for nm in args.queries]
    if not args.no_plain:
        # the fused engine on the plain formulations (edge atoms, default orders)
        ctx.profile(True)
        ctx.profile_read()
        c0 = ClockSampler(local).start()
        t_def, r_def = timed(ds, dd, 1, queries=plain_q, tri=False)
        kms, kn = ctx.profile_read()
        ctx.profile(False)
        clk_def = c0.stop()
        if list(r_def[0]) != list(ref[0]):
            raise RuntimeError("default orders give other counts")
        g = gj.Graph(ctx, ds, dd, n)
        b_def = 0
        for nm, q in zip(args.queries, plain_q):
            _, _, w = gj.count(g, q, engine=gj.ENGINE_FUSED, stats=True)
            b_def += algorithmic_bytes(w, QUERIES[nm][0])
        g.free()
        peak, _ = peaks()
        ach = b_def / (kms / max(kn, 1) / 1e3) / 1e9
        extra["default_orders"] = {
            "ms_per_step": t_def[0], "value": matches / (t_def[0] / 1e3), "steps": 1,
            "kernel_ms_per_launch": kms / max(kn, 1), "algorithmic_bytes_per_launch": b_def,
            "roofline_frac": ach / peak, "achieved_gbs": ach, "clocks": clk_def,
            "note": "fused engine, plain formulations (edge atoms, default orders): the formulation of the previous line"}
        # the plain level-synchronous engine, one query after another, plain formulations
        c0 = ClockSampler(local).start()
        ptimes = []
        for _ in range(max(1, args.plain_steps)):
            t_p, r_p = timed(ds, dd, 1, queries=plain_q, engine=gj.ENGINE_PLAIN, tri=False)
            if r_p != ref:
                raise RuntimeError("plain engine disagrees with the fused engine")
            ptimes += t_p
        clk_p = c0.stop()
        pms = sum(ptimes) / len(ptimes)
        extra["plain"] = {"ms_per_step": pms, "value": matches / (pms / 1e3), "steps": len(ptimes),
                          "fused_speedup": pms / step_ms, "clocks": clk_p,
                          "engine": "level-synchronous, one query at a time, edge atoms in default orders"}

    if rank == 0 and not args.no_delta:
        extra["delta"] = sub_record("delta", measure_delta, local, 22 if args.scale == SCALE else args.scale + 2,
                                    args.batch_sizes, args.delta_batches, 3, host_inputs=True)
    if rank == 0 and not args.no_serve:
        serve_scale = 16 if args.scale == SCALE else max(8, args.scale - 4)
        extra["serve"] = sub_record("serve", measure_serve, local, serve_scale, args.hub_degree,
                                    args.serve_requests, (0.8,))

    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    kern_avg_ms = kern_ms / max(kern_n, 1)
    achieved = abytes / (kern_avg_ms / 1e3) / 1e9 if kern_avg_ms > 0 else 0.0
    traffic, traffic_src = profiled_traffic() if args.scale == SCALE else (None, "small profiling scale")
    if args.cpu_seconds > 0:
        cpu_v, cpu_sample_desc, _, _ = cpu_sample(s, d, n, args.cpu_seconds, args.queries)
        cpu = {"value": cpu_v, "unit": "matches/s", "cores": 1, "kind": "oracle", "sample": cpu_sample_desc}
    else:
        cpu = None
    line = {
        "metric": METRIC,
        "value": world * matches / (step_ms / 1e3),
        "unit": "matches/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": step_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": workload_name(args.scale, args.queries), "graph_edges": m_edges,
                   "queries": args.queries,
                   "formulations": {nm: {"order": formulation(FORMULATIONS[nm])[2],
                                         "tri_atoms": formulation(FORMULATIONS[nm])[3]} for nm in args.queries},
                   "engine": "fused (one persistent launch for the three queries) after GPU index and "
                             "triangle-index builds",
                   "l2": "flushed between steps (256 MiB write)", "parallelism": "replicas" if world > 1 else "1 GPU",
                   "seed": 1},
        "matches": dict(zip(args.queries, res[0])),
        "parity": parity,
        "e2e": {"value": world * matches / (e2e_ms / 1e3), "unit": "matches/s",
                "h2d_bytes_per_step": int(hs.numel() * 4 + hd.numel() * 4),
                "d2h_bytes_per_step": 16 * len(args.queries), "ms_per_step": e2e_ms, "clocks": clk_e2e},
        "roofline": {"bound": "hbm", "kernel": "k_fused", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                     "traffic_source": traffic_src, "algorithmic_bytes_per_launch": abytes,
                     "algorithmic_bytes_source": bytes_source, "kernel_ms_per_launch": kern_avg_ms,
                     "launches": kern_n},
        "cpu_baseline": cpu,
        "clocks": clk,
        "gpu_launches": launches,
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measure_delta(local, scale, batch_sizes, batches, warmup, host_inputs=True, seed=1):
    """Dynamic maintenance: per batch size, a stream of update batches over the
    same R-MAT base graph, each applied with gj_apply_batch (normalise, delta
    triangle and 4-clique counts, commit), its inputs read from pinned host
    memory (host_inputs) or from the device. Returns edge-updates/s and the
    batch-latency percentiles per size, with the clocks seen meanwhile."""
    import torch
    from paper_1802_03760_b300 import gj
    from paper_1802_03760_b300.inputs import UpdateStream

    n = 1 << scale
    s, d = rmat_edges(scale, seed=seed)
    stream_gen = UpdateStream(s, d, scale, seed=seed)
    qnames = ["triangle", "4-clique"]
    stream = torch.cuda.Stream()
    ctx = gj.Context(local, stream=stream.cuda_stream)
    qs = [gj.Query(ctx, *QUERIES[nm]) for nm in qnames]
    ds = torch.from_numpy(s.view(np.int32)).cuda()
    dd = torch.from_numpy(d.view(np.int32)).cuda()
    sizes = [int(x) for x in str(batch_sizes).split(",")]
    per_size = {}
    all_updates, all_ms = 0, 0.0
    clocks = ClockSampler(local).start()
    launches0 = ctx.launches
    for b in sizes:
        stream_gen.del_cursor = 0  # every size starts from the same base graph
        stream_gen.ins_cursor = 0
        g = gj.Graph(ctx, ds, dd, n)
        prepared = []
        for _ in range(batches + warmup):
            bs, bd, bg = stream_gen.next_batch(b)
            ts = [torch.from_numpy(bs.view(np.int32)), torch.from_numpy(bd.view(np.int32)), torch.from_numpy(bg)]
            prepared.append([t.pin_memory() if host_inputs else t.cuda() for t in ts])
        torch.cuda.synchronize()
        lat = []
        changes = 0
        dsum = [0, 0]
        for i, (bs, bd, bg) in enumerate(prepared):
            torch.cuda.synchronize()
            e0, e1 = _events(torch, stream)
            e0.record(stream)
            dc, _ = gj.apply_batch(g, bs, bd, bg, qs)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                lat.append(e0.elapsed_time(e1))
                changes += gj.last_batch_changes(g)
                dsum = [x + y for x, y in zip(dsum, dc)]
        g.free()
        tot_ms = sum(lat)
        per_size[str(b)] = {"batches": len(lat), "updates_per_s": b * len(lat) / (tot_ms / 1e3),
                            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                            "mean_ms": tot_ms / len(lat), "net_changes": changes,
                            "delta_matches": dict(zip(qnames, dsum))}
        all_updates += b * len(lat)
        all_ms += tot_ms
    clk = clocks.stop()
    launches = ctx.launches - launches0
    ctx.close()
    return {"metric": "edge-updates/sec (delta triangle + 4-clique maintenance)",
            "value": all_updates / (all_ms / 1e3), "unit": "edge-updates/s",
            "workload": "R-MAT scale %d base, update batches of %s edges (90%% R-MAT inserts, 10%% deletes of "
                        "existing edges), delta triangle + 4-clique per batch, %d timed batches per size after %d "
                        "warm-up" % (scale, batch_sizes, batches, warmup),
            "inputs": "pinned host memory, copied inside each timed batch" if host_inputs else "device memory",
            "per_size": per_size, "clocks": clk, "gpu_launches": launches,
            "engine": "delta queries dQ_i with old/new views on the engine chosen by batch size (level-synchronous "
                      "below 8,192 normalised changes, fused from there), then the commit proportional to the change"}


def run_delta(args):
    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    scale = args.scale if args.scale != SCALE else 22
    r = measure_delta(local, scale, args.batch_sizes, args.batches, args.warmup, host_inputs=True)
    if rank != 0:
        return 0
    nb = sum(v["batches"] for v in r["per_size"].values())
    line = {"metric": r["metric"], "value": r["value"], "unit": r["unit"], "n_gpus": world, "steps": args.batches,
            "warmup": args.warmup, "ms_per_step": sum(v["mean_ms"] * v["batches"] for v in r["per_size"].values()) / nb,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": r["workload"], "per_size": r["per_size"], "engine": r["engine"],
                       "inputs": r["inputs"]},
            "clocks": r["clocks"], "gpu_launches": r["gpu_launches"]}
    print(json.dumps(line), flush=True)
    return 0


def serve_trace(scale, hubs, hub_deg, nreq, seed=1):
    """Base graph (R-MAT plus planted hubs) and a seeded request mix: half
    counts of one query (triangle, diamond or 4-clique), half update batches
    of log-uniform size in [1e3, 1e5] reporting delta triangle and 4-clique."""
    from paper_1802_03760_b300.inputs import UpdateStream, hub_edges
    s, d = rmat_edges(scale, seed=seed)
    _, hs, hd = hub_edges(1 << scale, hubs, hub_deg, seed=seed)
    s = np.concatenate([s, hs])
    d = np.concatenate([d, hd])
    stream = UpdateStream(s, d, scale, seed=seed)
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(nreq):
        if rng.random() < 0.5:
            reqs.append(("count", None, [BENCH_QUERIES[int(rng.integers(0, 3))]]))
        else:
            b = int(round(10 ** rng.uniform(3, 5)))
            reqs.append(("batch", stream.next_batch(b), ["triangle", "4-clique"]))
    return s, d, reqs


def measure_serve(local, scale, hub_degree, nreq, loads=(0.5, 0.8, 0.95)):
    """Requests arrive as a Poisson process at f x the capacity of the
    sequential plain path. Served: submitted to the request loop at their
    arrival times. Plain: the same trace handled one request at a time, in
    order, through the synchronous API with the level-synchronous engine.
    Latency = completion - arrival. Returns p50/p99 and throughput per load."""
    import threading
    import torch
    from paper_1802_03760_b300 import gj

    n = 1 << scale
    s, d, reqs = serve_trace(scale, 32, hub_degree, nreq)
    rng = np.random.default_rng(2)

    def fresh():
        ctx = gj.Context(local, engine=gj.ENGINE_PLAIN)
        g = gj.Graph(ctx, s, d, n)
        qmap = {nm: gj.Query(ctx, *QUERIES[nm]) for nm in BENCH_QUERIES}
        return ctx, g, qmap

    def run_plain(arrivals):
        ctx, g, qmap = fresh()
        t0 = time.perf_counter()
        lat, res = [], []
        for (kind, batch, names), a in zip(reqs, arrivals):
            now = time.perf_counter() - t0
            if now < a:
                time.sleep(a - now)
            qs = [qmap[nm] for nm in names]
            if kind == "count":
                r = gj.count_many(g, qs, engine=gj.ENGINE_PLAIN)
            else:
                r = gj.apply_batch(g, *batch, qs)
            res.append(r)
            lat.append((time.perf_counter() - t0 - a) * 1e3)
        span = time.perf_counter() - t0
        ctx.close()
        return lat, res, span

    def run_served(arrivals):
        ctx, g, qmap = fresh()
        srv = gj.Server(g)
        ids = [None] * len(reqs)
        sub_t = [0.0] * len(reqs)
        t0 = time.perf_counter()

        def submitter():
            for i, ((kind, batch, names), a) in enumerate(zip(reqs, arrivals)):
                now = time.perf_counter() - t0
                if now < a:
                    time.sleep(a - now)
                qs = [qmap[nm] for nm in names]
                ids[i] = srv.submit_count(qs) if kind == "count" else srv.submit_batch(*batch, qs)
                sub_t[i] = time.perf_counter() - t0

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        out = [srv.poll(i) for i in ids]
        srv.stop()
        ctx.close()
        # the loop's own clock gives each request's time in the system; add the
        # submitter's lag behind the arrival time
        lat = [(o["end_ms"] - o["submit_ms"]) + (st - a) * 1e3 for o, st, a in zip(out, sub_t, arrivals)]
        span = max(a + l / 1e3 for a, l in zip(arrivals, lat))
        res = [(o["counts"], o["checksums"]) for o in out]
        return lat, res, span

    clocks = ClockSampler(local).start()
    # capacity of the plain path: back-to-back service of the trace
    lat0, ref, span0 = run_plain([0.0] * len(reqs))
    capacity = len(reqs) / span0
    out = {}
    for f in loads:
        gaps = rng.exponential(1.0 / (f * capacity), len(reqs))
        arrivals = list(np.cumsum(gaps) - gaps[0])
        lp, rp, sp = run_plain(arrivals)
        ls, rs, ss = run_served(arrivals)
        if [tuple(map(tuple, r)) for r in rp] != [tuple(map(tuple, r)) for r in rs] or \
                [tuple(map(tuple, r)) for r in rp] != [tuple(map(tuple, r)) for r in ref]:
            raise RuntimeError("served results differ from the sequential plain path")
        out[str(f)] = {"arrival_rate_per_s": f * capacity,
                       "served": {"p50_ms": float(np.percentile(ls, 50)), "p99_ms": float(np.percentile(ls, 99)),
                                  "throughput_req_per_s": len(reqs) / ss},
                       "plain": {"p50_ms": float(np.percentile(lp, 50)), "p99_ms": float(np.percentile(lp, 99)),
                                 "throughput_req_per_s": len(reqs) / sp}}
    clk = clocks.stop()
    return {"metric": "p99 request latency (served vs sequential plain)", "unit": "ms",
            "workload": "serving: R-MAT scale %d + 32 hubs of out/in degree %d, %d requests (50%% counts of "
                        "triangle/diamond/4-clique, 50%% update batches of 1e3-1e5 edges), Poisson arrivals"
                        % (scale, hub_degree, len(reqs)),
            "plain_capacity_req_per_s": capacity, "loads": out, "clocks": clk,
            "results": "served results equal the sequential replay's, request by request"}


def run_serve(args):
    world, rank, local = dist_setup()
    import torch
    torch.cuda.set_device(local)
    scale = args.scale if args.scale != SCALE else 16
    r = measure_serve(local, scale, args.hub_degree, args.requests)
    if rank != 0:
        return 0
    mid = r["loads"]["0.8"]
    line = {"metric": "p99 request latency at 0.8 x plain capacity (served vs sequential plain)",
            "value": mid["served"]["p99_ms"], "unit": "ms", "n_gpus": world, "steps": args.requests, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": r["workload"], "plain_capacity_req_per_s": r["plain_capacity_req_per_s"],
                       "loads": r["loads"]},
            "plain_p99_ms": mid["plain"]["p99_ms"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def run_multi(args):
    """Batched uneven workload: 64 mixed queries (the five shapes and seeded
    variants) counted in one persistent launch over a first-attribute sample
    of an R-MAT graph, after the autotuner picks the launch settings on a
    smaller sample; the plain path counts the same queries one at a time."""
    import torch
    from paper_1802_03760_b300 import gj
    from paper_1802_03760_b300.inputs import mixed_queries

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    scale = args.scale if args.scale != SCALE else 24
    n = 1 << scale
    s, d = rmat_edges(scale, seed=1)
    stream = torch.cuda.Stream()
    ctx = gj.Context(local, stream=stream.cuda_stream)
    mq = mixed_queries(64, seed=1)
    qs = [gj.Query(ctx, k, at, o) for _, k, at, o in mq]
    ds = torch.from_numpy(s.view(np.int32)).cuda()
    dd = torch.from_numpy(d.view(np.int32)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = gj.Graph(ctx, ds, dd, n)
    build_s = time.perf_counter() - t0
    hi = max(1, min(n, args.sample_vertices))
    # launch settings chosen on the sample itself (untimed)
    tune = gj.autotune(g, qs, v_range=(0, hi), prefix_cap_bytes=2 << 30)
    times = []
    res = None
    for i in range(args.warmup + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = gj.count_many(g, qs, engine=gj.ENGINE_FUSED, v_range=(0, hi))
        e1.record(stream)
        e1.synchronize()
        if res is not None and r != res:
            raise RuntimeError("counts changed between steps")
        res = r
        if i >= args.warmup:
            times.append(e0.elapsed_time(e1))
    fms = sum(times) / len(times)
    matches = sum(res[0])
    plain = None
    if not args.no_plain:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rp = gj.count_many(g, qs, engine=gj.ENGINE_PLAIN, v_range=(0, hi))
        e1.record(stream)
        e1.synchronize()
        if rp != res:
            raise RuntimeError("plain and fused counts differ")
        pms = e0.elapsed_time(e1)
        # the fused engine one query at a time (no batching across queries)
        e0.record(stream)
        for q in qs:
            gj.count(g, q, engine=gj.ENGINE_FUSED, v_range=(0, hi))
        e1.record(stream)
        e1.synchronize()
        sms = e0.elapsed_time(e1)
        plain = {"ms": pms, "value": matches / (pms / 1e3), "fused_speedup": pms / fms,
                 "fused_one_query_at_a_time_ms": sms}
    by_shape = {}
    for (nm, _, _, _), c in zip(mq, res[0]):
        key = nm.split("-v")[0]
        by_shape[key] = by_shape.get(key, 0) + c
    if rank != 0:
        return 0
    line = {"metric": "matches/sec (64 mixed queries, one persistent launch)", "value": world * matches / (fms / 1e3),
            "unit": "matches/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": fms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "R-MAT scale %d (%d distinct edges), 64 queries (triangle, 4-cycle, diamond, "
                                   "4-clique, 5-clique and seeded direction/order variants), first attribute in "
                                   "[0, %d)" % (scale, g.m, hi),
                       "index_build_s": build_s, "tuning": tune, "matches_by_shape": by_shape},
            "plain": plain}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="0 skips the CPU baseline")
    ap.add_argument("--scale", type=int, default=SCALE, help="R-MAT scale (profiling runs use smaller ones)")
    ap.add_argument("--queries", default=",".join(BENCH_QUERIES))
    ap.add_argument("--workload", default="static", choices=["static", "delta", "serve", "multi"])
    ap.add_argument("--sample-vertices", type=int, default=64,
                    help="multi workload: first-attribute values [0, V) of the sample")
    ap.add_argument("--requests", type=int, default=120, help="serve workload: requests in the trace")
    ap.add_argument("--hub-degree", type=int, default=8192, help="serve workload: planted hub degree")
    ap.add_argument("--batch-sizes", default="1000,10000,100000", help="delta workload")
    ap.add_argument("--batches", type=int, default=20, help="delta workload: timed batches per size")
    ap.add_argument("--no-delta", action="store_true", help="static workload: skip the delta sub-record")
    ap.add_argument("--no-serve", action="store_true", help="static workload: skip the serving sub-record")
    ap.add_argument("--delta-batches", type=int, default=12, help="static workload: timed batches per size")
    ap.add_argument("--serve-requests", type=int, default=60, help="static workload: requests of the serving trace")
    args = ap.parse_args()
    args.queries = [q for q in args.queries.split(",") if q]
    for q in args.queries:
        if q not in QUERIES:
            ap.error("unknown query %r" % q)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "delta":
        return run_delta(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "multi":
        return run_multi(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
