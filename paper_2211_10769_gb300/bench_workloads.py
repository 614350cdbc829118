"""Measurements of the non-headline workloads for bench.py.

Each function times one workload through the public API on cuda:0 with
CUDA events on the context's stream and returns a small dict:

* dna2k    -- sw_align of the 2,000 x 2,000 DNA pair;
* dbsearch -- sw_dbsearch of the five protein queries (144 .. 5,478) against
              the 500,000-subject database (top-20), plus its kernel's
              share of the integer peak;
* variants -- sw_align of the 2 kbp and 200 kbp DNA pairs with each of the
              four algorithms (local, global, semi-global, overlap);
* batch    -- sw_batch (one graph-captured, autotuned launch) over the 10,000
              uneven pairs versus one sw_score call per pair;
* serve    -- the continuous-batching server under Poisson arrivals at each
              rate: p50 / p99 latency (arrival to result on the host),
              sustained GCUPS, admitted / deferred submissions;
* dna5m    -- sw_align of the 5 Mbp x 5 Mbp variant of the long DNA pair.
"""
from __future__ import annotations

import hashlib
import statistics
import time

import numpy as np

from . import workloads as W

OPS_PER_CELL = 10
REPEATS = 20                  # timed runs per measurement: median and mean are reported


_DB_CACHE = {}


def _protein_db(nseq=500_000):
    """The database (500,000 subjects unless a profiling run asks for fewer) with the five
    planted queries (generated once)."""
    if nseq not in _DB_CACHE:
        qs = W.protein_queries()
        _DB_CACHE[nseq] = (qs, W.protein_db(nseq, queries=qs))
    return _DB_CACHE[nseq]


def _stats(ts):
    """Median and mean of a list of seconds."""
    return statistics.median(ts), statistics.mean(ts)


def _int_peak(torch):
    """Integer-lane issue peak (lanes / s): SMs x 128 x the maximum SM clock."""
    import subprocess
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    try:
        mhz = float(subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                                   capture_output=True, text=True, timeout=20).stdout.split()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        mhz = 2070.0
    return nsm * 128 * mhz * 1e6


def _timed(torch, stream, fn, reps):
    out = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1) / 1e3)
    return out


def dna2k(ctx, torch, stream, args):
    sc = W.dna_scoring()
    a, b = W.dna_pair_2k()
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    ctx.align(da, db, sc.matrix, sc.gap_open, sc.gap_extend)
    ts = _timed(torch, stream, lambda: ctx.align(da, db, sc.matrix, sc.gap_open, sc.gap_extend), 20)
    t = statistics.median(ts)
    return {"workload": "dna_pair_2kbp_align", "cells": len(a) * len(b), "ms_median": round(1e3 * t, 3),
            "gcups": round(len(a) * len(b) / t / 1e9, 2)}


def variants(ctx, torch, stream, args):
    """sw_align of the 2 kbp pair and of the 200 kbp pair with each algorithm of paper Section 2.1."""
    from .binding import KT_FILL
    sc = W.dna_scoring()
    out = {}
    for name, alg in (("local", 0), ("global", 1), ("semiglobal", 2), ("overlap", 3)):
        row = {}
        for tag, (a, b), reps in (("dna2k", W.dna_pair_2k(), REPEATS), ("dna200k", W.dna_long_pair(200_000), 5)):
            da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
            aln = ctx.align(da, db, sc.matrix, sc.gap_open, sc.gap_extend, algorithm=alg)
            ctx.timing(True)
            ts = _timed(torch, stream, lambda: ctx.align(da, db, sc.matrix, sc.gap_open, sc.gap_extend,
                                                         algorithm=alg), reps)
            fms, fn = ctx.kernel_time(KT_FILL)
            ctx.timing(False)
            t = statistics.median(ts)
            row[tag] = {"ms": round(1e3 * t, 3), "gcups": round(len(a) * len(b) / t / 1e9, 1),
                        "fill_gcups": round(len(a) * len(b) / (fms / 1e3 / max(1, fn)) / 1e9, 1),
                        "score": aln.score, "a": [aln.a_begin, aln.a_end], "b": [aln.b_begin, aln.b_end]}
        out[name] = row
    return {"workload": "dna_pairs_by_algorithm", "call": "sw_align", "timing": "CUDA events, median", **out}


def dbsearch(ctx, torch, stream, args):
    from .binding import Database
    sc = W.protein_scoring()
    qs, pdb = _protein_db(args.db_subjects)
    db = Database(ctx, pdb.residues, pdb.offsets)
    total_res = int(pdb.residues.size)
    from .binding import KT_DB16
    per_query = []
    kern_s = 0.0
    for q in qs:
        db.search(q, sc.matrix, sc.gap_open, sc.gap_extend, k=20)
        ctx.timing(True)
        ts = _timed(torch, stream, lambda: db.search(q, sc.matrix, sc.gap_open, sc.gap_extend, k=20), REPEATS)
        kms, kn = ctx.kernel_time(KT_DB16)
        ctx.timing(False)
        t, tm = _stats(ts)
        kern_s += kms / 1e3 / max(1, kn)
        per_query.append({"m": len(q), "ms": round(1e3 * t, 2), "ms_mean": round(1e3 * tm, 2),
                          "gcups": round(len(q) * total_res / t / 1e9, 1), "fill_ms": round(kms / max(1, kn), 2)})
    cells = sum(len(q) for q in qs) * total_res
    t_all = sum(x["ms"] for x in per_query) / 1e3
    peak16 = _int_peak(torch) * 2                         # two 16-bit lanes per 32-bit lane
    db.close()
    # the packed fill reads every subject residue once per query sweep (1 B per residue)
    return {"workload": "protein_dbsearch_5q_x_500k", "nseq": pdb.nseq, "residues": total_res,
            "cells": cells, "seconds": round(t_all, 3), "gcups": round(cells / t_all / 1e9, 1),
            "timing": "CUDA events, median of %d searches per query" % REPEATS, "per_query": per_query,
            "alu_frac_16bit_lanes": round(OPS_PER_CELL * cells / t_all / peak16, 4),
            "fill_hbm_gbs": round(len(qs) * total_res / kern_s / 1e9, 1)}


def batch(ctx, torch, stream, args):
    from . import binding
    d, p = W.dna_scoring(), W.protein_scoring()
    scorings = [(d.matrix, d.gap_open, d.gap_extend), (p.matrix, p.gap_open, p.gap_extend)]
    raw = W.batch_pairs(10_000)
    pairs = [(a, b, 0 if kind == "dna" else 1) for a, b, kind in raw]
    cells = sum(len(a) * len(b) for a, b, _ in pairs)
    ares, aoff, bres, boff, sidx = binding.Batch.packed(pairs)
    dev = (torch.from_numpy(ares).cuda(), torch.from_numpy(bres).cuda())
    plan = binding.Batch(ctx, pairs, scorings, flags=binding.SW_BATCH_GRAPH | binding.SW_BATCH_AUTOTUNE,
                         device_inputs=dev)
    plan.run()
    ts = _timed(torch, stream, plan.run, REPEATS)        # (the plan's own stream, joined by the host copy)
    t_batch, t_mean = _stats(ts)
    cfg = plan.config()
    bins = plan.bins()
    plan.close()
    # one sw_score launch per pair, inputs already on the device
    dpairs = []
    for k, (a, b, si) in enumerate(pairs):
        dpairs.append((dev[0][int(aoff[k]):int(aoff[k + 1])], dev[1][int(boff[k]):int(boff[k + 1])], si))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a, b, si in dpairs:
        mat, go, ge = scorings[si]
        ctx.score(a, b, mat, go, ge)
    t_pair = time.perf_counter() - t0
    return {"workload": "batch_10k_uneven_pairs", "cells": cells, "batched_s": round(t_batch, 4),
            "batched_s_mean": round(t_mean, 4),
            "batched_gcups": round(cells / t_batch / 1e9, 1), "per_pair_s": round(t_pair, 3),
            "per_pair_gcups": round(cells / t_pair / 1e9, 1), "speedup": round(t_pair / t_batch, 2),
            "tile": {"rows_per_lane": cfg[0], "warps": cfg[1]},
            "bins": [{"rows_per_lane": r, "warps": w, "lane_bits": lb, "pairs": npr} for r, w, lb, npr in bins],
            "timing": "CUDA events around each run (its results copied to the host inside), median of %d; "
                      "per pair: one pass of 10,000 sw_score calls, wall clock" % REPEATS}


# the server sweeps the database in 4 chunks: with pipelined steps, 4 sustain the serial search's
# rate on the same requests (8: 99.4 - 99.8% of it) and still admit a request every quarter sweep
SERVE_CHUNKS = 4


def serve(ctx, torch, stream, args):
    from . import binding
    sc = W.protein_scoring()
    qs, pdb = _protein_db(args.db_subjects)
    db = binding.Database(ctx, pdb.residues, pdb.offsets)
    total_res = int(pdb.residues.size)
    rates = [float(x) for x in args.serve_rates.split(",")]
    # the requests of the highest rate searched one at a time with sw_dbsearch: the serial rate
    # the server's continuous batching is compared with, on the same queries, and the device's
    # capacity for such requests (above it a queue grows)
    sample = [q for _, q in W.serving_requests(args.serve_requests, max(rates))]
    db.search(sample[0], sc.matrix, sc.gap_open, sc.gap_extend, k=20)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q in sample:
        db.search(q, sc.matrix, sc.gap_open, sc.gap_extend, k=20)
    serial_s = time.perf_counter() - t0
    serial_gcups = round(sum(len(q) for q in sample) * total_res / serial_s / 1e9, 1)
    out = []
    for rate in rates:
        reqs = W.serving_requests(args.serve_requests, rate)
        srv = binding.Server(ctx, db, sc.matrix, sc.gap_open, sc.gap_extend, mem_budget=8 << 30, k=20,
                             max_slots=64, chunks=SERVE_CHUNKS)
        queue, inflight, lat = [], {}, []
        deferred = 0
        nxt, ndone, steps = 0, 0, 0
        t0 = time.perf_counter()
        busy = 0.0
        while ndone < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt][0] <= now:
                queue.append(nxt)
                nxt += 1
            while queue:
                t = srv.submit(reqs[queue[0]][1])
                if t is None:
                    deferred += 1
                    break
                inflight[t] = queue.pop(0)
            if inflight:
                s0 = time.perf_counter()
                srv.step()
                busy += time.perf_counter() - s0
                steps += 1
                done_now = time.perf_counter() - t0
                for t, i in list(inflight.items()):
                    r = srv.poll(t)
                    if r is not None:
                        lat.append(done_now - reqs[i][0])
                        del inflight[t]
                        ndone += 1
            elif nxt < len(reqs):
                time.sleep(max(0.0, min(0.01, reqs[nxt][0] - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
        cells = sum(len(q) for _, q in reqs) * total_res
        srv.close()
        lat.sort()
        out.append({"rate_per_s": rate, "requests": len(reqs), "p50_s": round(float(np.percentile(lat, 50)), 3),
                    "p99_s": round(float(np.percentile(lat, 99)), 3), "sustained_gcups": round(cells / wall / 1e9, 1),
                    "busy_gcups": round(cells / busy / 1e9, 1), "steps": steps, "deferred_submits": deferred,
                    "offered_gcups": round(rate * cells / len(reqs) / 1e9, 1)})
        out[-1]["load"] = "overload" if out[-1]["offered_gcups"] > serial_gcups else "below capacity"
    db.close()
    return {"workload": "serving_poisson_protein_vs_500k", "chunks": SERVE_CHUNKS, "max_slots": 64, "k": 20,
            "serial_dbsearch_gcups": serial_gcups,
            "serial_note": "the highest rate's requests, one sw_dbsearch call each, wall clock",
            "note": "load = offered GCUPS (rate x mean cells per request) against the serial rate (the device's "
                    "capacity for these requests); under overload latency is queue-dominated.  busy_gcups: cells "
                    "over the host's time inside step() calls; steps are pipelined, so the device also works "
                    "while the host admits and polls, and under overload it exceeds the device's rate",
            "rates": out}


def dna5m(ctx, torch, stream, args):
    """The 5 Mbp x 5 Mbp variant of the long pair: one warm-up and one timed sw_align."""
    from .binding import KT_FILL, KT_FILL_TB, KT_WALK
    sc = W.dna_scoring()
    A, B = W.dna_long_pair(5_000_000)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ref = ctx.align(dA, dB, sc.matrix, sc.gap_open, sc.gap_extend)
    ctx.timing(True)
    ts = _timed(torch, stream, lambda: ctx.align(dA, dB, sc.matrix, sc.gap_open, sc.gap_extend), 1)
    k = {nm: ctx.kernel_time(kind) for nm, kind in (("fill", KT_FILL), ("fill_tb", KT_FILL_TB), ("walk", KT_WALK))}
    ctx.timing(False)
    t = ts[0]
    cells = len(A) * len(B)
    return {"workload": "dna_pair_5mbp_align", "m": len(A), "n": len(B), "cells": cells,
            "seconds": round(t, 3), "gcups": round(cells / t / 1e9, 1),
            "kernel_s": {nm: round(v[0] / 1e3, 3) for nm, v in k.items()},
            "result": {"score": ref.score, "a": [ref.a_begin, ref.a_end], "b": [ref.b_begin, ref.b_end],
                       "cigar_len": len(ref.cigar), "cigar_sha256": hashlib.sha256(ref.cigar.encode()).hexdigest()}}


def bounded(ctx, torch, stream, args):
    """sw_align of the long pair (default 5 Mbp) under a small checkpoint budget (two checkpoint
    levels): one timed call in a context of its own, and the device memory that context holds."""
    import os
    from .binding import Context, KT_FILL, KT_FILL_TB, KT_WALK
    sc = W.dna_scoring()
    A, B = W.dna_long_pair(args.bounded_length)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    old = os.environ.get("SWGB_CKPT_BUDGET_MB")
    os.environ["SWGB_CKPT_BUDGET_MB"] = str(args.bounded_budget_mb)
    try:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        bctx = Context(0, stream)
    finally:
        if old is None:
            del os.environ["SWGB_CKPT_BUDGET_MB"]
        else:
            os.environ["SWGB_CKPT_BUDGET_MB"] = old
    try:
        bctx.timing(True)
        got = []
        ts = _timed(torch, stream, lambda: got.append(bctx.align(dA, dB, sc.matrix, sc.gap_open, sc.gap_extend)), 1)
        k = {nm: bctx.kernel_time(kind) for nm, kind in (("fill", KT_FILL), ("fill_tb", KT_FILL_TB),
                                                        ("walk", KT_WALK))}
        aln = got[0]
        free1, _ = torch.cuda.mem_get_info()
    finally:
        bctx.close()
    t = ts[0]
    cells = len(A) * len(B)
    return {"workload": "dna_pair_long_align_bounded_memory", "m": len(A), "n": len(B), "cells": cells,
            "checkpoint_budget_mb": args.bounded_budget_mb,
            "context_device_mb": round((free0 - free1) / 2**20, 1),
            "seconds": round(t, 3), "gcups": round(cells / t / 1e9, 1),
            "kernel_s": {nm: round(v[0] / 1e3, 3) for nm, v in k.items()},
            "note": "fill counts the forward fill and the coarse tiles' refills",
            "result": {"score": aln.score, "a": [aln.a_begin, aln.a_end], "b": [aln.b_begin, aln.b_end],
                       "cigar_len": len(aln.cigar), "cigar_sha256": hashlib.sha256(aln.cigar.encode()).hexdigest()}}


def run_all(names, args):
    import torch
    from .binding import Context
    stream = torch.cuda.current_stream()
    ctx = Context(0, stream)
    res = {}
    for nm in names:
        fn = {"dna2k": dna2k, "variants": variants, "dbsearch": dbsearch, "batch": batch, "serve": serve,
              "dna5m": dna5m, "bounded": bounded}[nm]
        t0 = time.perf_counter()
        try:
            res[nm] = fn(ctx, torch, stream, args)
        except Exception as exc:  # noqa: BLE001 - report, keep the headline line
            res[nm] = {"error": repr(exc)}
        res[nm]["bench_wall_s"] = round(time.perf_counter() - t0, 1)
    ctx.close()
    return res
