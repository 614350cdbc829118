#!/usr/bin/env python
"""Benchmark of the Smith-Waterman/Gotoh hot path on one GB300 (or N replicas).

Default workload: the long DNA pair with full reconstruction -- sequence A of
200 kbp uniform ACGT, B = A's 150 kbp window mutated (10% substitutions, 2%
indels of geometric length, mean 3) between random flanks, match +1,
mismatch -3, gap open 5, gap extend 2 -- aligned with sw_align (score, end
cell, canonical CIGAR).  One step = one sw_align of that pair.  GCUPS counts
the m x n matrix cells per second (paper Section 4.2: GCUPS).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl swgb|reference]

Prints one JSON line (rank 0).  With --gpus N > 1 (launched by torchrun)
every rank runs its own replica of the workload ("replicas only": the
pairwise path has no exchange step); value = all ranks' cells / the
slowest rank's time.

--impl reference times the CPU oracle (oracle/, test infrastructure) on the
host cores, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2211_10769_gb300 import workloads as W  # noqa: E402

INT_LANES_PER_SM = 128          # 4 sub-partitions x 32 integer lanes
OPS_PER_CELL = 10               # E: 2 sub + max, F: 2 sub + max, H: add + 3 max (incl. 0), running max
WORKLOAD = "dna_pair_200kbp_align"
# DRAM traffic of the forward fill measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of one full-size launch) per cell, and the kernel
# sources it was taken on (None: not measured on the current kernel).
FILL_TRAFFIC = {"mode": "align", "bytes_per_cell": 395.31e6 / (200_000 * 200_000),
                "source_sha256": "3f0f0a5b28f5ef9f15e8d489472384b80bb35c223c097b602f4424626c8cbfac"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="swgb", choices=["swgb", "reference"])
    ap.add_argument("--length", type=int, default=200_000, help="length of sequence A")
    ap.add_argument("--cpu-sample-rows", type=int, default=12_000,
                    help="rows of A the CPU baseline aligns against all of B")
    ap.add_argument("--mode", default="align", choices=["align", "score"],
                    help="align: sw_align per step (default); score: sw_score per step (profiling)")
    ap.add_argument("--no-extras", action="store_true", help="skip the instruction-rate probe")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the timed CPU oracle sample")
    ap.add_argument("--workloads", default="all",
                    help="comma list of the other workloads to measure after the headline: "
                         "dna2k,variants,dbsearch,batch,serve,dna5m,bounded (default all; 'none' for the headline only)")
    ap.add_argument("--serve-requests", type=int, default=500, help="requests per arrival rate")
    ap.add_argument("--db-subjects", type=int, default=500_000,
                    help="subjects of the search database (fewer only for profiling captures)")
    ap.add_argument("--bounded-length", type=int, default=5_000_000,
                    help="length of the long pair aligned under a small checkpoint budget")
    ap.add_argument("--bounded-budget-mb", type=int, default=1024, help="that checkpoint budget (MB)")
    ap.add_argument("--serve-rates", default="10,20,50,2000",
                    help="arrival rates (requests/s): below, near and above the device's capacity")
    return ap.parse_args()


def slowest_rank_time(total, world, device):
    """Timed-region seconds of the slowest rank (every rank gets it): replicas
    run independently, so the job is done when the last one is."""
    if world <= 1:
        return total
    import torch
    import torch.distributed as dist
    t = torch.tensor([total], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_rate(units_per_rank, world, slowest_total, steps):
    """Units per second of the whole job: every rank's units over the slowest rank's time per step."""
    return world * units_per_rank / (slowest_total / steps)


def dist_init(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if n > 0 else "gloo")
    return rank, world


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_swgb(args, rank, world):
    import torch
    from paper_2211_10769_gb300 import binding, build
    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ctx = binding.Context(dev, stream)
    sc = W.dna_scoring()
    A, B = W.dna_long_pair(args.length)
    m, n = len(A), len(B)
    cells = m * n
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    def step():
        if args.mode == "score":
            h = ctx.score(dA, dB, sc.matrix, sc.gap_open, sc.gap_extend)
            return binding.Alignment(h.score, 0, h.a_end, 0, h.b_end, "")
        return ctx.align(dA, dB, sc.matrix, sc.gap_open, sc.gap_extend)

    # the clock sampler (an nvidia-smi process) starts before the warm-up steps, so that its
    # start-up never falls inside the timed region
    clocks = ClockSampler(dev)
    clocks.start()
    ref_aln = None
    # per-kernel device time on the context stream; enabled during the warm-up too, so that
    # the context creates its event pool before the timed region
    ctx.timing(True)
    for _ in range(args.warmup):
        ref_aln = step()
    if ref_aln is None:
        ref_aln = step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()

    ctx.timing(True)                 # clears the totals
    launches0 = ctx.launches()
    times = []
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        aln = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        assert aln == ref_aln
    torch.cuda.synchronize()
    launches = ctx.launches() - launches0
    kt = {name: ctx.kernel_time(kind) for name, kind in
          (("fill", binding.KT_FILL), ("fill_tb", binding.KT_FILL_TB), ("walk", binding.KT_WALK))}
    ctx.timing(False)
    total = slowest_rank_time(sum(times), world, "cuda")

    # dominant kernel: the forward wavefront fill, timed alone through sw_score
    fill_times = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hit = ctx.score(dA, dB, sc.matrix, sc.gap_open, sc.gap_extend)
        e1.record(stream)
        e1.synchronize()
        fill_times.append(e0.elapsed_time(e1) / 1e3)
    clk = clocks.stop()
    assert (hit.score, hit.a_end, hit.b_end) == (ref_aln.score, ref_aln.a_end, ref_aln.b_end)

    # end to end through the public API with the inputs in pinned host memory: every call copies
    # them to the device and its result back inside the timed region
    hA, hB = torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory()
    e2e = []
    for _ in range(max(3, min(args.steps, 10))):
        t0 = time.perf_counter()
        if args.mode == "score":
            h = ctx.score(hA, hB, sc.matrix, sc.gap_open, sc.gap_extend)
            aln = binding.Alignment(h.score, 0, h.a_end, 0, h.b_end, "")
        else:
            aln = ctx.align(hA, hB, sc.matrix, sc.gap_open, sc.gap_extend)
        e2e.append(time.perf_counter() - t0)
    assert (aln.score, aln.cigar) == (ref_aln.score, ref_aln.cigar)
    d2h = 48 + len(aln.cigar)

    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or device_max_sm_mhz()
    peak_ops = nsm * INT_LANES_PER_SM * max_mhz * 1e6
    score_t = statistics.mean(fill_times)
    # the dominant kernel: the forward fill (one launch per step), timed by
    # events recorded around its launches inside the timed steps
    fill_ms, fill_n = kt["fill"]
    fill_t = fill_ms / 1e3 / max(1, fill_n)
    achieved = OPS_PER_CELL * cells / fill_t
    probe = {}
    if not args.no_extras:
        from paper_2211_10769_gb300.binding import probe_int_rates
        probe = probe_int_rates(ctx)
    out = {
        "metric": "GCUPS on 1 GB300 (exact scores); batched vs per-pair GCUPS; p50/p99 latency",
        "value": round(whole_job_rate(cells, world, total, args.steps) / 1e9, 2),
        "unit": "GCUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * total / args.steps, 3),
        "ms_per_step_median": round(1e3 * statistics.median(times), 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (seeded generator; paper's genome pairs unavailable)",
        "config": {"workload": WORKLOAD if args.mode == "align" else WORKLOAD.replace("align", "score"), "m": m, "n": n, "scoring": "+1/-3, open 5, extend 2",
                   "call": "sw_align (score + canonical CIGAR)" if args.mode == "align" else "sw_score", "l2": "flushed (512 MB write) before each step",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "result": {"score": ref_aln.score, "a": [ref_aln.a_begin, ref_aln.a_end],
                              "b": [ref_aln.b_begin, ref_aln.b_end], "cigar_len": len(ref_aln.cigar)}},
        "gpu_launches": launches,
        "e2e": {"value": round(cells / statistics.median(e2e) / 1e9, 2), "unit": "GCUPS",
                "h2d_bytes_per_step": m + n, "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu",
                     "kernel": "wavefront16_kernel (packed 16-bit pair fill), forward fill (%s mode)" % (
                         "checkpoint" if args.mode == "align" else "score"),
                     "achieved": round(achieved / 1e12, 3), "peak": round(peak_ops / 1e12, 3),
                     "unit": "Tint-op/s", "frac": round(achieved / peak_ops, 4),
                     "traffic": fill_traffic(m, n, args.mode),
                     "ops_per_cell": OPS_PER_CELL, "fill_ms": round(1e3 * fill_t, 3),
                     "fill_launches": fill_n, "fill_gcups": round(cells / fill_t / 1e9, 2),
                     "score_call_gcups": round(cells / score_t / 1e9, 2),
                     "peak_basis": "%d SMs x 128 int32 lanes x %.0f MHz (SM count from the device, "
                                   "maximum SM clock from nvidia-smi; plain integer ALU issue)" % (nsm, max_mhz)},
        "kernel_ms_per_step": {k: round(v[0] / max(1, args.steps), 3) for k, v in kt.items()},
        "clocks": clk,
    }
    if probe:
        out["roofline"]["measured_int_rates_per_sm_clk"] = probe
    return out


def device_max_sm_mhz():
    """Maximum SM clock of GPU 0 as nvidia-smi reports it (2070 MHz on GB300 if it cannot be read)."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip().splitlines()
        return float(out[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return 2070.0


def fill_traffic(m, n, mode):
    """DRAM bytes (read + write) of one forward-fill launch: an ncu capture
    of dram__bytes_read.sum + dram__bytes_write.sum on the full-size launch,
    scaled by cells; None when none was taken on the current kernel sources."""
    if FILL_TRAFFIC is None or mode != FILL_TRAFFIC["mode"]:
        return None
    import hashlib
    h = hashlib.sha256()
    for f in ("wavefront16.cuh", "wavefront.cuh", "sw_device.cuh"):
        with open(os.path.join(ROOT, "paper_2211_10769_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != FILL_TRAFFIC["source_sha256"]:
        return None
    return int(FILL_TRAFFIC["bytes_per_cell"] * m * n)


def run_reference(args, rank, world):
    """CPU oracle on a bounded sample: the first --cpu-sample-rows rows of A against all of B."""
    from oracle import oracle
    sc = W.dna_scoring()
    A, B = W.dna_long_pair(args.length)
    rows = min(args.cpu_sample_rows, len(A))
    a = A[:rows]
    times = []
    oracle.sw_score(a[:100], B[:100], sc.matrix, sc.gap_open, sc.gap_extend)
    for _ in range(args.warmup):
        oracle.sw_score(a[:1000], B, sc.matrix, sc.gap_open, sc.gap_extend)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sw_score(a, B, sc.matrix, sc.gap_open, sc.gap_extend)
        times.append(time.perf_counter() - t0)
    cells = rows * len(B)
    gcups = cells / statistics.mean(times) / 1e9
    sample = "score-only oracle, rows 0..%d of A (%d x %d = %.2e cells) per step" % (rows, rows, len(B), cells)
    return {
        "metric": "GCUPS on 1 GB300 (exact scores); batched vs per-pair GCUPS; p50/p99 latency",
        "impl": "reference",
        "value": round(gcups, 4), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(times), 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "m": len(A), "n": len(B)},
        "cpu_baseline": {"value": round(gcups, 4), "unit": "GCUPS", "cores": 1, "kind": "oracle",
                         "host_cores": os.cpu_count(), "sample": sample},
        "e2e": {"value": round(gcups, 4), "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def cpu_baseline_leg(args):
    """The oracle timed on a bounded sample (about 10-30 s of CPU work)."""
    from oracle import oracle
    sc = W.dna_scoring()
    A, B = W.dna_long_pair(args.length)
    rows = min(args.cpu_sample_rows, len(A))
    t0 = time.perf_counter()
    oracle.sw_score(A[:rows], B, sc.matrix, sc.gap_open, sc.gap_extend)
    dt = time.perf_counter() - t0
    return {"value": round(rows * len(B) / dt / 1e9, 4), "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "host_cores": os.cpu_count(),
            "sample": "score-only oracle on rows 0..%d of A against all of B (%.2e cells, %.1f s); one pair "
                      "is one dynamic programme, so one core" % (rows, rows * len(B), dt)}


def _threaded_oracle(jobs, fn):
    """Run fn over jobs on every host core (the oracle is a ctypes call, which
    releases the interpreter lock, so threads run it in parallel); returns
    (seconds, threads)."""
    from concurrent.futures import ThreadPoolExecutor
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(fn, jobs))
    return time.perf_counter() - t0, threads


def cpu_workload_legs(wl):
    """The oracle timed on seeded samples of the database search and of the
    batch, over all host cores (threads over subjects / pairs), in GCUPS."""
    from oracle import oracle
    from paper_2211_10769_gb300 import bench_workloads as BW
    out = {}
    g = np.random.default_rng(W.BASE_SEED + 99)
    if "dbsearch" in wl:
        sc = W.protein_scoring()
        qs, pdb = BW._protein_db()
        q = qs[2]                                        # the 1,000-residue query
        subj = sorted(g.choice(pdb.nseq, size=20_000, replace=False).tolist())
        cells = len(q) * sum(len(pdb.subject(s)) for s in subj)
        dt, th = _threaded_oracle(subj, lambda s: oracle.sw_score(q, pdb.subject(s), sc.matrix, sc.gap_open,
                                                                   sc.gap_extend))
        out["dbsearch"] = {"value": round(cells / dt / 1e9, 3), "unit": "GCUPS", "cores": th, "kind": "oracle",
                           "sample": "query of %d residues against 20,000 seeded subjects of the database "
                                     "(%.2e cells, %.1f s)" % (len(q), cells, dt)}
    if "batch" in wl:
        d, p = W.dna_scoring(), W.protein_scoring()
        scs = [(d.matrix, d.gap_open, d.gap_extend), (p.matrix, p.gap_open, p.gap_extend)]
        ks = sorted(g.choice(10_000, size=300, replace=False).tolist())
        pairs = [W.batch_pair(k) for k in ks]
        cells = sum(len(a) * len(b) for a, b, _ in pairs)
        dt, th = _threaded_oracle(pairs, lambda x: oracle.sw_score(x[0], x[1], *scs[0 if x[2] == "dna" else 1]))
        out["batch"] = {"value": round(cells / dt / 1e9, 3), "unit": "GCUPS", "cores": th, "kind": "oracle",
                        "sample": "300 seeded pairs of the 10,000 (%.2e cells, %.1f s)" % (cells, dt)}
    return out


def main():
    args = parse()
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    out = run_swgb(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_leg(args)
        wl = [] if args.workloads == "none" else (
            ["dna2k", "variants", "dbsearch", "batch", "serve", "dna5m", "bounded"] if args.workloads == "all"
            else args.workloads.split(","))
        if wl and args.mode == "align":
            from paper_2211_10769_gb300 import bench_workloads as BW
            out["workloads"] = BW.run_all(wl, args)
            if not args.no_cpu_baseline:
                for nm, leg in cpu_workload_legs(wl).items():
                    out["workloads"][nm]["cpu_baseline"] = leg
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
