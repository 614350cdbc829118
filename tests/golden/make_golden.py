"""Write the stored expected values of the full-size pairwise workloads.

Calls only the CPU oracle (oracle/) on the seeded synthetic inputs of
paper_2211_10769_gb300.workloads and writes one JSON file per workload:

    python tests/golden/make_golden.py dna_2k          # 2,000 x 2,000 DNA pair (seconds)
    python tests/golden/make_golden.py dna_200k        # 200 kbp pair: ~40 GB RAM, minutes

The 200 kbp pair is aligned with the traceback-pointer form of the oracle
(one byte per cell).  The CIGAR itself is stored as its SHA-256 plus its
first and last 120 characters, which keeps the fixture small while still
pinning every operation.
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_2211_10769_gb300 import workloads as W  # noqa: E402


def record(name, a, b, sc, aln, seconds):
    cig = aln.cigar
    return {
        "workload": name,
        "m": int(len(a)), "n": int(len(b)),
        "gap_open": sc.gap_open, "gap_extend": sc.gap_extend,
        "score": aln.score, "a_begin": aln.a_begin, "a_end": aln.a_end,
        "b_begin": aln.b_begin, "b_end": aln.b_end,
        "cigar_len": len(cig), "cigar_sha256": hashlib.sha256(cig.encode()).hexdigest(),
        "cigar_head": cig[:120], "cigar_tail": cig[-120:],
        "oracle_seconds": round(seconds, 1),
        "generator": "paper_2211_10769_gb300.workloads (base seed %d)" % W.BASE_SEED,
    }


def main(which):
    sc = W.dna_scoring()
    if which == "dna_2k":
        a, b = W.dna_pair_2k()
        fn = oracle.sw_align
    elif which == "dna_200k":
        a, b = W.dna_long_pair(200_000)
        fn = oracle.sw_align_ptr
    else:
        raise SystemExit("unknown workload %r" % which)
    t = time.time()
    aln = fn(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    rec = record(which, a, b, sc, aln, time.time() - t)
    path = os.path.join(HERE, "%s.json" % which)
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(path, rec["score"], rec["oracle_seconds"], "s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "dna_2k")
