"""Seeded synthetic inputs and scoring tables.

This module holds input data only -- alphabets, substitution tables and the
seeded generators of the five workloads -- and none of the alignment
arithmetic.  Both the CUDA library's tests/benchmarks and the CPU oracle's
tests draw their inputs from here, so the two sides see identical bytes.

The paper's datasets (UniProtKB/Swiss-Prot 2022_07, Env. NR 2021_04, the 20
Swiss-Prot queries and the bacterial genome pairs of Table 2; Section 3.2)
are not available, so every workload below is a synthetic stand-in with the
paper's shapes and sizes.  Base seed 20221119; item k of a workload uses
seed BASE_SEED + k (plus a per-workload offset where a workload draws
several independent streams).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 20221119

DNA_ALPHABET = "ACGT"
PROTEIN_ALPHABET = "ARNDCQEGHILKMFPSTWYVBZX*"

# BLOSUM62 (Henikoff & Henikoff, PNAS 89:10915, 1992), in the 24-letter order
# and half-bit units of the matrix file NCBI distributes with BLAST.  Rows and
# columns follow PROTEIN_ALPHABET.
_BLOSUM62_ROWS = """
 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0 -2 -1  0 -4
-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3 -1  0 -1 -4
-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3  3  0 -1 -4
-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3  4  1 -1 -4
 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1 -3 -3 -2 -4
-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2  0  3 -1 -4
-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3 -1 -2 -1 -4
-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3  0  0 -1 -4
-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3 -3 -3 -1 -4
-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1 -4 -3 -1 -4
-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2  0  1 -1 -4
-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1 -3 -1 -1 -4
-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1 -3 -3 -1 -4
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2 -2 -1 -2 -4
 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2  0  0  0 -4
 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0 -1 -1  0 -4
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3 -4 -3 -2 -4
-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1 -3 -2 -1 -4
 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4 -3 -2 -1 -4
-2 -1  3  4 -3  0  1 -1  0 -3 -4  0 -3 -3 -2  0 -1 -4 -3 -3  4  1 -1 -4
-1  0  0  1 -3  3  4 -2  0 -3 -3  1 -1 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -1 -1 -1 -2 -1 -1 -1 -1 -1 -1 -1 -1 -1 -2  0  0 -2 -1 -1 -1 -1 -1 -4
-4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4  1
"""


def blosum62() -> np.ndarray:
    """24 x 24 int8 BLOSUM62 in PROTEIN_ALPHABET order."""
    vals = [int(t) for t in _BLOSUM62_ROWS.split()]
    return np.array(vals, dtype=np.int8).reshape(24, 24)


def dna_matrix(match: int = 1, mismatch: int = -3) -> np.ndarray:
    """4 x 4 match/mismatch table over ACGT (the paper's DNA scheme is +1/-3)."""
    m = np.full((4, 4), mismatch, dtype=np.int8)
    np.fill_diagonal(m, match)
    return m


# Background amino-acid frequencies of Robinson & Robinson (PNAS 88:8880,
# 1991), the composition BLAST uses, over the 20 standard letters in
# PROTEIN_ALPHABET order.
_ROBINSON = np.array([0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295,
                      0.07377, 0.02199, 0.05142, 0.09019, 0.05744, 0.02243, 0.03856,
                      0.05203, 0.07120, 0.05841, 0.01330, 0.03216, 0.06441])


def aa_background() -> np.ndarray:
    p = _ROBINSON / _ROBINSON.sum()
    return p


@dataclass(frozen=True)
class Scoring:
    """A substitution table plus positive gap penalties (gap of k costs open + (k-1)*extend)."""
    matrix: np.ndarray
    gap_open: int
    gap_extend: int

    @property
    def alphabet(self) -> int:
        return int(self.matrix.shape[0])


def dna_scoring() -> Scoring:
    """+1 / -3, gap open 5, gap extend 2 (paper Section 3.2, DNA runs)."""
    return Scoring(dna_matrix(1, -3), 5, 2)


def protein_scoring(gap_open: int = 10, gap_extend: int = 1) -> Scoring:
    """BLOSUM62 with open 10 / extend 1 (the protein workload's setting)."""
    return Scoring(blosum62(), gap_open, gap_extend)


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def uniform_dna(length: int, seed: int) -> np.ndarray:
    return rng(seed).integers(0, 4, size=length, dtype=np.uint8)


def random_protein(length: int, seed: int) -> np.ndarray:
    """i.i.d. residues over the 20 standard letters with background frequencies."""
    return rng(seed).choice(20, size=length, p=aa_background()).astype(np.uint8)


def mutate(seq: np.ndarray, alphabet_size: int, seed: int, p_sub: float = 0.10,
           p_indel: float = 0.02 / 3, mean_indel: float = 3.0) -> np.ndarray:
    """Homologous copy of ``seq``.

    Per base: a substitution with probability p_sub (to one of the other
    letters, uniformly); independently an indel event with probability
    p_indel, insertion or deletion with equal odds, of geometric length on
    {1, 2, ...} with the given mean (inserted letters uniform).  With the
    defaults about 2% of bases fall in indels (10% substitutions, 2% indels,
    mean indel length 3).
    """
    g = rng(seed)
    n = len(seq)
    sub = g.random(n) < p_sub
    shift = g.integers(1, alphabet_size, size=n)
    out_base = np.where(sub, (seq.astype(np.int64) + shift) % alphabet_size, seq).astype(np.uint8)
    ev = g.random(n) < p_indel
    kind = g.random(n) < 0.5
    lens = g.geometric(1.0 / mean_indel, size=n)
    pieces = []
    evpos = np.flatnonzero(ev)
    e = 0
    k = 0
    while k < n:
        while e < len(evpos) and evpos[e] < k:     # events inside a deletion are skipped
            e += 1
        nxt = int(evpos[e]) if e < len(evpos) else n
        if nxt > k:                                  # bases up to the next event are kept
            pieces.append(out_base[k:nxt])
            k = nxt
            continue
        if kind[k]:  # insertion before base k
            pieces.append(g.integers(0, alphabet_size, size=int(lens[k]), dtype=np.uint8))
            pieces.append(out_base[k:k + 1])
            k += 1
        else:        # deletion of lens[k] bases starting at k
            k += int(lens[k])
    return np.concatenate(pieces) if pieces else np.zeros(0, dtype=np.uint8)


# ---------------------------------------------------------------- workloads

def dna_pair_2k():
    """Two i.i.d. uniform ACGT sequences of 2,000 bases (seeds BASE+0, BASE+1)."""
    return uniform_dna(2000, BASE_SEED + 0), uniform_dna(2000, BASE_SEED + 1)


def dna_long_pair(length: int = 200_000, window: int | None = None,
                  offset: int | None = None, seed_offset: int = 100):
    """Long DNA pair with a planted homologous window.

    A: ``length`` uniform bases.  B: random left flank + mutate(A[offset :
    offset + window]) + random right flank, flanks sized so that |B| is about
    ``length``.  Defaults: window = 3/4 of the length centred (150 kbp at
    offset 25 kbp for 200 kbp; 3.75 Mbp at 625 kbp for 5 Mbp).
    """
    if window is None:
        window = (3 * length) // 4
    if offset is None:
        offset = (length - window) // 2
    A = uniform_dna(length, BASE_SEED + seed_offset)
    core = mutate(A[offset:offset + window], 4, BASE_SEED + seed_offset + 1)
    g = rng(BASE_SEED + seed_offset + 2)
    rest = max(0, length - len(core))
    left = rest // 2
    B = np.concatenate([g.integers(0, 4, size=left, dtype=np.uint8), core,
                        g.integers(0, 4, size=rest - left, dtype=np.uint8)])
    return A, B


PROTEIN_QUERY_LENGTHS = (144, 464, 1000, 2005, 5478)


def protein_queries(lengths=PROTEIN_QUERY_LENGTHS, seed_offset: int = 200):
    return [random_protein(L, BASE_SEED + seed_offset + k) for k, L in enumerate(lengths)]


def lognormal_lengths(nseq: int, seed: int, median: float = 300.0, sigma: float = 0.61,
                      lo: int = 20, hi: int = 35_000) -> np.ndarray:
    """Lognormal lengths (median 300, sigma 0.61 -> mean about 361), rounded and clipped."""
    x = rng(seed).lognormal(mean=math.log(median), sigma=sigma, size=nseq)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


@dataclass
class ProteinDB:
    residues: np.ndarray   # uint8, all subjects back to back
    offsets: np.ndarray    # int64, nseq + 1
    planted: dict          # query index -> list of planted subject indices

    @property
    def nseq(self) -> int:
        return len(self.offsets) - 1

    def subject(self, s: int) -> np.ndarray:
        return self.residues[self.offsets[s]:self.offsets[s + 1]]


def protein_db(nseq: int = 500_000, queries=None, seed_offset: int = 300,
               planted_per_query=(1, 3), identity_sub: float = 0.15) -> ProteinDB:
    """Synthetic protein database with background composition.

    Lengths lognormal (median 300, sigma 0.61, clipped 20..35,000).  For each
    query, 1-3 planted subjects are mutated copies of it (substitutions at
    ``identity_sub``, indels as in ``mutate``) placed at seeded positions, so
    that every query has non-trivial top hits.
    """
    lens = lognormal_lengths(nseq, BASE_SEED + seed_offset)
    g = rng(BASE_SEED + seed_offset + 1)
    res = g.choice(20, size=int(lens.sum()), p=aa_background()).astype(np.uint8)
    offsets = np.zeros(nseq + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    planted = {}
    if queries:
        gp = rng(BASE_SEED + seed_offset + 2)
        taken = set()
        subjects = [res[offsets[s]:offsets[s + 1]] for s in range(nseq)]
        for qi, q in enumerate(queries):
            cnt = int(gp.integers(planted_per_query[0], planted_per_query[1] + 1))
            planted[qi] = []
            for c in range(cnt):
                s = int(gp.integers(0, nseq))
                while s in taken:
                    s = int(gp.integers(0, nseq))
                taken.add(s)
                subjects[s] = mutate(q, 20, BASE_SEED + seed_offset + 1000 + 10 * qi + c,
                                     p_sub=identity_sub)
                planted[qi].append(s)
        lens = np.array([len(x) for x in subjects], dtype=np.int64)
        offsets = np.zeros(nseq + 1, dtype=np.int64)
        np.cumsum(lens, out=offsets[1:])
        res = np.concatenate(subjects)
    return ProteinDB(res, offsets, planted)


def log_uniform_int(g: np.random.Generator, lo: int, hi: int) -> int:
    return int(round(math.exp(g.uniform(math.log(lo), math.log(hi)))))


def batch_pair(k: int):
    """Pair k of the batched workload: lengths log-uniform on [100, 20,000];
    k even -> DNA (+1/-3, 5/2), k odd -> protein (BLOSUM62, 10/1)."""
    g = rng(BASE_SEED + 10_000 + k)
    m = log_uniform_int(g, 100, 20_000)
    n = log_uniform_int(g, 100, 20_000)
    if k % 2 == 0:
        a = g.integers(0, 4, size=m, dtype=np.uint8)
        b = g.integers(0, 4, size=n, dtype=np.uint8)
        return a, b, "dna"
    a = g.choice(20, size=m, p=aa_background()).astype(np.uint8)
    b = g.choice(20, size=n, p=aa_background()).astype(np.uint8)
    return a, b, "protein"


def batch_pairs(npairs: int = 10_000, start: int = 0):
    return [batch_pair(k) for k in range(start, start + npairs)]


def serving_requests(nreq: int, rate: float, seed_offset: int = 500):
    """Poisson arrivals (exponential gaps at ``rate`` per second) of protein
    queries with log-uniform lengths on [50, 5,000].  Returns (arrival_s, query) list."""
    g = rng(BASE_SEED + seed_offset + int(rate))
    t = 0.0
    out = []
    for _ in range(nreq):
        t += g.exponential(1.0 / rate)
        L = log_uniform_int(g, 50, 5000)
        q = g.choice(20, size=L, p=aa_background()).astype(np.uint8)
        out.append((t, q))
    return out
