"""The 5 Mbp x 5 Mbp variant of the long DNA pair (GPU only).

The full oracle cannot hold a 2.5e13-cell matrix, so the alignment is
checked by what fixes it without one:

(i)   rescoring: the reported CIGAR, placed at the reported begin cell and
      scored from the definition, gives the reported score and end cell;
(ii)  an independent launch: sw_score (score mode, no checkpoints, no
      traceback) gives the same score and end cell;
(iii) sampled pieces: a piece of an optimal path that starts and ends
      inside M runs is an optimal global alignment of the sub-block it
      spans, so its score must equal the oracle's global Gotoh score of that
      sub-block.
"""
import re

import numpy as np
import pytest

from paper_2211_10769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _runs(cigar):
    return [(int(n), op) for n, op in re.findall(r"(\d+)([MID])", cigar)]


def _piece_score(A, B, S, go, ge, i, j, runs):
    """Score of consecutive runs placed at (i, j): M columns by the matrix,
    every gap run open + (L - 1) * extend.  Returns (score, i, j) at the end."""
    sc = 0
    for L, op in runs:
        if op == "M":
            sc += int(S[A[i:i + L], B[j:j + L]].astype(np.int64).sum())
            i += L
            j += L
        else:
            sc -= go + (L - 1) * ge
            if op == "D":
                i += L
            else:
                j += L
    return sc, i, j


@pytest.fixture(scope="module")
def long5m():
    """The 5 Mbp pair, its alignment and its score-mode hit with the default
    checkpoint budget (one checkpoint level)."""
    from paper_2211_10769_gb300 import binding, build
    build.build()
    sc = W.dna_scoring()
    A, B = W.dna_long_pair(5_000_000)
    ctx = binding.Context(0)
    try:
        aln = ctx.align(A, B, sc.matrix, sc.gap_open, sc.gap_extend)
        hit = ctx.score(A, B, sc.matrix, sc.gap_open, sc.gap_extend)
    finally:
        ctx.close()
    return A, B, aln, hit


def test_dna_5mbp_pair(oracle_mod, long5m):
    sc = W.dna_scoring()
    S, go, ge = sc.matrix, sc.gap_open, sc.gap_extend
    A, B, aln, hit = long5m
    # the planted window aligns: most of A's 3.75 Mbp core is covered
    assert aln.score > 1_000_000
    assert aln.a_end - aln.a_begin > 3_000_000
    # (ii) the score-mode launch agrees
    assert (hit.score, hit.a_end, hit.b_end) == (aln.score, aln.a_end, aln.b_end)
    # (i) rescoring the whole path
    runs = _runs(aln.cigar)
    assert "".join("%d%s" % r for r in runs) == aln.cigar
    total, ie, je = _piece_score(A, B, S, go, ge, aln.a_begin, aln.b_begin, runs)
    assert (total, ie, je) == (aln.score, aln.a_end, aln.b_end)
    assert runs[0][1] == "M" and runs[-1][1] == "M"
    # (iii) sampled pieces between cuts inside M runs
    starts = []                                   # (run index, i, j) at the start of every run
    i, j = aln.a_begin, aln.b_begin
    for k, (L, op) in enumerate(runs):
        starts.append((i, j))
        if op != "I":
            i += L
        if op != "D":
            j += L
    mruns = [k for k, (L, op) in enumerate(runs) if op == "M" and L >= 2]
    rng = np.random.default_rng(W.BASE_SEED + 9950)
    checked = 0
    for k1 in rng.choice(mruns[: len(mruns) * 9 // 10], size=8, replace=False):
        # end cut: the first long-enough M run at least 1,500 path columns further on
        i1 = starts[k1][0] + runs[k1][0] // 2
        k2 = k1 + 1
        while k2 < len(runs) and not (runs[k2][1] == "M" and runs[k2][0] >= 2 and starts[k2][0] - i1 >= 1500):
            k2 += 1
        if k2 >= len(runs):
            continue
        c1, c2 = runs[k1][0] // 2, runs[k2][0] // 2
        i1, j1 = starts[k1][0] + c1, starts[k1][1] + c1
        piece = [(runs[k1][0] - c1, "M")] + runs[k1 + 1:k2] + [(c2, "M")]
        ps, i2, j2 = _piece_score(A, B, S, go, ge, i1, j1, piece)
        assert (i2, j2) == (starts[k2][0] + c2, starts[k2][1] + c2)
        assert oracle_mod.nw_score(A[i1:i2], B[j1:j2], S, go, ge) == ps, (i1, j1, i2, j2)
        checked += 1
    assert checked >= 6


def test_dna_5mbp_bounded_memory(monkeypatch, long5m):
    """A 1 GB checkpoint budget takes two checkpoint levels at 5 Mbp: the
    alignment (score, coordinates, canonical CIGAR) is the one-level one,
    and the context's device memory after the call stays within the budget
    plus one band of traceback bits (the one-level run keeps checkpoints
    every 4,096 rows and columns, about 100 GB)."""
    import torch
    from paper_2211_10769_gb300 import binding
    A, B, want, _ = long5m
    sc = W.dna_scoring()
    monkeypatch.setenv("SWGB_CKPT_BUDGET_MB", "1024")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ctx = binding.Context(0)
    try:
        got = ctx.align(A, B, sc.matrix, sc.gap_open, sc.gap_extend)
        free1, _ = torch.cuda.mem_get_info()
    finally:
        ctx.close()
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end) == \
        (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end)
    assert got.cigar == want.cigar
    used = free0 - free1
    assert used < (1 << 30) + (4 << 30), used
