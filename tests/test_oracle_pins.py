"""Pins for the CPU oracle: checks against things other than the oracle itself.

* brute-force enumeration of every local alignment (|a|, |b| <= 7): score,
  canonical end cell and canonical traceback;
* closed forms: DNA and protein self-alignment;
* score symmetry under swapping the sequences (with the transposed matrix);
* open == extend against an independent linear-gap Smith-Waterman;
* prohibitive gap penalties against Kadane's maximum subarray on diagonals;
* rescoring of every emitted CIGAR by a separate scorer;
* BLOSUM62 table invariants.
"""
import itertools

import numpy as np
import pytest

from bruteforce import brute_force, rescore
from paper_2211_10769_gb300 import workloads as W


def _rand_case(g, K, Lmax, strict_gap=False):
    m = int(g.integers(0, Lmax + 1))
    n = int(g.integers(0, Lmax + 1))
    a = g.integers(0, K, size=m).astype(np.uint8)
    b = g.integers(0, K, size=n).astype(np.uint8)
    S = g.integers(-4, 7, size=(K, K)).astype(np.int8)
    o = int(g.integers(0, 7))
    e = int(g.integers(0, o + 1))
    if strict_gap and e == o:
        o += 1
    return a, b, S, o, e


def _check_against_brute(oracle_mod, a, b, S, o, e, check_path):
    score, i_end, j_end, canon = brute_force(a, b, S, o, e)
    assert oracle_mod.sw_score(a, b, S, o, e) == (score, i_end, j_end)
    for aln in (oracle_mod.sw_align(a, b, S, o, e), oracle_mod.sw_align_ptr(a, b, S, o, e)):
        assert (aln.score, aln.a_end, aln.b_end) == (score, i_end, j_end)
        if score == 0:
            assert aln.cigar == "" and (aln.a_begin, aln.b_begin) == (0, 0)
            continue
        assert rescore(a, b, S, o, e, aln.a_begin, aln.b_begin, aln.cigar) == (score, i_end, j_end)
        if check_path:
            ops = oracle_mod.cigar_from_ops(canon[2])
            assert (aln.a_begin, aln.b_begin, aln.cigar) == (canon[0], canon[1], ops)


@pytest.mark.parametrize("K", [2, 4])
def test_bruteforce_random_small(oracle_mod, K):
    g = np.random.default_rng(W.BASE_SEED + 7 + K)
    for _ in range(150):
        a, b, S, o, e = _rand_case(g, K, 6)
        _check_against_brute(oracle_mod, a, b, S, o, e, check_path=(e < o))


def test_bruteforce_length7(oracle_mod):
    g = np.random.default_rng(W.BASE_SEED + 77)
    for _ in range(12):
        a, b, S, o, e = _rand_case(g, 4, 7, strict_gap=True)
        a = g.integers(0, 4, size=7).astype(np.uint8)
        b = g.integers(0, 4, size=7).astype(np.uint8)
        _check_against_brute(oracle_mod, a, b, S, o, e, check_path=True)


def test_bruteforce_gappy_scoring(oracle_mod):
    """Large match reward and cheap gaps, so that optimal alignments carry gaps."""
    g = np.random.default_rng(W.BASE_SEED + 78)
    S = np.full((4, 4), -3, dtype=np.int8)
    np.fill_diagonal(S, 6)
    seen_gap = False
    for _ in range(60):
        m, n = int(g.integers(3, 7)), int(g.integers(3, 7))
        a = g.integers(0, 4, size=m).astype(np.uint8)
        b = g.integers(0, 4, size=n).astype(np.uint8)
        o = int(g.integers(1, 4))
        e = int(g.integers(0, o))
        _check_against_brute(oracle_mod, a, b, S, o, e, check_path=True)
        aln = oracle_mod.sw_align(a, b, S, o, e)
        seen_gap |= ("I" in aln.cigar) or ("D" in aln.cigar)
    assert seen_gap


def test_bruteforce_exhaustive_binary(oracle_mod):
    """Every pair of binary strings of length <= 4 under two scorings."""
    seqs = [np.array(s, dtype=np.uint8) for L in range(5) for s in itertools.product([0, 1], repeat=L)]
    S1 = np.array([[2, -1], [-1, 3]], dtype=np.int8)
    S2 = np.array([[5, -4], [-2, 4]], dtype=np.int8)     # not symmetric on purpose
    for S, o, e in ((S1, 2, 1), (S2, 3, 0), (S1, 1, 1)):
        for a in seqs:
            for b in seqs:
                _check_against_brute(oracle_mod, a, b, S, o, e, check_path=(e < o))


def test_self_alignment_dna_closed_form(oracle_mod):
    sc = W.dna_scoring()
    for L in (1, 17, 500, 2000):
        a = W.uniform_dna(L, W.BASE_SEED + 900 + L)
        aln = oracle_mod.sw_align(a, a, sc.matrix, sc.gap_open, sc.gap_extend)
        assert aln.score == L
        assert (aln.a_begin, aln.a_end, aln.b_begin, aln.b_end, aln.cigar) == (0, L, 0, L, "%dM" % L)


def test_blosum62_invariants():
    B = W.blosum62()
    assert B.shape == (24, 24)
    assert (B == B.T).all()
    assert B.min() == -4 and B.max() == 11
    assert B[W.PROTEIN_ALPHABET.index("W"), W.PROTEIN_ALPHABET.index("W")] == 11
    d = np.diag(B)[:20]
    assert (d > 0).all()
    # S(x,y) <= (S(x,x) + S(y,y)) / 2 for the 20 standard letters, which is
    # what makes self-alignment the sum of the diagonal.
    for x in range(20):
        for y in range(20):
            if x != y:
                assert 2 * int(B[x, y]) <= int(B[x, x]) + int(B[y, y])
    # a few entries that are easy to misplace
    P = W.PROTEIN_ALPHABET.index
    assert B[P("C"), P("C")] == 9 and B[P("H"), P("H")] == 8 and B[P("P"), P("P")] == 7
    assert B[P("I"), P("V")] == 3 and B[P("D"), P("E")] == 2 and B[P("*"), P("*")] == 1
    assert B[P("B"), P("D")] == 4 and B[P("Z"), P("E")] == 4 and B[P("X"), P("X")] == -1


def test_self_alignment_protein_closed_form(oracle_mod):
    sc = W.protein_scoring()
    B = sc.matrix
    for L in (1, 50, 700):
        a = W.random_protein(L, W.BASE_SEED + 950 + L)
        aln = oracle_mod.sw_align(a, a, B, sc.gap_open, sc.gap_extend)
        assert aln.score == int(sum(int(B[x, x]) for x in a))
        assert aln.cigar == "%dM" % L


def test_symmetry(oracle_mod):
    g = np.random.default_rng(W.BASE_SEED + 31)
    for _ in range(40):
        K = int(g.integers(2, 8))
        m, n = int(g.integers(0, 60)), int(g.integers(0, 60))
        a = g.integers(0, K, size=m).astype(np.uint8)
        b = g.integers(0, K, size=n).astype(np.uint8)
        S = g.integers(-5, 6, size=(K, K)).astype(np.int8)
        o = int(g.integers(0, 8))
        e = int(g.integers(0, o + 1))
        s1 = oracle_mod.sw_score(a, b, S, o, e)[0]
        s2 = oracle_mod.sw_score(b, a, np.ascontiguousarray(S.T), o, e)[0]
        assert s1 == s2


def _linear_gap_sw(a, b, S, g):
    """Textbook one-matrix Smith-Waterman with linear gap cost g per gap letter."""
    m, n = len(a), len(b)
    prev = [0] * (n + 1)
    best = 0
    for i in range(1, m + 1):
        cur = [0] * (n + 1)
        for j in range(1, n + 1):
            cur[j] = max(0, prev[j - 1] + int(S[a[i - 1]][b[j - 1]]), prev[j] - g, cur[j - 1] - g)
            best = max(best, cur[j])
        prev = cur
    return best


def test_open_equals_extend_is_linear_gap(oracle_mod):
    g = np.random.default_rng(W.BASE_SEED + 41)
    for _ in range(30):
        K = int(g.integers(2, 6))
        m, n = int(g.integers(0, 80)), int(g.integers(0, 80))
        a = g.integers(0, K, size=m).astype(np.uint8)
        b = g.integers(0, K, size=n).astype(np.uint8)
        S = g.integers(-3, 6, size=(K, K)).astype(np.int8)
        gap = int(g.integers(0, 5))
        assert oracle_mod.sw_score(a, b, S, gap, gap)[0] == _linear_gap_sw(a, b, S, gap)


def _kadane_diagonals(a, b, S):
    best = 0
    m, n = len(a), len(b)
    for d in range(-m + 1, n):
        run = 0
        for i in range(m):
            j = i + d
            if 0 <= j < n:
                run = max(0, run + int(S[a[i]][b[j]]))
                best = max(best, run)
    return best


def test_huge_gaps_is_kadane(oracle_mod):
    g = np.random.default_rng(W.BASE_SEED + 51)
    for _ in range(30):
        K = int(g.integers(2, 6))
        m, n = int(g.integers(0, 70)), int(g.integers(0, 70))
        a = g.integers(0, K, size=m).astype(np.uint8)
        b = g.integers(0, K, size=n).astype(np.uint8)
        S = g.integers(-4, 5, size=(K, K)).astype(np.int8)
        assert oracle_mod.sw_score(a, b, S, 10_000, 10_000)[0] == _kadane_diagonals(a, b, S)


def test_rescoring_medium_cases(oracle_mod):
    """Larger random cases: both traceback forms agree and every CIGAR rescores."""
    g = np.random.default_rng(W.BASE_SEED + 61)
    dna, prot = W.dna_scoring(), W.protein_scoring()
    for t in range(16):
        if t % 2 == 0:
            A = W.uniform_dna(int(g.integers(50, 400)), W.BASE_SEED + 2000 + t)
            B = W.mutate(A, 4, W.BASE_SEED + 3000 + t, p_sub=0.1, p_indel=0.03)
            sc = dna
        else:
            A = W.random_protein(int(g.integers(50, 300)), W.BASE_SEED + 2000 + t)
            B = W.mutate(A, 20, W.BASE_SEED + 3000 + t, p_sub=0.3, p_indel=0.03)
            sc = prot
        full = oracle_mod.sw_align(A, B, sc.matrix, sc.gap_open, sc.gap_extend)
        ptr = oracle_mod.sw_align_ptr(A, B, sc.matrix, sc.gap_open, sc.gap_extend)
        assert full == ptr
        assert full.score == oracle_mod.sw_score(A, B, sc.matrix, sc.gap_open, sc.gap_extend)[0]
        assert rescore(A, B, sc.matrix, sc.gap_open, sc.gap_extend, full.a_begin, full.b_begin,
                       full.cigar) == (full.score, full.a_end, full.b_end)


def test_encode(oracle_mod):
    assert list(oracle_mod.encode("ACGT", "ACGTacgt")) == [0, 1, 2, 3, 0, 1, 2, 3]
    codes = oracle_mod.encode(W.PROTEIN_ALPHABET, "ARNDCQEGHILKMFPSTWYVBZX*")
    assert list(codes) == list(range(24))
    with pytest.raises(ValueError):
        oracle_mod.encode("ACGT", "ACGN")


def test_global_score_bruteforce(oracle_mod):
    """The global Gotoh score equals the best of all enumerated global
    alignments (leading and trailing gaps included), for random tiny pairs,
    2- and 4-letter alphabets and several gap costs, empty sides included."""
    from bruteforce import brute_force_global
    rng = np.random.default_rng(W.BASE_SEED + 7100)
    for _ in range(120):
        K = int(rng.choice([2, 4]))
        S = rng.integers(-4, 5, size=(K, K)).astype(np.int8)
        S = np.triu(S) + np.triu(S, 1).T
        go = int(rng.integers(0, 7))
        ge = int(rng.integers(0, go + 1))
        a = rng.integers(0, K, size=int(rng.integers(0, 6))).astype(np.uint8)
        b = rng.integers(0, K, size=int(rng.integers(0, 6))).astype(np.uint8)
        assert oracle_mod.nw_score(a, b, S, go, ge) == brute_force_global(list(a), list(b), S, go, ge), \
            (list(a), list(b), S.tolist(), go, ge)


def test_global_score_closed_forms(oracle_mod):
    """Identical DNA aligns end to end with no gap; one side empty costs one gap."""
    S = W.dna_matrix()
    a = W.uniform_dna(300, W.BASE_SEED + 7200)
    assert oracle_mod.nw_score(a, a, S, 5, 2) == 300
    assert oracle_mod.nw_score(a[:7], a[:0], S, 5, 2) == -(5 + 6 * 2)
    assert oracle_mod.nw_score(a[:0], a[:0], S, 5, 2) == 0
    # a local alignment that spans both sequences end to end scores the global optimum
    b = W.mutate(a, 4, W.BASE_SEED + 7201, p_sub=0.02, p_indel=0.0)
    loc = oracle_mod.sw_align(a, b, S, 5, 2)
    if (loc.a_begin, loc.b_begin, loc.a_end, loc.b_end) == (0, 0, len(a), len(b)):
        assert oracle_mod.nw_score(a, b, S, 5, 2) == loc.score


# Hand-written expected rankings for the database top-k (score descending,
# then subject index ascending; subjects scoring 0 are still ranked).  Each
# case: (scores, k, expected [(subject, score), ...]).
TOP_K_CASES = [
    ([5, 9, 1, 9, 7], 3, [(1, 9), (3, 9), (4, 7)]),              # tie on score: lower subject first
    ([3, 3, 3, 3], 4, [(0, 3), (1, 3), (2, 3), (3, 3)]),          # all tied
    ([0, 0, 0], 2, [(0, 0), (1, 0)]),                             # all-zero scores are still ranked
    ([4, 0, 2], 10, [(0, 4), (2, 2), (1, 0)]),                    # k > n: every subject, in order
    ([8, 1], 0, []),                                              # k = 0
    ([], 5, []),                                                  # empty database
    ([1, 2, 3, 4, 5, 6], 6, [(5, 6), (4, 5), (3, 4), (2, 3), (1, 2), (0, 1)]),   # strictly ascending input
    ([2, 10, 0, 10, 2, 7], 5, [(1, 10), (3, 10), (5, 7), (0, 2), (4, 2)]),        # two tie groups
]


def check_top_k(top_k):
    """Pins a top-k function against the hand-written rankings above."""
    for scores, k, want in TOP_K_CASES:
        got = [(int(s), int(v)) for s, v in top_k(np.asarray(scores, dtype=np.int64), k)]
        assert got == want, (scores, k, got, want)


def test_top_k_hand_written_rankings(oracle_mod):
    check_top_k(oracle_mod.top_k)


# ---- the global (NW), semi-global (HW) and overlap (OV) algorithms of Section 2.1

ALGS = (1, 2, 3)


def check_variants_bruteforce(oracle_mod, cases=120, seed=W.BASE_SEED + 7300):
    """Every NW / HW / OV alignment of tiny pairs, listed and scored from the
    definition: best score, canonical end cell and canonical path."""
    from bruteforce import brute_force_alg
    g = np.random.default_rng(seed)
    for _ in range(cases):
        K = int(g.choice([2, 4]))
        m, n = int(g.integers(0, 5)), int(g.integers(0, 5))
        a = g.integers(0, K, size=m).astype(np.uint8)
        b = g.integers(0, K, size=n).astype(np.uint8)
        S = g.integers(-4, 6, size=(K, K)).astype(np.int8)
        o = int(g.integers(0, 7))
        e = int(g.integers(0, o + 1))
        for alg in ALGS:
            sc, ie, je, canon = brute_force_alg(list(a), list(b), S, o, e, alg)
            aln = oracle_mod.align_alg(a, b, S, o, e, alg)
            assert (aln.score, aln.a_end, aln.b_end) == (sc, ie, je), (alg, list(a), list(b), S.tolist(), o, e)
            assert oracle_mod.score_alg(a, b, S, o, e, alg) == (sc, ie, je)
            if e < o:
                ops = oracle_mod.cigar_from_ops(canon[2])
                assert (aln.a_begin, aln.b_begin, aln.cigar) == (canon[0], canon[1], ops), (alg, list(a), list(b))


def test_variants_bruteforce(oracle_mod):
    check_variants_bruteforce(oracle_mod)


def test_variants_local_equals_sw(oracle_mod):
    """Algorithm 0 through the variant entry points is the Smith-Waterman oracle."""
    g = np.random.default_rng(W.BASE_SEED + 7310)
    for _ in range(40):
        a, b, S, o, e = _rand_case(g, 4, 60)
        assert oracle_mod.score_alg(a, b, S, o, e, 0) == oracle_mod.sw_score(a, b, S, o, e)
        assert oracle_mod.align_alg(a, b, S, o, e, 0) == oracle_mod.sw_align(a, b, S, o, e)


def check_variants_closed_forms(oracle_mod):
    S = W.dna_matrix()
    a = W.uniform_dna(200, W.BASE_SEED + 7320)
    # global: identity end to end; one side empty costs one gap; equals the global score function
    def tup(x):
        return (x.score, x.a_begin, x.a_end, x.b_begin, x.b_end, x.cigar)
    assert tup(oracle_mod.align_alg(a, a, S, 5, 2, 1)) == (200, 0, 200, 0, 200, "200M")
    assert tup(oracle_mod.align_alg(a[:7], a[:0], S, 5, 2, 1)) == (-(5 + 6 * 2), 0, 7, 0, 0, "7D")
    assert tup(oracle_mod.align_alg(a[:0], a[:9], S, 5, 2, 1)) == (-(5 + 8 * 2), 0, 0, 0, 9, "9I")
    b = W.mutate(a, 4, W.BASE_SEED + 7321, p_sub=0.1, p_indel=0.02)
    assert oracle_mod.score_alg(a, b, S, 5, 2, 1)[0] == oracle_mod.nw_score(a, b, S, 5, 2)
    # semi-global: a copy of a inside b aligns end to end at no gap cost
    left, right = W.uniform_dna(37, W.BASE_SEED + 7322), W.uniform_dna(50, W.BASE_SEED + 7323)
    host = np.concatenate([left, a, right])
    aln = oracle_mod.align_alg(a, host, S, 5, 2, 2)
    assert (aln.score, aln.a_begin, aln.a_end, aln.b_begin, aln.b_end, aln.cigar) == (200, 0, 200, 37, 237, "200M")
    # semi-global with b empty: all of a deleted
    assert tup(oracle_mod.align_alg(a[:4], a[:0], S, 5, 2, 2)) == (-(5 + 3 * 2), 0, 4, 0, 0, "4D")
    # overlap: a suffix of a equal to a prefix of b, the rest random: free end gaps on both
    x = np.concatenate([W.uniform_dna(80, W.BASE_SEED + 7324), a[:120]])
    y = np.concatenate([a[:120], W.uniform_dna(90, W.BASE_SEED + 7325)])
    aln = oracle_mod.align_alg(x, y, S, 5, 2, 3)
    assert aln.score >= 120 and aln.a_end == len(x) and aln.b_begin == 0
    # overlap of two empty-ish sequences is the empty alignment at (0, n)
    assert oracle_mod.score_alg(a[:0], a[:5], S, 5, 2, 3) == (0, 0, 0)
    assert oracle_mod.score_alg(a[:3], a[:0], S, 5, 2, 3) == (0, 0, 0)


def test_variants_closed_forms(oracle_mod):
    check_variants_closed_forms(oracle_mod)


def check_variants_symmetry_and_rescoring(oracle_mod):
    """NW and OV scores are symmetric under swapping the sequences (with the
    transposed matrix); every variant CIGAR rescores to its score and spans
    the cells its algorithm requires."""
    g = np.random.default_rng(W.BASE_SEED + 7330)
    for t in range(30):
        K = 4
        A = g.integers(0, K, size=int(g.integers(1, 90))).astype(np.uint8)
        B = W.mutate(A, K, W.BASE_SEED + 7340 + t, p_sub=0.2, p_indel=0.05)[: int(g.integers(1, 120))]
        S = g.integers(-4, 6, size=(K, K)).astype(np.int8)
        o = int(g.integers(1, 8))
        e = int(g.integers(0, o + 1))
        for alg in (1, 3):
            assert oracle_mod.score_alg(A, B, S, o, e, alg)[0] == oracle_mod.score_alg(B, A, S.T.copy(), o, e, alg)[0]
        for alg in ALGS:
            aln = oracle_mod.align_alg(A, B, S, o, e, alg)
            assert rescore(A, B, S, o, e, aln.a_begin, aln.b_begin, aln.cigar) == (aln.score, aln.a_end, aln.b_end)
            if alg == 1:
                assert (aln.a_begin, aln.b_begin, aln.a_end, aln.b_end) == (0, 0, len(A), len(B))
            elif alg == 2:
                assert aln.a_begin == 0 and aln.a_end == len(A)
            else:
                assert (aln.a_begin == 0 or aln.b_begin == 0) and (aln.a_end == len(A) or aln.b_end == len(B))


def test_variants_symmetry_and_rescoring(oracle_mod):
    check_variants_symmetry_and_rescoring(oracle_mod)
