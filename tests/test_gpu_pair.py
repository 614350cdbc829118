"""GPU parity of the pairwise path (sw_score, sw_align) against the CPU oracle.

Every case compares score, end cell, begin cell and CIGAR exactly (integer
work: bit-exact).  Inputs come from the seeded generators shared with the
oracle tests.
"""
import json
import os

import numpy as np
import pytest

from bruteforce import rescore
from paper_2211_10769_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", params=["packed16", "int32", "one_round"])
def ctx(request):
    """A context on the packed 16-bit pair fill (forced at 8 rows a lane
    wherever it is exact), one restricted to the int32 fill, and one that
    reconstructs small pairs in one round (whole-matrix traceback bits)
    instead of through checkpoints and bands of traceback tiles: every test
    runs on all three."""
    from paper_2211_10769_gb300 import binding, build
    build.build()
    # packed16: the packed fill forced at 8 rows a lane (by default pairs up to 152 x 512 rows take
    # the int32 fill, which has more SMs to use there)
    env = {"SWGB_P16": "0" if request.param == "int32" else "1",
           "SWGB_ONE_ROUND": "1" if request.param == "one_round" else "0"}
    if request.param == "packed16":
        env["SWGB_FWD"] = "8,4,0,2,1"
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        c = binding.Context(0)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v
    yield c
    c.close()


_ORACLE_SCORES = {}


def _oracle_score(oracle_mod, a, b, S, o, e):
    """The oracle's score and end cell, computed once per input (both fills reuse it)."""
    import hashlib
    key = (hashlib.sha1(np.ascontiguousarray(a).tobytes()).hexdigest(),
           hashlib.sha1(np.ascontiguousarray(b).tobytes()).hexdigest(),
           np.asarray(S, np.int8).tobytes(), o, e)
    if key not in _ORACLE_SCORES:
        _ORACLE_SCORES[key] = oracle_mod.sw_score(a, b, S, o, e)
    return _ORACLE_SCORES[key]


def _score_case(ctx, oracle_mod, a, b, S, o, e):
    want = _oracle_score(oracle_mod, a, b, S, o, e)
    got = ctx.score(a, b, S, o, e)
    assert (got.score, got.a_end, got.b_end) == want, (len(a), len(b), o, e)


def _align_case(ctx, oracle_mod, a, b, S, o, e):
    want = oracle_mod.sw_align(a, b, S, o, e)
    got = ctx.align(a, b, S, o, e)
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end, got.cigar) == \
        (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end, want.cigar), (len(a), len(b))


EDGE_LENGTHS = [0, 1, 2, 31, 32, 33, 63, 64, 65, 255, 256, 257, 1023, 1024, 1025, 2049]


@pytest.mark.parametrize("m", [1, 33, 1024, 1025, 3000])
def test_score_edge_lengths_dna(ctx, oracle_mod, m):
    sc = W.dna_scoring()
    for n in EDGE_LENGTHS:
        a = W.uniform_dna(m, W.BASE_SEED + 5000 + m)
        b = W.mutate(a, 4, W.BASE_SEED + 6000 + n)[:n] if n else np.zeros(0, np.uint8)
        if len(b) < n:
            b = np.concatenate([b, W.uniform_dna(n - len(b), W.BASE_SEED + 7000 + n)])
        _score_case(ctx, oracle_mod, a, b, sc.matrix, sc.gap_open, sc.gap_extend)


def test_score_random_scorings(ctx, oracle_mod):
    g = np.random.default_rng(W.BASE_SEED + 8000)
    for t in range(60):
        K = int(g.integers(1, 25))
        m, n = int(g.integers(0, 1500)), int(g.integers(0, 1500))
        a = g.integers(0, K, size=m).astype(np.uint8)
        b = g.integers(0, K, size=n).astype(np.uint8)
        S = g.integers(-6, 8, size=(K, K)).astype(np.int8)
        o = int(g.integers(0, 12))
        e = int(g.integers(0, o + 1))
        _score_case(ctx, oracle_mod, a, b, S, o, e)


def test_score_protein_homologs(ctx, oracle_mod):
    sc = W.protein_scoring()
    for t in range(8):
        a = W.random_protein(300 + 211 * t, W.BASE_SEED + 8100 + t)
        b = W.mutate(a, 20, W.BASE_SEED + 8200 + t, p_sub=0.3)
        _score_case(ctx, oracle_mod, a, b, sc.matrix, sc.gap_open, sc.gap_extend)
        _score_case(ctx, oracle_mod, b, a, sc.matrix, sc.gap_open, sc.gap_extend)


def test_score_ties_and_degenerate(ctx, oracle_mod):
    sc = W.dna_scoring()
    runs = np.zeros(700, np.uint8)                      # one long run of one base
    _score_case(ctx, oracle_mod, runs, runs, sc.matrix, sc.gap_open, sc.gap_extend)
    alt = (np.arange(900) % 2).astype(np.uint8)         # many equal maxima
    _score_case(ctx, oracle_mod, alt, alt[::-1].copy(), sc.matrix, sc.gap_open, sc.gap_extend)
    mism = np.zeros(500, np.uint8)
    _score_case(ctx, oracle_mod, mism, mism + 1, sc.matrix, sc.gap_open, sc.gap_extend)   # score 0
    zero_gap = np.ones((4, 4), np.int8)
    _score_case(ctx, oracle_mod, runs[:300], alt[:400], zero_gap, 0, 0)


def test_score_row_ties_inside_lane_halves(ctx, oracle_mod):
    """Equal maxima in several rows of one column, in several columns of one
    row, and periodic repeats that put equal maxima two or three rows apart:
    the end cell is the first in row-major order."""
    sc = W.dna_scoring()
    A = np.zeros(100, np.uint8)
    _score_case(ctx, oracle_mod, A, A[:4], sc.matrix, sc.gap_open, sc.gap_extend)   # one column, rows 4..100
    _score_case(ctx, oracle_mod, A[:4], A, sc.matrix, sc.gap_open, sc.gap_extend)   # one row, columns 4..100
    g = np.random.default_rng(W.BASE_SEED + 8300)
    for period in (2, 3, 5):
        for t in range(6):
            unit = g.integers(0, 4, size=period).astype(np.uint8)
            rep = np.tile(unit, 12 + t)
            a = np.concatenate([W.uniform_dna(int(g.integers(0, 900)), W.BASE_SEED + 8310 + t), rep,
                                W.uniform_dna(int(g.integers(0, 900)), W.BASE_SEED + 8320 + t)])
            b = np.concatenate([W.uniform_dna(int(g.integers(0, 300)), W.BASE_SEED + 8330 + t),
                                rep[: len(rep) - period * (t % 3)],
                                W.uniform_dna(int(g.integers(0, 300)), W.BASE_SEED + 8340 + t)])
            _score_case(ctx, oracle_mod, a, b, sc.matrix, sc.gap_open, sc.gap_extend)
            _score_case(ctx, oracle_mod, b, a, sc.matrix, sc.gap_open, sc.gap_extend)


def test_score_above_16_bits(ctx, oracle_mod):
    """Scores far above 32,767: the packed fill keeps its values relative to a
    moving base and must still give exact scores and end cells."""
    sc = W.dna_scoring()
    a = W.uniform_dna(45_000, W.BASE_SEED + 8400)
    b = W.mutate(a, 4, W.BASE_SEED + 8401, p_sub=0.01, p_indel=0.001)
    _score_case(ctx, oracle_mod, a, a, sc.matrix, sc.gap_open, sc.gap_extend)
    _score_case(ctx, oracle_mod, a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    p = W.protein_scoring()
    q = W.random_protein(8_000, W.BASE_SEED + 8402)
    r = W.mutate(q, 20, W.BASE_SEED + 8403, p_sub=0.05, p_indel=0.005)
    _score_case(ctx, oracle_mod, q, r, p.matrix, p.gap_open, p.gap_extend)
    # a high-scoring region that ends, then a long low stretch, then a second one
    c = np.concatenate([a[:36_000], W.uniform_dna(20_000, W.BASE_SEED + 8404), a[36_000:40_000]])
    _score_case(ctx, oracle_mod, c, a[:40_000], sc.matrix, sc.gap_open, sc.gap_extend)


@pytest.mark.parametrize("seed", range(6))
def test_align_random(ctx, oracle_mod, seed):
    g = np.random.default_rng(W.BASE_SEED + 9000 + seed)
    dna, prot = W.dna_scoring(), W.protein_scoring()
    for t in range(6):
        if t % 2 == 0:
            A = W.uniform_dna(int(g.integers(1, 3000)), W.BASE_SEED + 9100 + 10 * seed + t)
            B = W.mutate(A, 4, W.BASE_SEED + 9200 + 10 * seed + t, p_sub=0.1, p_indel=0.02)
            sc = dna
        else:
            A = W.random_protein(int(g.integers(1, 2000)), W.BASE_SEED + 9100 + 10 * seed + t)
            B = W.mutate(A, 20, W.BASE_SEED + 9200 + 10 * seed + t, p_sub=0.3, p_indel=0.03)
            sc = prot
        _align_case(ctx, oracle_mod, A, B, sc.matrix, sc.gap_open, sc.gap_extend)


def test_align_gappy_small(ctx, oracle_mod):
    g = np.random.default_rng(W.BASE_SEED + 9300)
    S = np.full((4, 4), -3, np.int8)
    np.fill_diagonal(S, 6)
    for t in range(40):
        m, n = int(g.integers(0, 200)), int(g.integers(0, 200))
        a = g.integers(0, 4, size=m).astype(np.uint8)
        b = g.integers(0, 4, size=n).astype(np.uint8)
        o = int(g.integers(1, 5))
        e = int(g.integers(0, o + 1))
        _align_case(ctx, oracle_mod, a, b, S, o, e)


def test_dna_2k_golden(ctx):
    rec = json.load(open(os.path.join(GOLDEN, "dna_2k.json")))
    a, b = W.dna_pair_2k()
    sc = W.dna_scoring()
    got = ctx.align(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end) == \
        (rec["score"], rec["a_begin"], rec["a_end"], rec["b_begin"], rec["b_end"])
    import hashlib
    assert hashlib.sha256(got.cigar.encode()).hexdigest() == rec["cigar_sha256"]


def test_long_pair_golden(ctx):
    path = os.path.join(GOLDEN, "dna_200k.json")
    rec = json.load(open(path))
    a, b = W.dna_long_pair(200_000)
    sc = W.dna_scoring()
    hit = ctx.score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    assert (hit.score, hit.a_end, hit.b_end) == (rec["score"], rec["a_end"], rec["b_end"])
    got = ctx.align(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end) == \
        (rec["score"], rec["a_begin"], rec["a_end"], rec["b_begin"], rec["b_end"])
    import hashlib
    assert len(got.cigar) == rec["cigar_len"]
    assert got.cigar[:120] == rec["cigar_head"] and got.cigar[-120:] == rec["cigar_tail"]
    assert hashlib.sha256(got.cigar.encode()).hexdigest() == rec["cigar_sha256"]
    assert rescore(a, b, sc.matrix, sc.gap_open, sc.gap_extend, got.a_begin, got.b_begin,
                   got.cigar) == (got.score, got.a_end, got.b_end)


def test_device_pointers_and_encode(ctx, oracle_mod):
    import torch
    sc = W.dna_scoring()
    a, b = W.dna_pair_2k()
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    assert ctx.score(ta, tb, sc.matrix, sc.gap_open, sc.gap_extend) == ctx.score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    txt = "".join("ACGT"[x] for x in a[:500])
    assert (ctx.encode("ACGT", txt) == a[:500]).all()
    assert (ctx.encode("ACGT", txt.lower()) == oracle_mod.encode("ACGT", txt)).all()


def test_invalid_arguments(ctx):
    from paper_2211_10769_gb300 import binding
    sc = W.dna_scoring()
    a = W.uniform_dna(100, 1)
    bad = a.copy()
    bad[50] = 4
    with pytest.raises(binding.SwError) as ei:
        ctx.score(a, bad, sc.matrix, sc.gap_open, sc.gap_extend)
    assert ei.value.status == binding.SW_EINVAL
    with pytest.raises(binding.SwError):
        ctx.score(a, a, sc.matrix, 1, 2)                    # extend > open
    with pytest.raises(binding.SwError):
        ctx.encode("ACGT", "ACGN")
    # the context stays usable after errors
    assert ctx.score(a, a, sc.matrix, sc.gap_open, sc.gap_extend).score == 100


def _long_gap_pair(seed, length, cut0, cut1, insert):
    """A and B share A's sequence except that B lacks A[cut0:cut1] (a long
    deletion) or, with insert=True, carries extra random bases there."""
    A = W.uniform_dna(length, seed)
    if insert:
        extra = W.uniform_dna(cut1 - cut0, seed + 1)
        B = np.concatenate([A[:cut0], extra, A[cut0:]])
    else:
        B = np.concatenate([A[:cut0], A[cut1:]])
    B = W.mutate(B, 4, seed + 2, p_sub=0.08, p_indel=0.01)
    return A, B


@pytest.mark.parametrize("case", range(6))
def test_align_paths_cross_tiles(ctx, oracle_mod, case):
    """Paths that cross many 1024 x 1024 tiles, including long vertical and
    horizontal gap runs that leave the diagonal band of recomputed tiles."""
    S = np.full((4, 4), -4, np.int8)
    np.fill_diagonal(S, 5)
    seed = W.BASE_SEED + 9400 + 10 * case
    if case == 0:
        A = W.uniform_dna(5000, seed)
        B = W.mutate(A, 4, seed + 1, p_sub=0.1, p_indel=0.02)
        o, e = 5, 2
        S = W.dna_matrix()
    elif case in (1, 2):
        A, B = _long_gap_pair(seed, 6000, 2100, 3700, insert=(case == 2))
        o, e = 20, 1
    elif case == 3:
        A, B = _long_gap_pair(seed, 4500, 1000, 3300, insert=False)
        o, e = 10, 0
    elif case == 4:
        A = W.random_protein(3500, seed)
        B = W.mutate(A, 20, seed + 1, p_sub=0.25, p_indel=0.03)
        sc = W.protein_scoring()
        S, o, e = sc.matrix, sc.gap_open, sc.gap_extend
    else:
        A, B = _long_gap_pair(seed, 3000, 600, 2800, insert=True)
        o, e = 12, 1
    want = oracle_mod.sw_align_ptr(A, B, S, o, e)
    got = ctx.align(A, B, S, o, e)
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end) == \
        (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end)
    assert got.cigar == want.cigar


@pytest.mark.parametrize("lookahead", ["0", "1"])
def test_bands_with_and_without_lookahead(oracle_mod, monkeypatch, lookahead):
    """The banded reconstruction with bands of two tile rows (many rounds),
    with and without the look-ahead band recomputed while the walk runs:
    a path along the diagonal (the look-ahead band serves) and paths with
    long gaps that leave it (the look-ahead band is discarded)."""
    from paper_2211_10769_gb300 import binding
    monkeypatch.setenv("SWGB_ONE_ROUND", "0")
    monkeypatch.setenv("SWGB_LOOKAHEAD", lookahead)
    monkeypatch.setenv("SWGB_TB_BAND", "2")
    c = binding.Context(0)
    try:
        seed = W.BASE_SEED + 9950
        S2 = np.full((4, 4), -4, np.int8)
        np.fill_diagonal(S2, 5)
        A = W.uniform_dna(9000, seed)
        cases = [(A, W.mutate(A, 4, seed + 1, p_sub=0.08, p_indel=0.01), W.dna_matrix(), 5, 2),
                 (*_long_gap_pair(seed + 10, 8000, 2500, 4200, insert=False), S2, 20, 1),
                 (*_long_gap_pair(seed + 20, 8000, 3000, 4400, insert=True), S2, 20, 1)]
        for a, b, S, o, e in cases:
            want = oracle_mod.sw_align_ptr(a, b, S, o, e)
            got = c.align(a, b, S, o, e)
            assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end, got.cigar) == \
                (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end, want.cigar)
    finally:
        c.close()


@pytest.mark.parametrize("fwd", ["8,8,5", "8,8,6", "8,4,3", "16,4,1", "12,4", "4,4",
                                 "8,4,0,2,1", "12,4,0,2,1", "16,4,0,2,1", "12,4,2,2,1"])
def test_strip_heights(oracle_mod, monkeypatch, fwd):
    """Forward strips of 1280, 1536, 768, 512, 1536 (12 rows a lane) and 512 rows, and the packed
    16-bit fill with 8, 12 and 16 rows a lane (two-positions checkpoint columns entered by the
    int32 traceback tiles), one of them with strips of two warps: strip bottoms, row
    checkpoints and traceback tiles (sides that are multiples of both strip heights) must
    still meet exactly."""
    from paper_2211_10769_gb300 import binding, build
    build.build()
    monkeypatch.setenv("SWGB_FWD", fwd)
    c = binding.Context(0)
    try:
        seed = W.BASE_SEED + 9700
        A, B = _long_gap_pair(seed, 13000, 4100, 6900, insert=False)
        S = np.full((4, 4), -4, np.int8)
        np.fill_diagonal(S, 5)
        for (a, b, o, e) in [(A, B, 20, 1), (A[:7000], W.mutate(A[:7000], 4, seed + 5, p_sub=0.1, p_indel=0.02), 5, 2)]:
            want = oracle_mod.sw_align_ptr(a, b, S, o, e)
            got = c.align(a, b, S, o, e)
            assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end) == \
                (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end), fwd
            assert got.cigar == want.cigar, fwd
            h = c.score(a, b, S, o, e)
            assert (h.score, h.a_end, h.b_end) == (want.score, want.a_end, want.b_end), fwd
    finally:
        c.close()


@pytest.mark.parametrize("side", [8192, 8193])
def test_align_one_round_limit(ctx, oracle_mod, side):
    """The largest pair reconstructed in one round (both sides 8,192, one
    traceback tile of 8,192 x 8,192 cells) and the smallest that is not."""
    seed = W.BASE_SEED + 9900 + side
    A = W.uniform_dna(side, seed)
    B = W.mutate(A, 4, seed + 1, p_sub=0.1, p_indel=0.02)
    B = np.concatenate([B, W.uniform_dna(side, seed + 2)])[:side]
    S = W.dna_matrix()
    want = oracle_mod.sw_align_ptr(A, B, S, 5, 2)
    got = ctx.align(A, B, S, 5, 2)
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end, got.cigar) == \
        (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end, want.cigar)


@pytest.mark.parametrize("sides,env", [("3072,1024", {}), ("3072,1024", {"SWGB_P16": "0"}),
                                       ("3072,1024", {"SWGB_FWD": "8,4,0,2,1"}),
                                       ("4608,1536", {"SWGB_FWD": "12,4,0,2,1"}), ("2048,1024", {})])
def test_two_level_checkpoints(oracle_mod, monkeypatch, sides, env):
    """Two levels of checkpoints (forced small sides): the forward fill keeps
    every BT1-th row and column, each coarse tile the path enters is filled
    again from them with checkpoints every BT2 (by the packed fill entering its
    own checkpoint column, or the int32 fill), and the traceback tiles start
    from either level.  Paths with long gaps cross coarse tiles in both
    directions; DNA (packed and int32 forward fills) and protein."""
    from paper_2211_10769_gb300 import binding
    monkeypatch.setenv("SWGB_TWO_LEVEL", sides)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    c = binding.Context(0)
    try:
        seed = W.BASE_SEED + 9800
        S = np.full((4, 4), -4, np.int8)
        np.fill_diagonal(S, 5)
        cases = [_long_gap_pair(seed, 12000, 3100, 6400, insert=False) + (S, 20, 1),
                 _long_gap_pair(seed + 10, 11000, 2500, 5200, insert=True) + (S, 12, 1)]
        A = W.uniform_dna(9000, seed + 20)
        cases.append((A, W.mutate(A, 4, seed + 21, p_sub=0.1, p_indel=0.02), W.dna_matrix(), 5, 2))
        P = W.random_protein(7000, seed + 30)
        p = W.protein_scoring()
        cases.append((P, W.mutate(P, 20, seed + 31, p_sub=0.25, p_indel=0.03), p.matrix, p.gap_open, p.gap_extend))
        for a, b, M, o, e in cases:
            want = oracle_mod.sw_align_ptr(a, b, M, o, e)
            got = c.align(a, b, M, o, e)
            assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end) == \
                (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end), (sides, env, len(a))
            assert got.cigar == want.cigar, (sides, env, len(a))
    finally:
        c.close()


def test_kernel_timing(ctx):
    """Per-kernel device time: one forward fill per sw_align, walks and
    traceback fills counted, totals cleared when timing is re-enabled."""
    from paper_2211_10769_gb300 import binding
    sc = W.dna_scoring()
    a, b = W.dna_pair_2k()
    ctx.timing(True)
    for _ in range(3):
        ctx.align(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    ms, n = ctx.kernel_time(binding.KT_FILL)
    assert n == 3 and ms > 0
    ms_tb, n_tb = ctx.kernel_time(binding.KT_FILL_TB)
    ms_w, n_w = ctx.kernel_time(binding.KT_WALK)
    assert n_tb >= 3 and n_w == n_tb and ms_tb > 0 and ms_w > 0
    ctx.timing(True)
    assert ctx.kernel_time(binding.KT_FILL) == (0.0, 0)
    ctx.timing(False)
    ctx.score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    assert ctx.kernel_time(binding.KT_FILL) == (0.0, 0)
    with pytest.raises(binding.SwError):
        ctx.kernel_time(7)


def test_bounded_wait_timeout(oracle_mod, monkeypatch):
    """Failure detection without a GPU fault: with a spin limit of one poll
    every cross-warp wait of the fill gives up at once, the kernel records
    the timeout in its error word and returns; the call reports SW_ETIMEOUT
    and the process and device stay usable."""
    from paper_2211_10769_gb300 import binding, build
    build.build()
    sc = W.dna_scoring()
    a = W.uniform_dna(20_000, W.BASE_SEED + 9900)
    b = W.mutate(a, 4, W.BASE_SEED + 9901, p_sub=0.1, p_indel=0.02)
    monkeypatch.setenv("SWGB_SPIN_LIMIT", "1")
    c = binding.Context(0)
    try:
        for call in (c.score, c.align):
            with pytest.raises(binding.SwError) as ei:
                call(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
            assert ei.value.status == binding.SW_ETIMEOUT
    finally:
        c.close()
    monkeypatch.delenv("SWGB_SPIN_LIMIT")
    c2 = binding.Context(0)
    try:
        want = oracle_mod.sw_score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
        got = c2.score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
        assert (got.score, got.a_end, got.b_end) == want
    finally:
        c2.close()
