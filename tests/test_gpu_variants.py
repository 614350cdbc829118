"""GPU parity of the global (NW), semi-global (HW) and overlap (OV)
algorithms of paper Section 2.1 against the CPU oracle: score, canonical end
cell, begin cell and CIGAR, exactly, through sw_score, sw_align and the
batch; calls that take the local algorithm only reject the others."""
import os

import numpy as np
import pytest

from bruteforce import rescore
from paper_2211_10769_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ALGS = (1, 2, 3)


@pytest.fixture(scope="module", params=["banded", "one_round"])
def ctx(request):
    """Small pairs reconstructed through checkpoints and bands of traceback
    tiles (the default) and in one round."""
    from paper_2211_10769_gb300 import binding, build
    build.build()
    old = os.environ.get("SWGB_ONE_ROUND")
    os.environ["SWGB_ONE_ROUND"] = "1" if request.param == "one_round" else "0"
    try:
        c = binding.Context(0)
    finally:
        if old is None:
            del os.environ["SWGB_ONE_ROUND"]
        else:
            os.environ["SWGB_ONE_ROUND"] = old
    yield c
    c.close()


def _score_case(ctx, oracle_mod, a, b, S, o, e, alg):
    want = oracle_mod.score_alg(a, b, S, o, e, alg)
    got = ctx.score(a, b, S, o, e, algorithm=alg)
    assert (got.score, got.a_end, got.b_end) == want, (alg, len(a), len(b), o, e)


def _align_case(ctx, oracle_mod, a, b, S, o, e, alg):
    want = oracle_mod.align_alg(a, b, S, o, e, alg)
    got = ctx.align(a, b, S, o, e, algorithm=alg)
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end, got.cigar) == \
        (want.score, want.a_begin, want.a_end, want.b_begin, want.b_end, want.cigar), (alg, len(a), len(b), o, e)
    if got.cigar:
        assert rescore(a, b, S, o, e, got.a_begin, got.b_begin, got.cigar) == (got.score, got.a_end, got.b_end)


EDGE = [0, 1, 2, 31, 33, 64, 65, 255, 1023, 1025, 2049]


@pytest.mark.parametrize("alg", ALGS)
def test_score_edge_lengths(ctx, oracle_mod, alg):
    sc = W.dna_scoring()
    for m in (0, 1, 33, 1025, 3000):
        a = W.uniform_dna(m, W.BASE_SEED + 15000 + m)
        for n in EDGE:
            b = W.mutate(a, 4, W.BASE_SEED + 15100 + n)[:n]
            if len(b) < n:
                b = np.concatenate([b, W.uniform_dna(n - len(b), W.BASE_SEED + 15200 + n)])
            _score_case(ctx, oracle_mod, a, b, sc.matrix, sc.gap_open, sc.gap_extend, alg)


@pytest.mark.parametrize("alg", ALGS)
def test_score_random_scorings(ctx, oracle_mod, alg):
    g = np.random.default_rng(W.BASE_SEED + 15300 + alg)
    for t in range(30):
        K = int(g.integers(1, 25))
        m, n = int(g.integers(0, 1400)), int(g.integers(0, 1400))
        a = g.integers(0, K, size=m).astype(np.uint8)
        b = g.integers(0, K, size=n).astype(np.uint8)
        S = g.integers(-6, 8, size=(K, K)).astype(np.int8)
        o = int(g.integers(0, 12))
        e = int(g.integers(0, o + 1))
        _score_case(ctx, oracle_mod, a, b, S, o, e, alg)


@pytest.mark.parametrize("alg", ALGS)
def test_align_random(ctx, oracle_mod, alg):
    g = np.random.default_rng(W.BASE_SEED + 15400 + alg)
    dna, prot = W.dna_scoring(), W.protein_scoring()
    for t in range(8):
        if t % 2 == 0:
            A = W.uniform_dna(int(g.integers(1, 2500)), W.BASE_SEED + 15410 + t)
            B = W.mutate(A, 4, W.BASE_SEED + 15420 + t, p_sub=0.1, p_indel=0.02)[: int(g.integers(1, 2500))]
            sc = dna
        else:
            A = W.random_protein(int(g.integers(1, 1800)), W.BASE_SEED + 15410 + t)
            B = W.mutate(A, 20, W.BASE_SEED + 15420 + t, p_sub=0.3, p_indel=0.03)
            sc = prot
        _align_case(ctx, oracle_mod, A, B, sc.matrix, sc.gap_open, sc.gap_extend, alg)


@pytest.mark.parametrize("alg", ALGS)
def test_align_small_and_empty(ctx, oracle_mod, alg):
    g = np.random.default_rng(W.BASE_SEED + 15500 + alg)
    S = np.full((4, 4), -3, np.int8)
    np.fill_diagonal(S, 6)
    for t in range(40):
        m, n = int(g.integers(0, 150)), int(g.integers(0, 150))
        a = g.integers(0, 4, size=m).astype(np.uint8)
        b = g.integers(0, 4, size=n).astype(np.uint8)
        o = int(g.integers(1, 6))
        e = int(g.integers(0, o + 1))
        _align_case(ctx, oracle_mod, a, b, S, o, e, alg)


@pytest.mark.parametrize("alg", ALGS)
def test_align_paths_cross_tiles(ctx, oracle_mod, alg):
    """Paths over many 1024 x 1024 traceback tiles with long gap runs, and
    paths that end on the border (overlap, semi-global)."""
    S = np.full((4, 4), -4, np.int8)
    np.fill_diagonal(S, 5)
    seed = W.BASE_SEED + 15600 + alg
    A = W.uniform_dna(2900, seed)
    B = np.concatenate([A[:900], W.uniform_dna(700, seed + 1), A[1500:]])
    B = W.mutate(B, 4, seed + 2, p_sub=0.08, p_indel=0.01)
    _align_case(ctx, oracle_mod, A, B, S, 20, 1, alg)
    # overlap / semi-global shapes: a suffix of A against a prefix of B, A inside B
    C = np.concatenate([W.uniform_dna(1200, seed + 3), A[:1600]])
    D = np.concatenate([A[:1600], W.uniform_dna(1300, seed + 4)])
    _align_case(ctx, oracle_mod, C, D, W.dna_matrix(), 5, 2, alg)
    H = np.concatenate([W.uniform_dna(1100, seed + 5), W.mutate(A[:2000], 4, seed + 6, p_sub=0.05), W.uniform_dna(900, seed + 7)])
    _align_case(ctx, oracle_mod, A[:2000], H, W.dna_matrix(), 5, 2, alg)


@pytest.mark.parametrize("alg", ALGS)
def test_score_long_pair(ctx, oracle_mod, alg):
    """20,000 x 20,000 (many strips, the strip chain and its borders)."""
    sc = W.dna_scoring()
    A, B = W.dna_long_pair(20_000)
    _score_case(ctx, oracle_mod, A, B, sc.matrix, sc.gap_open, sc.gap_extend, alg)


@pytest.mark.parametrize("R", [12, 16])
@pytest.mark.parametrize("alg", ALGS)
def test_strip_heights(oracle_mod, monkeypatch, alg, R):
    """The taller strips that long pairs take (12 and 16 rows a lane, forced
    here): score and alignment across several strips, with the task's last row
    inside a lane, equal the oracle's."""
    from paper_2211_10769_gb300 import binding
    monkeypatch.setenv("SWGB_FWD", "%d,4" % R)
    c = binding.Context(0)
    try:
        seed = W.BASE_SEED + 15700 + 10 * R + alg
        sc = W.dna_scoring()
        A = W.uniform_dna(3 * 4 * 32 * R + 37, seed)
        B = W.mutate(A, 4, seed + 1, p_sub=0.1, p_indel=0.02)
        _score_case(c, oracle_mod, A, B, sc.matrix, sc.gap_open, sc.gap_extend, alg)
        _align_case(c, oracle_mod, A, B, sc.matrix, sc.gap_open, sc.gap_extend, alg)
        p = W.protein_scoring()
        P = W.random_protein(2 * 4 * 32 * R + 5, seed + 2)
        Q = W.mutate(P, 20, seed + 3, p_sub=0.3)
        _score_case(c, oracle_mod, P, Q, p.matrix, p.gap_open, p.gap_extend, alg)
        _align_case(c, oracle_mod, P[: 4 * 32 * R + 9], Q, p.matrix, p.gap_open, p.gap_extend, alg)
    finally:
        c.close()


@pytest.mark.parametrize("alg", ALGS)
def test_two_level_checkpoints(oracle_mod, monkeypatch, alg):
    """Two levels of checkpoints (forced: coarse every 3,072, fine every
    1,024) with the algorithms' borders on the coarse tiles of the first row
    and column."""
    from paper_2211_10769_gb300 import binding
    monkeypatch.setenv("SWGB_TWO_LEVEL", "3072,1024")
    c = binding.Context(0)
    try:
        seed = W.BASE_SEED + 15800 + alg
        sc = W.dna_scoring()
        A = W.uniform_dna(8500, seed)
        B = np.concatenate([W.uniform_dna(700, seed + 1), W.mutate(A[:7000], 4, seed + 2, p_sub=0.1, p_indel=0.02)])
        _align_case(c, oracle_mod, A, B, sc.matrix, sc.gap_open, sc.gap_extend, alg)
        _align_case(c, oracle_mod, B, A, sc.matrix, sc.gap_open, sc.gap_extend, alg)
    finally:
        c.close()


def test_batch_mixed_algorithms(ctx, oracle_mod):
    """One batch mixing the four algorithms, DNA and protein, empty sides included."""
    from paper_2211_10769_gb300 import binding
    d, p = W.dna_scoring(), W.protein_scoring()
    scorings = [(d.matrix, d.gap_open, d.gap_extend, alg) for alg in (0, 1, 2, 3)] + \
               [(p.matrix, p.gap_open, p.gap_extend, alg) for alg in (0, 1, 2, 3)]
    g = np.random.default_rng(W.BASE_SEED + 15700)
    pairs = []
    for k in range(200):
        si = int(g.integers(0, 8))
        m = int(g.integers(0, 1800)) if k % 9 else 0
        n = int(g.integers(0, 1800)) if k % 11 else 0
        if si < 4:
            a = W.uniform_dna(m, W.BASE_SEED + 15710 + k)
            b = W.mutate(a, 4, W.BASE_SEED + 15720 + k)[:n] if k % 2 else W.uniform_dna(n, W.BASE_SEED + 15730 + k)
        else:
            a = W.random_protein(m, W.BASE_SEED + 15710 + k)
            b = W.mutate(a, 20, W.BASE_SEED + 15720 + k, p_sub=0.3)[:n] if k % 2 else W.random_protein(n, W.BASE_SEED + 15730 + k)
        pairs.append((a, b, si))
    want = []
    for a, b, si in pairs:
        mat, go, ge, alg = scorings[si]
        want.append(oracle_mod.score_alg(a, b, mat, go, ge, alg))
    for flags in (0, binding.SW_BATCH_GRAPH):
        plan = binding.Batch(ctx, pairs, scorings, flags=flags)
        got = plan.run()
        assert [(h.score, h.a_end, h.b_end) for h in got] == want
        plan.close()


def test_local_only_calls_reject_other_algorithms(ctx):
    import ctypes
    import torch
    from paper_2211_10769_gb300 import binding
    p = W.protein_scoring()
    db = binding.Database(ctx, W.random_protein(500, 1), np.array([0, 200, 500], dtype=np.int64))
    lib = binding.load()
    sc, keep = binding._scoring(p.matrix, p.gap_open, p.gap_extend, binding.ALG_GLOBAL)
    hits = (binding._DbHit * 4)()
    nh = ctypes.c_int32()
    q = W.random_protein(100, 2)
    rc = lib.sw_dbsearch(ctx.handle, db.handle, q.ctypes.data, q.size, ctypes.byref(sc), 4, hits,
                         ctypes.byref(nh), None)
    assert rc == binding.SW_EINVAL
    a = torch.from_numpy(W.uniform_dna(100, 3)).cuda()
    d = W.dna_scoring()
    sc2, keep2 = binding._scoring(d.matrix, d.gap_open, d.gap_extend, binding.ALG_OVERLAP)
    hit = binding._Hit()
    lib.sw_score_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.POINTER(binding._Scoring), ctypes.POINTER(binding._Hit)]
    rc = lib.sw_score_noalloc(None, ctypes.c_void_p(a.data_ptr()), a.numel(), ctypes.c_void_p(a.data_ptr()),
                              a.numel(), ctypes.byref(sc2), ctypes.byref(hit))
    assert rc == binding.SW_EINVAL
    bad, keep3 = binding._scoring(d.matrix, d.gap_open, d.gap_extend, 4)   # no such algorithm
    rc = lib.sw_score(ctx.handle, ctypes.c_void_p(a.data_ptr()), a.numel(), ctypes.c_void_p(a.data_ptr()),
                      a.numel(), ctypes.byref(bad), ctypes.byref(hit))
    assert rc == binding.SW_EINVAL
    db.close()
