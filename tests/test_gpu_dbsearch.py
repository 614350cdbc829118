"""GPU parity of the database search (sw_db_create / sw_dbsearch) against the
CPU oracle: every subject's score exactly, the top-k order (score
descending, subject index ascending), the packed-16-bit saturation path and
its exact 32-bit rescoring, long queries, and degenerate databases."""
import numpy as np
import pytest

from paper_2211_10769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2211_10769_gb300 import binding, build
    build.build()
    c = binding.Context(0)
    yield c
    c.close()


def _db(ctx, subjects):
    from paper_2211_10769_gb300 import binding
    lens = np.array([len(s) for s in subjects], dtype=np.int64)
    off = np.zeros(len(subjects) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    res = np.concatenate(subjects) if len(subjects) and off[-1] > 0 else np.zeros(0, np.uint8)
    return binding.Database(ctx, res, off)


def _check_all(ctx, oracle_mod, db, subjects, q, sc, k=20):
    hits, scores = db.search(q, sc.matrix, sc.gap_open, sc.gap_extend, k=k, all_scores=True)
    want = oracle_mod.db_scores(q, subjects, sc.matrix, sc.gap_open, sc.gap_extend)
    bad = np.nonzero(scores != want)[0]
    assert bad.size == 0, (bad[:10], scores[bad[:10]], want[bad[:10]])
    assert hits == oracle_mod.top_k(want, min(k, len(subjects)))
    return want


def test_small_database_all_scores(ctx, oracle_mod):
    sc = W.protein_scoring()
    qs = W.protein_queries((144, 464))
    pdb = W.protein_db(3000, queries=qs, seed_offset=700)
    subjects = [pdb.subject(s) for s in range(pdb.nseq)]
    db = _db(ctx, subjects)
    for qi, q in enumerate(qs):
        want = _check_all(ctx, oracle_mod, db, subjects, q, sc)
        top = oracle_mod.top_k(want, 3)
        assert {s for s, _ in top} & set(pdb.planted[qi])     # the planted homologs are found


def test_every_tile_shape(ctx, oracle_mod):
    """Query lengths that pick each tile shape of the packed search (two
    16-lane wavefronts a warp at 4, 6, 9 and 12 rows a lane; one 32-lane
    wavefront at 8 and 16 rows; 16-warp blocks for long queries), with one or
    several passes, the last pass partly padding, and warps whose second
    wavefront finds no pair left."""
    sc = W.protein_scoring()
    lengths = (1, 31, 80, 100, 128, 144, 160, 161, 190, 250, 300, 350, 384, 464, 700, 1000, 1500, 4100)
    qs = W.protein_queries(lengths, seed_offset=760)
    pdb = W.protein_db(400, queries=qs, seed_offset=770)
    subjects = [pdb.subject(s) for s in range(pdb.nseq)]
    db = _db(ctx, subjects)
    for q in qs:
        _check_all(ctx, oracle_mod, db, subjects, q, sc)


@pytest.mark.parametrize("nseq", [1, 2, 3, 5, 7])
def test_tiny_databases_short_queries(ctx, oracle_mod, nseq):
    """One to four subject pairs against queries that take the two-wavefront
    shapes: most warps find one pair or none, and a warp's second wavefront
    often has no pair (its lanes still take part in the shuffles)."""
    sc = W.protein_scoring()
    g = np.random.default_rng(W.BASE_SEED + 780 + nseq)
    subjects = [W.random_protein(int(g.integers(1, 400)), W.BASE_SEED + 790 + 10 * nseq + i) for i in range(nseq)]
    db = _db(ctx, subjects)
    for m in (5, 60, 90, 140, 190):
        q = W.random_protein(m, W.BASE_SEED + 800 + m)
        if nseq > 2:
            subjects_q = list(subjects)
            subjects_q[1] = W.mutate(q, 20, W.BASE_SEED + 801 + m, p_sub=0.2)   # a homolog among them
            dbq = _db(ctx, subjects_q)
            _check_all(ctx, oracle_mod, dbq, subjects_q, q, sc, k=min(4, nseq))
        _check_all(ctx, oracle_mod, db, subjects, q, sc, k=min(4, nseq))


def test_long_query_and_dna(ctx, oracle_mod):
    sc = W.protein_scoring()
    q = W.protein_queries((5478,))[0]
    pdb = W.protein_db(160, queries=[q], seed_offset=710)
    subjects = [pdb.subject(s) for s in range(pdb.nseq)]
    _check_all(ctx, oracle_mod, _db(ctx, subjects), subjects, q, sc)
    dna = W.dna_scoring()
    dsubj = [W.uniform_dna(int(L), W.BASE_SEED + 720 + i) for i, L in enumerate(np.linspace(1, 900, 97))]
    dq = W.uniform_dna(700, W.BASE_SEED + 719)
    dsubj[5] = W.mutate(dq, 4, W.BASE_SEED + 730)
    _check_all(ctx, oracle_mod, _db(ctx, dsubj), dsubj, dq, dna, k=10)


def test_saturating_subjects_are_rescored(ctx, oracle_mod):
    """Scores above 32767 - max(S) cannot stay in 16-bit lanes: a W-rich query
    against W-rich subjects pushes them over; those must come back exact."""
    sc = W.protein_scoring()
    Wc = W.PROTEIN_ALPHABET.index("W")
    g = np.random.default_rng(W.BASE_SEED + 740)
    q = np.full(3300, Wc, np.uint8)
    q[g.integers(0, 3300, 40)] = 0
    subjects = []
    for i in range(40):
        if i % 4 == 0:
            s = q.copy()
            s[g.integers(0, len(s), 30)] = 3
        else:
            s = W.random_protein(int(g.integers(50, 900)), W.BASE_SEED + 750 + i)
        subjects.append(s)
    want = _check_all(ctx, oracle_mod, _db(ctx, subjects), subjects, q, sc)
    assert (want > 32767 - 11).sum() >= 10


def test_degenerate_databases(ctx, oracle_mod):
    sc = W.protein_scoring()
    q = W.random_protein(200, W.BASE_SEED + 760)
    subjects = [np.zeros(0, np.uint8), W.random_protein(1, 1), np.zeros(0, np.uint8), W.random_protein(31, 2),
                W.random_protein(33, 3)]
    _check_all(ctx, oracle_mod, _db(ctx, subjects), subjects, q, sc, k=64)      # k > nseq
    one = [W.random_protein(250, 4)]
    _check_all(ctx, oracle_mod, _db(ctx, one), one, q, sc, k=5)
    hits, scores = _db(ctx, one).search(np.zeros(0, np.uint8), sc.matrix, 10, 1, k=3, all_scores=True)
    assert hits == [(0, 0)] and scores.tolist() == [0]


def test_full_size_database_sampled(ctx, oracle_mod):
    """The 500,000-subject database: every query's top hits and a seeded
    sample of subjects checked against the oracle one by one."""
    sc = W.protein_scoring()
    qs = W.protein_queries()
    pdb = W.protein_db(500_000, queries=qs)
    from paper_2211_10769_gb300 import binding
    db = binding.Database(ctx, pdb.residues, pdb.offsets)
    g = np.random.default_rng(W.BASE_SEED + 770)
    for qi, q in enumerate(qs):
        hits, scores = db.search(q, sc.matrix, sc.gap_open, sc.gap_extend, k=20, all_scores=True)
        nsample = 400 if len(q) < 1500 else 120
        sample = sorted(set(g.integers(0, pdb.nseq, nsample).tolist()) | set(pdb.planted[qi]) |
                        {s for s, _ in hits[:5]})
        for s in sample:
            assert scores[s] == oracle_mod.sw_score(q, pdb.subject(s), sc.matrix, sc.gap_open, sc.gap_extend)[0]
        # top-k is consistent with the score array (score desc, index asc)
        order = np.lexsort((np.arange(pdb.nseq), -scores.astype(np.int64)))[:20]
        assert hits == [(int(s), int(scores[s])) for s in order]
        assert set(pdb.planted[qi]) <= {s for s, _ in hits}
