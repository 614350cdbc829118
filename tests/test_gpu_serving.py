"""GPU tests of the serving loop (sw_server_*): continuous batching over a
device-resident database.  Every request's hits must be the same alone
(sw_dbsearch) and in the mix, admission follows the slot count and the
memory budget, and results match the oracle."""
import numpy as np
import pytest

from paper_2211_10769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2211_10769_gb300 import binding, build
    build.build()
    ctx = binding.Context(0)
    pdb = W.protein_db(6000, seed_offset=800)
    db = binding.Database(ctx, pdb.residues, pdb.offsets)
    yield ctx, pdb, db, binding
    db.close()
    ctx.close()


def _queries(n, seed):
    g = np.random.default_rng(seed)
    return [W.random_protein(W.log_uniform_int(g, 50, 5000), seed + i) for i in range(n)]


def test_alone_equals_mix(env):
    """Requests arrive while others are in the sweep; between steps (with a
    step in flight) the context also runs plain searches, which must not
    disturb the server's buffers nor be disturbed by them."""
    ctx, pdb, db, binding = env
    sc = W.protein_scoring()
    qs = _queries(14, W.BASE_SEED + 810)
    qs[3] = W.mutate(pdb.subject(77), 20, W.BASE_SEED + 820, p_sub=0.2)     # a query with a true homolog
    alone = [db.search(q, sc.matrix, sc.gap_open, sc.gap_extend, k=20)[0] for q in qs]
    srv = binding.Server(ctx, db, sc.matrix, sc.gap_open, sc.gap_extend, mem_budget=1 << 30, k=20,
                         max_slots=5, chunks=7)
    pending = list(range(len(qs)))
    tickets, results, step = {}, {}, 0
    while len(results) < len(qs):
        # arrivals: two new requests every other step, admitted as slots free up
        if step % 2 == 0:
            for _ in range(2):
                if pending:
                    t = srv.submit(qs[pending[0]])
                    if t is None:
                        break
                    tickets[t] = pending.pop(0)
        srv.step()
        if step % 3 == 1:
            qi = (step // 3) % len(qs)
            assert db.search(qs[qi], sc.matrix, sc.gap_open, sc.gap_extend, k=20)[0] == alone[qi]
        for t, qi in list(tickets.items()):
            r = srv.poll(t)
            if r is not None:
                results[qi] = r
                del tickets[t]
        step += 1
        assert step < 1000
    for qi in range(len(qs)):
        assert results[qi] == alone[qi], qi
    assert results[3][0][0] == 77
    srv.close()


def test_admission_by_slots_and_memory(env):
    ctx, pdb, db, binding = env
    sc = W.protein_scoring()
    qs = _queries(6, W.BASE_SEED + 830)
    # device bytes the server reserves per request: two int32 arrays per subject plus the query
    per_request = [8 * pdb.nseq + len(q) + 512 for q in qs]
    srv = binding.Server(ctx, db, sc.matrix, sc.gap_open, sc.gap_extend,
                         mem_budget=per_request[0] + per_request[1], k=5, max_slots=8, chunks=3)
    t0, t1 = srv.submit(qs[0]), srv.submit(qs[1])
    assert t0 is not None and t1 is not None
    assert srv.submit(qs[2]) is None                 # memory budget full
    assert srv.stats()[0] == 2
    for _ in range(3):
        srv.step()
    # steps are pipelined: the third call enqueued the last chunk, the fourth completes it
    assert srv.poll(t0) is None and srv.poll(t1) is None
    srv.step()
    assert srv.poll(t0) is not None and srv.poll(t1) is not None
    assert srv.stats()[:2] == (0, 0)
    assert srv.submit(qs[2]) is not None             # admitted once memory is back
    srv.close()
    srv = binding.Server(ctx, db, sc.matrix, sc.gap_open, sc.gap_extend, mem_budget=1 << 30, k=5,
                         max_slots=1, chunks=2)
    assert srv.submit(qs[3]) is not None and srv.submit(qs[4]) is None   # one slot
    srv.close()


def test_serving_matches_oracle_and_rejects_bad_input(env, oracle_mod):
    ctx, pdb, db, binding = env
    sc = W.protein_scoring()
    small = [pdb.subject(s) for s in range(300)]
    off = np.zeros(301, np.int64)
    np.cumsum([len(x) for x in small], out=off[1:])
    sdb = binding.Database(ctx, np.concatenate(small), off)
    srv = binding.Server(ctx, sdb, sc.matrix, sc.gap_open, sc.gap_extend, mem_budget=1 << 28, k=10,
                         max_slots=4, chunks=4)
    qs = _queries(4, W.BASE_SEED + 840)
    ts = [srv.submit(q) for q in qs]
    for _ in range(4 + 1):
        srv.step()
    for t, q in zip(ts, qs):
        want = oracle_mod.top_k(oracle_mod.db_scores(q, small, sc.matrix, sc.gap_open, sc.gap_extend), 10)
        assert srv.poll(t) == want
    bad = qs[0].copy()
    bad[3] = 30
    with pytest.raises(binding.SwError):
        srv.submit(bad)
    with pytest.raises(binding.SwError):
        srv.poll(123456)
    srv.close()
    sdb.close()


def test_destroy_with_a_step_in_flight(env, oracle_mod):
    """Steps are pipelined: after a step call the step it enqueued is still on
    the device.  Destroying the server then waits for it; the context and the
    database stay usable, and a new server gives the oracle's hits."""
    ctx, pdb, db, binding = env
    sc = W.protein_scoring()
    qs = _queries(3, W.BASE_SEED + 850)
    srv = binding.Server(ctx, db, sc.matrix, sc.gap_open, sc.gap_extend, mem_budget=1 << 30, k=5,
                         max_slots=4, chunks=3)
    for q in qs:
        assert srv.submit(q) is not None
    assert srv.step() == 3                    # one chunk of each request enqueued
    srv.close()
    small = [pdb.subject(s) for s in range(200)]
    off = np.zeros(201, np.int64)
    np.cumsum([len(x) for x in small], out=off[1:])
    sdb = binding.Database(ctx, np.concatenate(small), off)
    srv = binding.Server(ctx, sdb, sc.matrix, sc.gap_open, sc.gap_extend, mem_budget=1 << 28, k=5,
                         max_slots=2, chunks=2)
    t = srv.submit(qs[0])
    steps = 0
    while (hits := srv.poll(t)) is None:
        srv.step()
        steps += 1
        assert steps < 10
    assert steps == 3                         # chunks + 1 step calls
    assert hits == oracle_mod.top_k(oracle_mod.db_scores(qs[0], small, sc.matrix, sc.gap_open, sc.gap_extend), 5)
    srv.close()
    sdb.close()
