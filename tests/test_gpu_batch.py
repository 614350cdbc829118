"""GPU parity of the batched path (sw_batch_* / sw_score_batch): one launch
over many uneven DNA and protein pairs gives, pair by pair, the oracle's
score and end cell; graph replay and autotuning leave results unchanged."""
import os
from concurrent.futures import ThreadPoolExecutor

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


def _scorings():
    d, p = W.dna_scoring(), W.protein_scoring()
    return [(d.matrix, d.gap_open, d.gap_extend), (p.matrix, p.gap_open, p.gap_extend)]


def _mixed_pairs(seed, count, lo=0, hi=3000):
    g = np.random.default_rng(seed)
    pairs = []
    for k in range(count):
        m = int(np.exp(g.uniform(np.log(1), np.log(hi)))) if k % 7 else int(g.integers(lo, 40))
        n = int(np.exp(g.uniform(np.log(1), np.log(hi)))) if k % 5 else int(g.integers(lo, 40))
        if k % 2 == 0:
            a = g.integers(0, 4, size=m).astype(np.uint8)
            b = W.mutate(a, 4, seed + k)[:n] if k % 3 == 0 else g.integers(0, 4, size=n).astype(np.uint8)
            pairs.append((a, b, 0))
        else:
            a = W.random_protein(m, seed + k)
            b = W.mutate(a, 20, seed + k, p_sub=0.3)[:n] if k % 3 == 0 else W.random_protein(n, seed + 7 * k)
            pairs.append((a, b, 1))
    return pairs


def _oracle_hits(oracle_mod, pairs, scorings):
    out = []
    for a, b, si in pairs:
        mat, go, ge = scorings[si]
        out.append(oracle_mod.sw_score(a, b, mat, go, ge))
    return out


@pytest.mark.parametrize("flags", [0, 1, 3])
def test_batch_matches_oracle(ctx, oracle_mod, flags):
    from paper_2211_10769_gb300 import binding
    sc = _scorings()
    pairs = _mixed_pairs(W.BASE_SEED + 12000 + flags, 240)
    want = _oracle_hits(oracle_mod, pairs, sc)
    plan = binding.Batch(ctx, pairs, sc, flags=flags)
    for _ in range(2):                       # a plan reruns (graph replay when flags has the bit)
        got = plan.run()
        assert [(h.score, h.a_end, h.b_end) for h in got] == want
    plan.close()


@pytest.mark.parametrize("R,Wc", [(8, 4), (12, 4), (16, 4), (8, 2), (12, 2), (16, 2)])
def test_batch_packed_lanes(oracle_mod, monkeypatch, R, Wc):
    """Bins forced onto the packed 16-bit fill (both alphabets keep it exact at
    these strip heights), in blocks of four or two compute warps: every pair's
    score and end cell equal the oracle's, including pairs that span several
    strips and last strips that leave warps without rows."""
    from paper_2211_10769_gb300 import binding
    monkeypatch.setenv("SWGB_BATCH", "%d,%d,1" % (R, Wc))
    c = binding.Context(0)
    try:
        sc = _scorings()
        pairs = _mixed_pairs(W.BASE_SEED + 12100 + R, 160, hi=4500)
        assert sum(len(a) > 32 * Wc * R for a, _, _ in pairs) >= 3
        want = _oracle_hits(oracle_mod, pairs, sc)
        plan = binding.Batch(c, pairs, sc, flags=0)
        bins = plan.bins()
        assert bins and all(lb == 16 and r == R and w == Wc for r, w, lb, _ in bins), bins
        got = plan.run()
        assert [(h.score, h.a_end, h.b_end) for h in got] == want
        plan.close()
    finally:
        c.close()


def test_batch_device_inputs_and_empty(ctx, oracle_mod):
    import torch
    from paper_2211_10769_gb300 import binding
    sc = _scorings()
    pairs = _mixed_pairs(W.BASE_SEED + 12100, 60)
    ares, aoff, bres, boff, sidx = binding.Batch.packed(pairs)
    dev = (torch.from_numpy(ares).cuda(), torch.from_numpy(bres).cuda())
    plan = binding.Batch(ctx, pairs, sc, flags=1, device_inputs=dev)
    assert [(h.score, h.a_end, h.b_end) for h in plan.run()] == _oracle_hits(oracle_mod, pairs, sc)
    plan.close()
    empty = binding.Batch(ctx, [], sc)
    assert empty.run() == []
    empty.close()


def test_batch_rejects_bad_codes(ctx):
    from paper_2211_10769_gb300 import binding
    sc = _scorings()
    a = W.uniform_dna(50, 1)
    bad = W.random_protein(50, 2)           # protein codes against the DNA scoring
    with pytest.raises(binding.SwError) as ei:
        binding.Batch(ctx, [(a, a, 0), (a, bad, 0)], sc)
    assert ei.value.status == binding.SW_EINVAL


def test_full_batch_workload(ctx, oracle_mod):
    """The 10,000-pair workload (lengths log-uniform on [100, 20,000], half DNA,
    half protein): batched results equal one sw_score per pair for every pair,
    and the oracle on a seeded sample of the smaller pairs."""
    from paper_2211_10769_gb300 import binding
    sc = _scorings()
    raw = W.batch_pairs(10_000)
    pairs = [(a, b, 0 if kind == "dna" else 1) for a, b, kind in raw]
    plan = binding.Batch(ctx, pairs, sc, flags=binding.SW_BATCH_GRAPH | binding.SW_BATCH_AUTOTUNE)
    got = plan.run()
    assert plan.run() == got
    for k, (a, b, si) in enumerate(pairs):
        mat, go, ge = sc[si]
        h = ctx.score(a, b, mat, go, ge)
        assert (h.score, h.a_end, h.b_end) == (got[k].score, got[k].a_end, got[k].b_end), k
    g = np.random.default_rng(W.BASE_SEED + 12200)
    small = [k for k, (a, b, _) in enumerate(pairs) if len(a) * len(b) < 4_000_000]
    check = [int(k) for k in g.choice(small, size=40, replace=False)]
    # and the largest pairs of each alphabet (near 20,000 x 20,000, the long-query bin)
    for si in (0, 1):
        ks = sorted((k for k in range(len(pairs)) if pairs[k][2] == si),
                    key=lambda k: -len(pairs[k][0]) * len(pairs[k][1]))
        check += [k for k in ks if len(pairs[k][0]) > 1024][:3]
    assert sum(len(pairs[k][0]) * len(pairs[k][1]) > 3e8 for k in check) >= 4

    def oracle_hit(k):
        a, b, si = pairs[k]
        mat, go, ge = sc[si]
        return oracle_mod.sw_score(a, b, mat, go, ge)

    # the oracle is a ctypes call, which releases the GIL: threads run it in parallel
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        want = list(ex.map(oracle_hit, check))
    for k, w in zip(check, want):
        assert w == (got[k].score, got[k].a_end, got[k].b_end), k
    plan.close()
