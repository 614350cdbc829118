"""sw_score_noalloc: the allocation-free variant of the pairwise score fill.

It serves callers that cannot call cudaMalloc (a process whose own caching
allocator owns the device memory budget, or a pipeline that must avoid the
device synchronisation cudaMalloc / cudaFree imply).  Its scratch is a fixed
array inside the library.  This file is collected last so that a run that
stops at the first failure has already run every other test; it passes
alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_2211_10769_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2211_10769_gb300 import binding, build
    build.build()
    lib = binding.load()
    lib.sw_score_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.POINTER(binding._Scoring), ctypes.POINTER(binding._Hit)]
    torch.cuda.set_device(0)
    ctx = binding.Context(0)
    yield lib, ctx, torch, binding
    ctx.close()


def _noalloc(env, a, b, sc):
    lib, ctx, torch, binding = env
    da = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    db = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    scoring, keep = binding._scoring(sc.matrix, sc.gap_open, sc.gap_extend)
    hit = binding._Hit()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.sw_score_noalloc(stream, da.data_ptr() if da.numel() else None, da.numel(),
                              db.data_ptr() if db.numel() else None, db.numel(),
                              ctypes.byref(scoring), ctypes.byref(hit))
    return rc, (hit.score, hit.a_end, hit.b_end)


def test_noalloc_matches_sw_score_and_oracle_twice_in_a_row(env, oracle_mod):
    lib, ctx, torch, binding = env
    cases = [
        (W.dna_scoring(), *W.dna_pair_2k()),
        (W.dna_scoring(), *W.dna_long_pair(20_000)),
        (W.protein_scoring(), W.random_protein(3000, W.BASE_SEED + 70),
         W.mutate(W.random_protein(3000, W.BASE_SEED + 70), 20, W.BASE_SEED + 71, p_sub=0.3)),
    ]
    for sc, a, b in cases:
        want = oracle_mod.sw_score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
        h = ctx.score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
        assert (h.score, h.a_end, h.b_end) == want
        for _ in range(2):                   # the shared array keeps the previous call's contents
            rc, got = _noalloc(env, a, b, sc)
            assert rc == 0
            assert got == want


def test_noalloc_more_strips_than_resident_blocks(env, oracle_mod):
    """About 1M rows x 2,000 columns: 977 strips of 1,024 rows, more than the
    blocks that fit the GPU at once, so later blocks take later tickets and
    reuse the two-slot boundary ring."""
    lib, ctx, torch, binding = env
    sc = W.dna_scoring()
    b = W.uniform_dna(2_000, W.BASE_SEED + 80)
    a = np.concatenate([W.uniform_dna(600_000, W.BASE_SEED + 81),
                        W.mutate(b, 4, W.BASE_SEED + 82, p_sub=0.05),
                        W.uniform_dna(398_000, W.BASE_SEED + 83)])
    want = oracle_mod.sw_score(a, b, sc.matrix, sc.gap_open, sc.gap_extend)
    assert want[0] > 1000                    # the planted copy, far down the rows
    for _ in range(2):
        rc, got = _noalloc(env, a, b, sc)
        assert rc == 0
        assert got == want


def test_noalloc_rejects_oversize_and_host_input(env):
    lib, ctx, torch, binding = env
    sc = W.dna_scoring()
    rc, _ = _noalloc(env, W.uniform_dna(10, 1), W.uniform_dna(262_145, 2), sc)
    assert rc == binding.SW_ERANGE
    rc, _ = _noalloc(env, W.uniform_dna(16_384 * 1_024 + 1, 4), W.uniform_dna(10, 5), sc)
    assert rc == binding.SW_ERANGE
    a = W.uniform_dna(100, 3)
    scoring, keep = binding._scoring(sc.matrix, sc.gap_open, sc.gap_extend)
    hit = binding._Hit()
    rc = lib.sw_score_noalloc(None, a.ctypes.data, a.size, a.ctypes.data, a.size,
                              ctypes.byref(scoring), ctypes.byref(hit))
    assert rc == binding.SW_EINVAL
    # still usable afterwards
    rc, got = _noalloc(env, a, a, sc)
    assert rc == 0 and got == (100, 100, 100)
