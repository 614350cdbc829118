"""Brute-force local alignment by enumeration, for tiny sequences.

Independent of the oracle's dynamic programme: it lists every local
alignment -- every start cell (i0, j0) and every string over {M, I, D}
that stays inside the sequences -- scores each one straight from the
definition (sum of S over M columns, minus open + (k-1)*extend for every
maximal run of k I's or k D's) and keeps the best.  Feasible for lengths up
to about 7.
"""
from __future__ import annotations


def enumerate_alignments(a, b, S, go, ge):
    """Yield (score, i0, j0, i1, j1, ops) for every non-empty local alignment."""
    m, n = len(a), len(b)
    for i0 in range(m + 1):
        for j0 in range(n + 1):
            # stack entries: (i, j, last_op, score, ops)
            stack = [(i0, j0, "", 0, "")]
            while stack:
                i, j, last, sc, ops = stack.pop()
                if ops:
                    yield sc, i0, j0, i, j, ops
                if i < m and j < n:
                    stack.append((i + 1, j + 1, "M", sc + int(S[a[i]][b[j]]), ops + "M"))
                if j < n:
                    stack.append((i, j + 1, "I", sc - (ge if last == "I" else go), ops + "I"))
                if i < m:
                    stack.append((i + 1, j, "D", sc - (ge if last == "D" else go), ops + "D"))


def brute_force_global(a, b, S, go, ge):
    """Best score over every global alignment (all of a against all of b),
    listed one by one and scored from the definition, for tiny sequences."""
    m, n = len(a), len(b)
    best = None
    stack = [(0, 0, "", 0)]
    while stack:
        i, j, last, sc = stack.pop()
        if i == m and j == n:
            best = sc if best is None else max(best, sc)
            continue
        if i < m and j < n:
            stack.append((i + 1, j + 1, "M", sc + int(S[a[i]][b[j]])))
        if j < n:
            stack.append((i, j + 1, "I", sc - (ge if last == "I" else go)))
        if i < m:
            stack.append((i + 1, j, "D", sc - (ge if last == "D" else go)))
    return best


def backward_moves(ops: str):
    """Rank sequence of the backward walk that reproduces ``ops``.

    Walking from the end cell: in state H a match column is rank 1, entering
    an I run rank 2, entering a D run rank 3 and stopping rank 0; inside a
    gap run, leaving it (the run was opened here) is rank 0 and extending
    is rank 1.  Runs are maximal, so the sequence is unique.
    """
    r = ops[::-1]
    out = []
    k = 0
    while k < len(r):
        c = r[k]
        t = k
        while t < len(r) and r[t] == c:
            t += 1
        L = t - k
        if c == "M":
            out.extend([1] * L)
        else:
            out.append(2 if c == "I" else 3)
            out.extend([1] * (L - 1))
            out.append(0)
        k = t
    out.append(0)
    return out


def brute_force(a, b, S, go, ge):
    """Best local score, its canonical end cell, and the canonical alignment.

    Returns (score, a_end, b_end, canonical) where canonical is
    (a_begin, b_begin, ops) or None for score 0.  The end cell is the
    smallest row then smallest column among optimal alignments; the
    canonical alignment is the optimal one ending there whose backward
    walk is lexicographically smallest by rank (see backward_moves).
    """
    best = 0
    cands = []
    for sc, i0, j0, i1, j1, ops in enumerate_alignments(a, b, S, go, ge):
        if sc > best:
            best = sc
            cands = [(i0, j0, i1, j1, ops)]
        elif sc == best and best > 0:
            cands.append((i0, j0, i1, j1, ops))
    if best == 0:
        return 0, 0, 0, None
    i_end, j_end = min((c[2], c[3]) for c in cands)
    at_end = [c for c in cands if c[2] == i_end and c[3] == j_end]
    canon = min(at_end, key=lambda c: backward_moves(c[4]))
    return best, i_end, j_end, (canon[0], canon[1], canon[4])


def rescore(a, b, S, go, ge, a_begin, b_begin, cigar):
    """Score a CIGAR (M/I/D runs) placed at (a_begin, b_begin) by the definition.

    Returns (score, a_end, b_end).  Written separately from the enumerator
    so it can check alignments reported by any implementation.
    """
    i, j, sc = a_begin, b_begin, 0
    num = ""
    for ch in cigar:
        if ch.isdigit():
            num += ch
            continue
        L = int(num)
        num = ""
        if ch == "M":
            for _ in range(L):
                sc += int(S[a[i]][b[j]])
                i += 1
                j += 1
        elif ch == "I":
            sc -= go + (L - 1) * ge
            j += L
        elif ch == "D":
            sc -= go + (L - 1) * ge
            i += L
        else:
            raise ValueError("bad CIGAR op %r" % ch)
    assert num == ""
    return sc, i, j


def _starts(alg, m, n):
    """Cells where an alignment of algorithm alg may start (NW, HW, OV)."""
    if alg == 1:
        return [(0, 0)]
    if alg == 2:
        return [(0, j) for j in range(n + 1)]
    return sorted(set([(i, 0) for i in range(m + 1)] + [(0, j) for j in range(n + 1)]))


def _end_ok(alg, i, j, m, n):
    if alg == 1:
        return i == m and j == n
    if alg == 2:
        return i == m
    return i == m or j == n


def brute_force_alg(a, b, S, go, ge, alg):
    """Best score, canonical end cell and canonical alignment of the global
    (alg 1), semi-global (alg 2, all of a inside b) or overlap (alg 3)
    problem, by listing every alignment that starts where the algorithm lets
    one start and ends where it lets one end, scored from the definition.

    Returns (score, a_end, b_end, (a_begin, b_begin, ops)).  The end cell is
    the smallest row, then column, among optimal alignments; the canonical
    alignment is the optimal one ending there whose backward walk is
    lexicographically smallest by rank (backward_moves).
    """
    m, n = len(a), len(b)
    best = None
    cands = []
    for i0, j0 in _starts(alg, m, n):
        stack = [(i0, j0, "", 0, "")]
        while stack:
            i, j, last, sc, ops = stack.pop()
            if _end_ok(alg, i, j, m, n):
                if best is None or sc > best:
                    best, cands = sc, [(i0, j0, i, j, ops)]
                elif sc == best:
                    cands.append((i0, j0, i, j, ops))
            if i < m and j < n:
                stack.append((i + 1, j + 1, "M", sc + int(S[a[i]][b[j]]), ops + "M"))
            if j < n:
                stack.append((i, j + 1, "I", sc - (ge if last == "I" else go), ops + "I"))
            if i < m:
                stack.append((i + 1, j, "D", sc - (ge if last == "D" else go), ops + "D"))
    i_end, j_end = min((c[2], c[3]) for c in cands)
    at_end = [c for c in cands if c[2] == i_end and c[3] == j_end]
    canon = min(at_end, key=lambda c: backward_moves(c[4]))
    return best, i_end, j_end, (canon[0], canon[1], canon[4])
