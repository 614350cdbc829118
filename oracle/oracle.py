"""Python face of the CPU oracle (``sw_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  The CUDA library and
its binding never do, and this module never imports them.

The oracle is plain scalar C (Smith-Waterman local alignment with Gotoh
affine gaps, paper Section 2.1.2; penalties and matrices as in Sections 2.2
and 3.2).  Every function here only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "sw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def compile_source(src: str, out: str) -> str:
    """Compile one C file of the oracle into a shared library (plain gcc -O2)."""
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, src])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile sw_oracle.c into liboracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(SOURCE):
        compile_source(SOURCE, _LIB)
    return _LIB


def _u8(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


def _mat(S) -> np.ndarray:
    S = np.ascontiguousarray(np.asarray(S, dtype=np.int8))
    assert S.ndim == 2 and S.shape[0] == S.shape[1]
    return S


def _ptr(arr: np.ndarray):
    return arr.ctypes.data if arr.size else None


@dataclass(frozen=True)
class Alignment:
    score: int
    a_begin: int
    a_end: int
    b_begin: int
    b_end: int
    cigar: str


def cigar_from_ops(ops: str) -> str:
    """Run-length encode a string of M/I/D operations."""
    out = []
    k = 0
    while k < len(ops):
        t = k
        while t < len(ops) and ops[t] == ops[k]:
            t += 1
        out.append("%d%s" % (t - k, ops[k]))
        k = t
    return "".join(out)


class OracleLib:
    """ctypes handle on one compiled copy of the oracle."""

    cigar_from_ops = staticmethod(cigar_from_ops)

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.c_void_p
        lib.oracle_sw_score.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, u8p,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i64p, i64p]
        for fn in (lib.oracle_sw_align_full, lib.oracle_sw_align_ptr):
            fn.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, u8p, ctypes.c_int,
                           ctypes.c_int, ctypes.c_int, i64p, i64p, i64p, i64p, i64p,
                           ctypes.c_char_p, i64p]
        lib.oracle_encode.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int64, u8p, i64p]
        lib.oracle_nw_score.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, u8p,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p]
        lib.oracle_align_alg.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, u8p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i64p, i64p,
                                         i64p, i64p, ctypes.c_char_p, i64p]
        lib.oracle_score_alg.argtypes = [u8p, ctypes.c_int64, u8p, ctypes.c_int64, u8p, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i64p, i64p]
        self.lib = lib

    def sw_score(self, a, b, S, gap_open: int, gap_extend: int):
        """(score, a_end, b_end) of the best local alignment, canonical end cell."""
        a, b, S = _u8(a), _u8(b), _mat(S)
        sc, ae, be = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = self.lib.oracle_sw_score(_ptr(a), a.size, _ptr(b), b.size, S.ctypes.data,
                                      S.shape[0], int(gap_open), int(gap_extend),
                                      ctypes.byref(sc), ctypes.byref(ae), ctypes.byref(be))
        if rc != 0:
            raise ValueError("oracle_sw_score failed with %d" % rc)
        return sc.value, ae.value, be.value

    def nw_score(self, a, b, S, gap_open: int, gap_extend: int) -> int:
        """Global (end-to-end) Gotoh score of a against b."""
        a, b, S = _u8(a), _u8(b), _mat(S)
        sc = ctypes.c_int64()
        rc = self.lib.oracle_nw_score(_ptr(a), a.size, _ptr(b), b.size, S.ctypes.data, S.shape[0],
                                      int(gap_open), int(gap_extend), ctypes.byref(sc))
        if rc != 0:
            raise ValueError("oracle_nw_score failed (%d)" % rc)
        return sc.value

    def align_alg(self, a, b, S, gap_open: int, gap_extend: int, alg: int) -> Alignment:
        """Canonical alignment of algorithm alg (0 SW, 1 NW, 2 HW, 3 OV) from full matrices."""
        a, b, S = _u8(a), _u8(b), _mat(S)
        ops = ctypes.create_string_buffer(a.size + b.size + 1)
        vals = [ctypes.c_int64() for _ in range(6)]
        rc = self.lib.oracle_align_alg(_ptr(a), a.size, _ptr(b), b.size, S.ctypes.data, S.shape[0],
                                       int(gap_open), int(gap_extend), int(alg),
                                       *[ctypes.byref(v) for v in vals[:5]], ops, ctypes.byref(vals[5]))
        if rc != 0:
            raise ValueError("oracle_align_alg failed with %d" % rc)
        score, ab, ae, bb, be, nops = (v.value for v in vals)
        return Alignment(score, ab, ae, bb, be, cigar_from_ops(ops.raw[:nops].decode()))

    def score_alg(self, a, b, S, gap_open: int, gap_extend: int, alg: int):
        """(score, a_end, b_end) of algorithm alg in linear memory."""
        a, b, S = _u8(a), _u8(b), _mat(S)
        sc, ae, be = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = self.lib.oracle_score_alg(_ptr(a), a.size, _ptr(b), b.size, S.ctypes.data, S.shape[0],
                                       int(gap_open), int(gap_extend), int(alg),
                                       ctypes.byref(sc), ctypes.byref(ae), ctypes.byref(be))
        if rc != 0:
            raise ValueError("oracle_score_alg failed with %d" % rc)
        return sc.value, ae.value, be.value

    def _align(self, fn, a, b, S, gap_open, gap_extend) -> Alignment:
        a, b, S = _u8(a), _u8(b), _mat(S)
        ops = ctypes.create_string_buffer(a.size + b.size + 1)
        vals = [ctypes.c_int64() for _ in range(6)]
        rc = fn(_ptr(a), a.size, _ptr(b), b.size, S.ctypes.data, S.shape[0], int(gap_open),
                int(gap_extend), *[ctypes.byref(v) for v in vals[:5]], ops,
                ctypes.byref(vals[5]))
        if rc != 0:
            raise ValueError("oracle alignment failed with %d" % rc)
        score, ab, ae, bb, be, nops = (v.value for v in vals)
        return Alignment(score, ab, ae, bb, be, cigar_from_ops(ops.raw[:nops].decode()))

    def sw_align(self, a, b, S, gap_open: int, gap_extend: int) -> Alignment:
        """Canonical alignment from the full H/E/F matrices (24 bytes per cell)."""
        return self._align(self.lib.oracle_sw_align_full, a, b, S, gap_open, gap_extend)

    def sw_align_ptr(self, a, b, S, gap_open: int, gap_extend: int) -> Alignment:
        """Canonical alignment from one traceback-pointer byte per cell."""
        return self._align(self.lib.oracle_sw_align_ptr, a, b, S, gap_open, gap_extend)

    def encode(self, alphabet: str, text: str) -> np.ndarray:
        """Residue codes of ``text`` in ``alphabet``; ValueError on a foreign letter."""
        raw = text.encode("ascii")
        codes = np.zeros(len(raw), dtype=np.uint8)
        bad = ctypes.c_int64()
        rc = self.lib.oracle_encode(alphabet.encode("ascii"), raw, len(raw), _ptr(codes),
                                    ctypes.byref(bad))
        if rc != 0:
            raise ValueError("character %d not in alphabet" % bad.value)
        return codes


_default = None


def _get() -> OracleLib:
    global _default
    if _default is None:
        _default = OracleLib(build())
    return _default


def sw_score(a, b, S, gap_open: int, gap_extend: int):
    """(score, a_end, b_end) of the best local alignment, canonical end cell."""
    return _get().sw_score(a, b, S, gap_open, gap_extend)


def sw_align(a, b, S, gap_open: int, gap_extend: int) -> Alignment:
    """Canonical alignment from the full H/E/F matrices."""
    return _get().sw_align(a, b, S, gap_open, gap_extend)


def sw_align_ptr(a, b, S, gap_open: int, gap_extend: int) -> Alignment:
    """Canonical alignment from traceback pointers."""
    return _get().sw_align_ptr(a, b, S, gap_open, gap_extend)


def nw_score(a, b, S, gap_open: int, gap_extend: int) -> int:
    """Global (end-to-end) Gotoh score: checks pieces of long local alignments."""
    return _get().nw_score(a, b, S, gap_open, gap_extend)


def encode(alphabet: str, text: str) -> np.ndarray:
    """Residue codes of ``text`` in ``alphabet``."""
    return _get().encode(alphabet, text)


# The algorithms of paper Section 2.1: local (Smith-Waterman), global
# (Needleman-Wunsch), semi-global (all of a inside b) and overlap.
ALG_SW, ALG_NW, ALG_HW, ALG_OV = 0, 1, 2, 3


def align_alg(a, b, S, gap_open: int, gap_extend: int, alg: int) -> Alignment:
    """Canonical alignment of one of the four algorithms (full matrices)."""
    return _get().align_alg(a, b, S, gap_open, gap_extend, alg)


def score_alg(a, b, S, gap_open: int, gap_extend: int, alg: int):
    """(score, a_end, b_end) of one of the four algorithms (linear memory)."""
    return _get().score_alg(a, b, S, gap_open, gap_extend, alg)


def db_scores(query, subjects, S, gap_open: int, gap_extend: int) -> np.ndarray:
    """Local score of the query against every subject, one oracle call each."""
    return np.array([sw_score(query, s, S, gap_open, gap_extend)[0] for s in subjects],
                    dtype=np.int64)


def top_k(scores, k: int):
    """Top-k (subject, score): score descending, then subject index ascending."""
    order = sorted(range(len(scores)), key=lambda s: (-int(scores[s]), s))
    return [(s, int(scores[s])) for s in order[:k]]
