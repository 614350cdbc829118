"""Thin Python binding of libswgb (include/sw.h): argument marshalling only.

Every step of the alignment runs in the CUDA library; this module converts
numpy arrays / torch tensors into pointers, calls the C entry points and
turns their outputs into Python values.  It raises if the compiled library
is missing -- there is no CPU fallback.

Sequences may be numpy uint8 arrays (host memory; the library copies them to
the device inside the call) or uint8 torch CUDA tensors (device memory).
"""
from __future__ import annotations

import ctypes
import os
import weakref
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libswgb.so")

SW_OK, SW_EINVAL, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT, SW_EAGAIN, SW_ERANGE = 0, -1, -2, -3, -4, -5, -6


class SwError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, _strerror(status), status))
        self.status = status


class _Scoring(ctypes.Structure):
    _fields_ = [("alphabet", ctypes.c_int32), ("matrix", ctypes.c_void_p),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32),
                ("algorithm", ctypes.c_int32)]


# sw_scoring.algorithm (paper Section 2.1): local, global, semi-global, overlap
ALG_LOCAL, ALG_GLOBAL, ALG_SEMIGLOBAL, ALG_OVERLAP = 0, 1, 2, 3


class _Hit(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("a_end", ctypes.c_int64), ("b_end", ctypes.c_int64)]


class _Alignment(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("a_begin", ctypes.c_int64), ("a_end", ctypes.c_int64),
                ("b_begin", ctypes.c_int64), ("b_end", ctypes.c_int64),
                ("cigar", ctypes.c_void_p), ("cigar_len", ctypes.c_int64)]


class _DbHit(ctypes.Structure):
    _fields_ = [("subject", ctypes.c_int64), ("score", ctypes.c_int32), ("flags", ctypes.c_uint32)]


_lib = None


def load():
    """Load libswgb.so (built by paper_2211_10769_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libswgb.so is not built (run `python -m paper_2211_10769_gb300.build`); "
                           "there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.sw_strerror.restype = ctypes.c_char_p
    lib.sw_strerror.argtypes = [i32]
    lib.sw_ctx_create.argtypes = [i32, vp, ctypes.POINTER(vp)]
    lib.sw_ctx_destroy.argtypes = [vp]
    lib.sw_ctx_destroy.restype = None
    lib.sw_encode.argtypes = [vp, ctypes.c_char_p, vp, i64, vp]
    lib.sw_score.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(_Scoring), ctypes.POINTER(_Hit)]
    lib.sw_align.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(_Scoring), ctypes.POINTER(_Alignment)]
    lib.sw_alignment_free.argtypes = [ctypes.POINTER(_Alignment)]
    lib.sw_alignment_free.restype = None
    lib.sw_ctx_launches.argtypes = [vp]
    lib.sw_ctx_launches.restype = i64
    lib.sw_ctx_timing.argtypes = [vp, i32]
    lib.sw_ctx_kernel_time.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.sw_db_create.argtypes = [vp, vp, vp, i64, ctypes.POINTER(vp)]
    lib.sw_db_destroy.argtypes = [vp]
    lib.sw_db_destroy.restype = None
    lib.sw_db_size.argtypes = [vp]
    lib.sw_db_size.restype = i64
    lib.sw_batch_create.argtypes = [vp, i64, vp, vp, vp, vp, vp, ctypes.c_int32, vp, ctypes.c_int32,
                                    ctypes.POINTER(vp)]
    lib.sw_batch_run.argtypes = [vp, vp]
    lib.sw_batch_destroy.argtypes = [vp]
    lib.sw_batch_destroy.restype = None
    lib.sw_batch_config.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.sw_batch_bin_config.argtypes = [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64)]
    lib.sw_score_batch.argtypes = [vp, i64, vp, vp, vp, vp, vp, ctypes.c_int32, vp, vp]
    lib.sw_server_create.argtypes = [vp, vp, ctypes.POINTER(_Scoring), ctypes.c_size_t, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(vp)]
    lib.sw_server_submit.argtypes = [vp, vp, i64, ctypes.POINTER(ctypes.c_uint64)]
    lib.sw_server_step.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    lib.sw_server_poll.argtypes = [vp, ctypes.c_uint64, vp, ctypes.POINTER(ctypes.c_int32)]
    lib.sw_server_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t),
                                    ctypes.POINTER(ctypes.c_int64)]
    lib.sw_server_destroy.argtypes = [vp]
    lib.sw_server_destroy.restype = None
    lib.sw_dbsearch.argtypes = [vp, vp, vp, i64, ctypes.POINTER(_Scoring), ctypes.c_int32,
                                ctypes.POINTER(_DbHit), ctypes.POINTER(ctypes.c_int32), vp]
    _lib = lib
    return lib


def _strerror(status: int) -> str:
    try:
        return load().sw_strerror(status).decode()
    except Exception:  # noqa: BLE001 - only for messages
        return "status"


def _check(status: int, what: str):
    if status != SW_OK:
        raise SwError(status, what)


def _seq(x):
    """(pointer, length, keepalive) for a numpy array or a torch tensor of residue codes."""
    if hasattr(x, "data_ptr"):              # torch tensor (host or device)
        assert x.dtype.itemsize == 1 and x.is_contiguous()
        return (x.data_ptr() if x.numel() else None), int(x.numel()), x
    arr = np.ascontiguousarray(np.asarray(x, dtype=np.uint8))
    return (arr.ctypes.data if arr.size else None), int(arr.size), arr


def _scoring(matrix, gap_open: int, gap_extend: int, algorithm: int = ALG_LOCAL):
    mat = np.ascontiguousarray(np.asarray(matrix, dtype=np.int8))
    assert mat.ndim == 2 and mat.shape[0] == mat.shape[1]
    return _Scoring(mat.shape[0], mat.ctypes.data, int(gap_open), int(gap_extend), int(algorithm)), mat


@dataclass(frozen=True)
class Hit:
    score: int
    a_end: int
    b_end: int


@dataclass(frozen=True)
class Alignment:
    score: int
    a_begin: int
    a_end: int
    b_begin: int
    b_end: int
    cigar: str


class Context:
    """One sw_ctx: a device and a CUDA stream (a torch stream handle or None)."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = load()
        h = ctypes.c_void_p()
        handle = None
        if stream is not None:
            handle = getattr(stream, "cuda_stream", stream)
        _check(self._lib.sw_ctx_create(int(device), handle, ctypes.byref(h)), "sw_ctx_create")
        self.handle = h
        self.device = device
        self._children = weakref.WeakSet()

    def _adopt(self, obj):
        """Objects built on this context are closed before it."""
        self._children.add(obj)

    def close(self):
        if self.handle:
            for ch in list(self._children):
                ch.close()
            self._lib.sw_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def launches(self) -> int:
        """Kernels launched by this context so far."""
        return int(self._lib.sw_ctx_launches(self.handle))

    def timing(self, enable: bool = True) -> None:
        """Start (or stop) per-kernel device timing; clears the totals."""
        _check(self._lib.sw_ctx_timing(self.handle, 1 if enable else 0), "sw_ctx_timing")

    def kernel_time(self, kind: int):
        """(total device ms, launches) of one kernel kind (KT_*) since timing() was enabled."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(self._lib.sw_ctx_kernel_time(self.handle, kind, ctypes.byref(ms), ctypes.byref(n)),
               "sw_ctx_kernel_time")
        return ms.value, n.value

    def encode(self, alphabet: str, text) -> np.ndarray:
        raw = text.encode("ascii") if isinstance(text, str) else bytes(text)
        buf = np.frombuffer(raw, dtype=np.uint8).copy()
        out = np.zeros(len(raw), dtype=np.uint8)
        _check(self._lib.sw_encode(self.handle, alphabet.encode("ascii"),
                                   buf.ctypes.data if buf.size else None, len(raw),
                                   out.ctypes.data if out.size else None), "sw_encode")
        return out

    def score(self, a, b, matrix, gap_open: int, gap_extend: int, algorithm: int = ALG_LOCAL) -> Hit:
        pa, m, ka = _seq(a)
        pb, n, kb = _seq(b)
        sc, keep = _scoring(matrix, gap_open, gap_extend, algorithm)
        hit = _Hit()
        _check(self._lib.sw_score(self.handle, pa, m, pb, n, ctypes.byref(sc), ctypes.byref(hit)),
               "sw_score")
        return Hit(hit.score, hit.a_end, hit.b_end)

    def align(self, a, b, matrix, gap_open: int, gap_extend: int, algorithm: int = ALG_LOCAL) -> Alignment:
        pa, m, ka = _seq(a)
        pb, n, kb = _seq(b)
        sc, keep = _scoring(matrix, gap_open, gap_extend, algorithm)
        aln = _Alignment()
        _check(self._lib.sw_align(self.handle, pa, m, pb, n, ctypes.byref(sc), ctypes.byref(aln)),
               "sw_align")
        try:
            cig = ctypes.string_at(aln.cigar, aln.cigar_len).decode() if aln.cigar else ""
        finally:
            self._lib.sw_alignment_free(ctypes.byref(aln))
        return Alignment(aln.score, aln.a_begin, aln.a_end, aln.b_begin, aln.b_end, cig)


SW_BATCH_GRAPH, SW_BATCH_AUTOTUNE = 1, 2
KT_FILL, KT_FILL_TB, KT_WALK, KT_DB16 = 0, 1, 2, 3     # kernel kinds of Context.kernel_time


def _pack_pairs(pairs):
    """Concatenated residues and offsets of the a and b sides of (a, b, scoring) pairs."""
    def cat(seqs):
        seqs = [np.ascontiguousarray(np.asarray(x, dtype=np.uint8)) for x in seqs]
        off = np.zeros(len(seqs) + 1, dtype=np.int64)
        np.cumsum([len(x) for x in seqs], out=off[1:])
        res = np.concatenate(seqs) if len(seqs) and off[-1] > 0 else np.zeros(1, np.uint8)
        return res, off
    ares, aoff = cat([p[0] for p in pairs])
    bres, boff = cat([p[1] for p in pairs])
    sidx = np.ascontiguousarray(np.array([p[2] for p in pairs], dtype=np.int32))
    return ares, aoff, bres, boff, sidx


def _scoring_array(scorings):
    arr = (_Scoring * len(scorings))()
    keep = []
    for i, s in enumerate(scorings):           # (matrix, open, extend[, algorithm])
        sc, k = _scoring(*s)
        arr[i] = sc
        keep.append(k)
    return arr, keep


class Batch:
    """A batch plan (sw_batch): pairs = [(a, b, scoring_index)], scorings = [(matrix, open, extend)].
    a/b residues may be given as device tensors through `device_inputs` = (a_res, b_res) tensors
    holding the concatenations."""

    def __init__(self, ctx: Context, pairs, scorings, flags: int = 0, device_inputs=None):
        self._lib = load()
        self.ctx = ctx
        self.npairs = len(pairs)
        ares, aoff, bres, boff, sidx = _pack_pairs(pairs)
        self._keep = [ares, aoff, bres, boff, sidx]
        pa, pb = ares.ctypes.data, bres.ctypes.data
        if device_inputs is not None:
            pa, pb = device_inputs[0].data_ptr(), device_inputs[1].data_ptr()
            self._keep.append(device_inputs)
        arr, keep = _scoring_array(scorings)
        self._keep += [arr, keep]
        h = ctypes.c_void_p()
        _check(self._lib.sw_batch_create(ctx.handle, self.npairs, pa, aoff.ctypes.data, pb, boff.ctypes.data,
                                         sidx.ctypes.data, len(scorings), arr, int(flags), ctypes.byref(h)),
               "sw_batch_create")
        self.handle = h
        self._out = (_Hit * max(1, self.npairs))()
        ctx._adopt(self)

    @staticmethod
    def packed(pairs):
        return _pack_pairs(pairs)

    def config(self):
        r, w = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.sw_batch_config(self.handle, ctypes.byref(r), ctypes.byref(w)), "sw_batch_config")
        return r.value, w.value

    def bins(self):
        """Per bin: (rows per lane, warps, lane bits, pairs), largest bin first."""
        out = []
        while True:
            r, w, lb, npr = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
            rc = self._lib.sw_batch_bin_config(self.handle, len(out), ctypes.byref(r), ctypes.byref(w),
                                               ctypes.byref(lb), ctypes.byref(npr))
            if rc == SW_ERANGE:
                return out
            _check(rc, "sw_batch_bin_config")
            out.append((r.value, w.value, lb.value, npr.value))

    def run(self):
        _check(self._lib.sw_batch_run(self.handle, self._out), "sw_batch_run")
        return [Hit(h.score, h.a_end, h.b_end) for h in self._out[:self.npairs]]

    def close(self):
        if self.handle:
            self._lib.sw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


class Database:
    """A device-resident database (sw_db) built from residues + offsets."""

    def __init__(self, ctx: Context, residues, offsets):
        self._lib = load()
        self.ctx = ctx
        res = np.ascontiguousarray(np.asarray(residues, dtype=np.uint8))
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        h = ctypes.c_void_p()
        _check(self._lib.sw_db_create(ctx.handle, res.ctypes.data if res.size else None,
                                      off.ctypes.data, len(off) - 1, ctypes.byref(h)), "sw_db_create")
        self.handle = h
        self.nseq = len(off) - 1
        self._children = weakref.WeakSet()
        ctx._adopt(self)

    def _adopt(self, obj):
        self._children.add(obj)

    def close(self):
        if self.handle:
            for ch in list(self._children):
                ch.close()
            self._lib.sw_db_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def search(self, q, matrix, gap_open: int, gap_extend: int, k: int = 20, all_scores: bool = False,
               scores_out=None):
        """(hits, scores): hits = [(subject, score)] best first; scores = int32 array or None.
        scores_out may be a preallocated int32 numpy array or torch CUDA tensor."""
        pq, m, kq = _seq(q)
        sc, keep = _scoring(matrix, gap_open, gap_extend)
        hits = (_DbHit * max(1, k))()
        nh = ctypes.c_int32()
        out = scores_out
        if out is None and all_scores:
            out = np.zeros(self.nseq, dtype=np.int32)
        ptr = None
        if out is not None:
            ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        _check(self._lib.sw_dbsearch(self.ctx.handle, self.handle, pq, m, ctypes.byref(sc), int(k),
                                     hits, ctypes.byref(nh), ptr), "sw_dbsearch")
        return [(int(hits[i].subject), int(hits[i].score)) for i in range(nh.value)], out


class Server:
    """Continuous-batching search server over a Database (sw_server)."""

    def __init__(self, ctx: Context, db: Database, matrix, gap_open: int, gap_extend: int,
                 mem_budget: int, k: int = 20, max_slots: int = 32, chunks: int = 16):
        self._lib = load()
        self.ctx, self.db, self.k = ctx, db, k
        self._sc, self._keep = _scoring(matrix, gap_open, gap_extend)
        h = ctypes.c_void_p()
        _check(self._lib.sw_server_create(ctx.handle, db.handle, ctypes.byref(self._sc), int(mem_budget), int(k),
                                          int(max_slots), int(chunks), ctypes.byref(h)), "sw_server_create")
        self.handle = h
        self._hits = (_DbHit * max(1, k))()
        ctx._adopt(self)
        db._adopt(self)

    def submit(self, q):
        """Ticket of the admitted request, or None when no slot / memory is free."""
        pq, m, keep = _seq(q)
        t = ctypes.c_uint64()
        rc = self._lib.sw_server_submit(self.handle, pq, m, ctypes.byref(t))
        if rc == SW_EAGAIN:
            return None
        _check(rc, "sw_server_submit")
        return int(t.value)

    def step(self) -> int:
        a = ctypes.c_int32()
        _check(self._lib.sw_server_step(self.handle, ctypes.byref(a)), "sw_server_step")
        return a.value

    def poll(self, ticket: int):
        """[(subject, score)] when finished, None while pending."""
        n = ctypes.c_int32()
        rc = self._lib.sw_server_poll(self.handle, ctypes.c_uint64(ticket), self._hits, ctypes.byref(n))
        if rc == SW_EAGAIN:
            return None
        _check(rc, "sw_server_poll")
        return [(int(self._hits[i].subject), int(self._hits[i].score)) for i in range(n.value)]

    def stats(self):
        a, mu, cells = ctypes.c_int32(), ctypes.c_size_t(), ctypes.c_int64()
        _check(self._lib.sw_server_stats(self.handle, ctypes.byref(a), ctypes.byref(mu), ctypes.byref(cells)),
               "sw_server_stats")
        return a.value, mu.value, cells.value

    def close(self):
        if self.handle:
            self._lib.sw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


PROBE_OPS = {"iadd": 0, "imax": 1, "viaddmax_s32": 2, "vimax3_s32_relu": 3,
             "viaddmax_s16x2": 4, "vimax3_s16x2_relu": 5, "prmt": 6, "shfl": 7,
             "vaddus4": 8, "vsubus4": 9, "vmaxu4": 10}


def probe_int_rates(ctx: Context, iters: int = 2000) -> dict:
    """Measured thread-level results per SM per clock of each instruction form
    (sw_probe_int_rate), plus the SM clock seen while they ran."""
    lib = load()
    fn = lib.sw_probe_int_rate
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    out = {}
    mhz = []
    for name, op in PROBE_OPS.items():
        r, f = ctypes.c_double(), ctypes.c_double()
        _check(fn(ctx.handle, op, iters, ctypes.byref(r), ctypes.byref(f)), "sw_probe_int_rate")
        out[name] = round(r.value, 2)
        mhz.append(f.value)
    out["sm_mhz"] = round(sum(mhz) / len(mhz), 1)
    return out


def probe_latencies(ctx: Context, iters: int = 2000) -> dict:
    """SM clocks from one instruction of each form to the next that needs its
    result (sw_probe_latency: one warp, one dependent chain)."""
    lib = load()
    fn = lib.sw_probe_latency
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    out = {}
    for name, op in PROBE_OPS.items():
        r = ctypes.c_double()
        _check(fn(ctx.handle, op, iters, ctypes.byref(r)), "sw_probe_latency")
        out[name] = round(r.value, 2)
    return out
