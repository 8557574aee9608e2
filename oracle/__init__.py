"""Python face of the plain C oracle (oracle.c, search.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg; the product path never imports it.

`align(...)` runs one pair; `align_batch(...)` runs many on a thread pool;
`search(...)` / `search_batch(...)` give the edit distance by the search
traversal.  All return plain dicts / numpy arrays.  The library is compiled with gcc on first
use (or by `build()`), next to this file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_SEARCH = os.path.join(_HERE, "search.c")
_SRC_FOLD = os.path.join(_HERE, "fold.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF = np.iinfo(np.int64).max
OP_CHARS = {1: "I", 2: "D", 7: "=", 8: "X"}
STATUS = {0: "OK", 1: "DROPPED", 2: "UNREACHABLE", 3: "EMPTY"}


class Params(C.Structure):
    _fields_ = [
        ("mode", C.c_int32), ("affine", C.c_int32), ("gap_open", C.c_int64),
        ("gap_extend", C.c_int64), ("alphabet", C.c_int32), ("subst", C.POINTER(C.c_int8)),
        ("use_band", C.c_int32), ("band_literal", C.c_int32), ("band", C.c_int64),
        ("use_xdrop", C.c_int32), ("xdrop", C.c_int64), ("traceback", C.c_int32),
        ("order", C.c_int32), ("zdrop", C.c_int32), ("running", C.c_int32),
        ("mid", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("score", C.c_int64), ("q_begin", C.c_int64), ("q_end", C.c_int64),
        ("r_begin", C.c_int64), ("r_end", C.c_int64), ("status", C.c_int32),
        ("cells", C.c_int64), ("n_ops", C.c_int64), ("last_k", C.c_int64),
    ]


class SearchParams(C.Structure):
    _fields_ = [("traceback", C.c_int32), ("use_band", C.c_int32), ("band", C.c_int64),
                ("adapt_min_len", C.c_int64), ("adapt_max_dist", C.c_int64)]


class SearchResult(C.Structure):
    _fields_ = [("distance", C.c_int64), ("cells", C.c_int64), ("n_ops", C.c_int64)]


SEARCH_RESULT_DTYPE = np.dtype([("distance", np.int64), ("cells", np.int64), ("n_ops", np.int64)])
assert SEARCH_RESULT_DTYPE.itemsize == C.sizeof(SearchResult)


class FoldParams(C.Structure):
    _fields_ = [("min_loop", C.c_int64), ("use_xdrop", C.c_int32), ("xdrop", C.c_int64),
                ("warmup", C.c_int64), ("traceback", C.c_int32)]


class FoldResult(C.Structure):
    _fields_ = [("score", C.c_int64), ("i_end", C.c_int64), ("j_end", C.c_int64),
                ("status", C.c_int32), ("cells", C.c_int64), ("last_k", C.c_int64)]


FOLD_RESULT_DTYPE = np.dtype([("score", np.int64), ("i_end", np.int64), ("j_end", np.int64),
                              ("status", np.int32), ("pad", np.int32), ("cells", np.int64),
                              ("last_k", np.int64)])
assert FOLD_RESULT_DTYPE.itemsize == C.sizeof(FoldResult)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no CUDA)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_SRC_SEARCH), os.path.getmtime(_SRC_FOLD),
            os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC,
                                   _SRC_SEARCH, _SRC_FOLD, "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_align.restype = C.c_int
        L.orc_align.argtypes = [C.POINTER(Params), C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                C.POINTER(Result), C.c_void_p, C.c_int64]
        L.orc_align_batch.restype = C.c_int
        L.orc_align_batch.argtypes = [C.POINTER(Params), C.c_int64] + [C.c_void_p] * 6 + [
            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orc_domain.restype = C.c_int64
        L.orc_domain.argtypes = [C.POINTER(Params), C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                 C.c_void_p, C.c_void_p, C.c_int64]
        L.orc_search.restype = C.c_int
        L.orc_search.argtypes = [C.POINTER(SearchParams), C.c_void_p, C.c_int64, C.c_void_p,
                                 C.c_int64, C.POINTER(SearchResult), C.c_void_p, C.c_int64]
        L.orc_search_batch.restype = C.c_int
        L.orc_search_batch.argtypes = [C.POINTER(SearchParams), C.c_int64] + [C.c_void_p] * 6 + [
            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.orc_fold.restype = C.c_int
        L.orc_fold.argtypes = [C.POINTER(FoldParams), C.c_void_p, C.c_int64, C.POINTER(FoldResult),
                               C.c_void_p]
        L.orc_fold_batch.restype = C.c_int
        L.orc_fold_batch.argtypes = [C.POINTER(FoldParams), C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        _lib = L
    return _lib


def make_params(subst, mode="global", affine=True, gap_open=0, gap_extend=1, band=None,
                band_literal=False, xdrop=None, zdrop=None, traceback=True, order=0,
                xdrop_running=False, mid=False, **_ignored):
    s = np.ascontiguousarray(np.asarray(subst, dtype=np.int8))
    a = int(s.shape[0])
    p = Params()
    p.mode = 1 if mode in ("local", 1) else 0
    p.affine = 1 if affine else 0
    p.gap_open = int(gap_open)
    p.gap_extend = int(gap_extend)
    p.alphabet = a
    p.subst = s.ctypes.data_as(C.POINTER(C.c_int8))
    p.use_band = 0 if band is None else 1
    p.band_literal = 1 if band_literal else 0
    p.band = 0 if band is None else int(band)
    if xdrop is not None and zdrop is not None:
        raise ValueError("xdrop and zdrop are exclusive")
    thr = xdrop if zdrop is None else zdrop
    p.use_xdrop = 0 if thr is None else 1
    p.xdrop = 0 if thr is None else (INF if thr == INF else int(thr))
    p.zdrop = 0 if zdrop is None else 1
    p.traceback = 1 if traceback else 0
    p.order = int(order)
    p.running = 1 if xdrop_running else 0
    p.mid = 1 if mid else 0
    p._keep = s  # keep the table alive
    return p


def _res_dict(r: Result, ops=None):
    d = dict(score=r.score, q_begin=r.q_begin, q_end=r.q_end, r_begin=r.r_begin,
             r_end=r.r_end, status=r.status, cells=r.cells, n_ops=r.n_ops, last_k=r.last_k)
    if ops is not None:
        d["cigar"] = ops
    return d


def align(q, r, subst, **kw) -> dict:
    """Align one pair; returns score, coordinates, status, cells and the CIGAR
    (numpy uint32 BAM ops) when traceback is on."""
    p = make_params(subst, **kw)
    q = np.ascontiguousarray(np.asarray(q, dtype=np.uint8))
    r = np.ascontiguousarray(np.asarray(r, dtype=np.uint8))
    res = Result()
    cap = int(q.shape[0] + r.shape[0] + 1)
    ops = np.zeros(cap, dtype=np.uint32)
    rc = lib().orc_align(C.byref(p), q.ctypes.data, q.shape[0], r.ctypes.data, r.shape[0],
                         C.byref(res), ops.ctypes.data, cap)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return _res_dict(res, ops[: res.n_ops].copy() if p.traceback else None)


RESULT_DTYPE = np.dtype([("score", np.int64), ("q_begin", np.int64), ("q_end", np.int64),
                         ("r_begin", np.int64), ("r_end", np.int64), ("status", np.int32),
                         ("pad", np.int32), ("cells", np.int64), ("n_ops", np.int64),
                         ("last_k", np.int64)])
assert RESULT_DTYPE.itemsize == C.sizeof(Result)


def align_batch(batch, nthreads: int | None = None, **kw):
    """Align every pair of a synth.Batch (or anything with the same fields).

    Returns (results, ops, ops_off): a structured array with one row per pair,
    the concatenated CIGAR ops and where each pair's ops start."""
    sc = dict(batch.scoring)
    sc.update(kw)
    p = make_params(batch.subst, **sc)
    n = int(batch.q_len.shape[0])
    res = np.zeros(n, dtype=RESULT_DTYPE)
    cap = (batch.q_len.astype(np.uint64) + batch.r_len.astype(np.uint64) + 1)
    off = np.zeros(n, dtype=np.uint64)
    if n:
        off[1:] = np.cumsum(cap[:-1])
    ops = np.zeros(int(cap.sum()) if (p.traceback and n) else 1, dtype=np.uint32)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    q = np.ascontiguousarray(batch.q_seq)
    r = np.ascontiguousarray(batch.r_seq)
    qo = np.ascontiguousarray(batch.q_off, dtype=np.uint64)
    ro = np.ascontiguousarray(batch.r_off, dtype=np.uint64)
    ql = np.ascontiguousarray(batch.q_len, dtype=np.uint32)
    rl = np.ascontiguousarray(batch.r_len, dtype=np.uint32)
    rc = lib().orc_align_batch(C.byref(p), n, q.ctypes.data, qo.ctypes.data, ql.ctypes.data,
                               r.ctypes.data, ro.ctypes.data, rl.ctypes.data, res.ctypes.data,
                               ops.ctypes.data if p.traceback else None,
                               off.ctypes.data, cap.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return res, ops, off


def domain(q, r, subst, **kw):
    """Every cell the run evaluated, as an (n, 2) int64 array of (i, j), and an
    alive (unpruned) flag per cell."""
    p = make_params(subst, **kw)
    q = np.ascontiguousarray(np.asarray(q, dtype=np.uint8))
    r = np.ascontiguousarray(np.asarray(r, dtype=np.uint8))
    n = lib().orc_domain(C.byref(p), q.ctypes.data, q.shape[0], r.ctypes.data, r.shape[0],
                         None, None, 0)
    ij = np.zeros((max(n, 1), 2), dtype=np.int64)
    alive = np.zeros(max(n, 1), dtype=np.uint8)
    lib().orc_domain(C.byref(p), q.ctypes.data, q.shape[0], r.ctypes.data, r.shape[0],
                     ij.ctypes.data, alive.ctypes.data, n)
    return ij[:n], alive[:n].astype(bool)


def cigar_str(ops) -> str:
    return "".join(f"{int(o) >> 4}{OP_CHARS[int(o) & 15]}" for o in ops)


def make_search_params(traceback=True, band=None, adapt=None):
    """adapt = (min_len, max_dist) turns WFA-Adapt on."""
    p = SearchParams()
    p.traceback = 1 if traceback else 0
    p.use_band = 0 if band is None else 1
    p.band = 0 if band is None else int(band)
    p.adapt_min_len, p.adapt_max_dist = (0, 0) if adapt is None else (int(adapt[0]),
                                                                      int(adapt[1]))
    return p


def search(q, r, traceback=True, band=None, adapt=None) -> dict:
    """Edit distance of one pair by the search traversal (Sec. 6.3): distance,
    wavefront cells evaluated, and the CIGAR when traceback is on."""
    p = make_search_params(traceback, band, adapt)
    q = np.ascontiguousarray(np.asarray(q, dtype=np.uint8))
    r = np.ascontiguousarray(np.asarray(r, dtype=np.uint8))
    res = SearchResult()
    cap = int(q.shape[0] + r.shape[0] + 1)
    ops = np.zeros(cap, dtype=np.uint32)
    rc = lib().orc_search(C.byref(p), q.ctypes.data, q.shape[0], r.ctypes.data, r.shape[0],
                          C.byref(res), ops.ctypes.data, cap)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    d = dict(distance=res.distance, cells=res.cells, n_ops=res.n_ops)
    if traceback:
        d["cigar"] = ops[: res.n_ops].copy()
    return d


def search_batch(batch, nthreads: int | None = None, traceback=True, band=None, adapt=None):
    """search() over every pair of a synth.Batch on a thread pool.  Returns
    (results, ops, ops_off) like align_batch."""
    p = make_search_params(traceback, band, adapt)
    n = int(batch.q_len.shape[0])
    res = np.zeros(n, dtype=SEARCH_RESULT_DTYPE)
    cap = (batch.q_len.astype(np.uint64) + batch.r_len.astype(np.uint64) + 1)
    off = np.zeros(n, dtype=np.uint64)
    if n:
        off[1:] = np.cumsum(cap[:-1])
    ops = np.zeros(int(cap.sum()) if (traceback and n) else 1, dtype=np.uint32)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    q = np.ascontiguousarray(batch.q_seq)
    r = np.ascontiguousarray(batch.r_seq)
    qo = np.ascontiguousarray(batch.q_off, dtype=np.uint64)
    ro = np.ascontiguousarray(batch.r_off, dtype=np.uint64)
    ql = np.ascontiguousarray(batch.q_len, dtype=np.uint32)
    rl = np.ascontiguousarray(batch.r_len, dtype=np.uint32)
    rc = lib().orc_search_batch(C.byref(p), n, q.ctypes.data, qo.ctypes.data, ql.ctypes.data,
                                r.ctypes.data, ro.ctypes.data, rl.ctypes.data, res.ctypes.data,
                                ops.ctypes.data if traceback else None, off.ctypes.data,
                                cap.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return res, ops, off


def make_fold_params(min_loop=3, xdrop=None, warmup=15, traceback=True):
    p = FoldParams()
    p.min_loop = int(min_loop)
    p.use_xdrop = 0 if xdrop is None else 1
    p.xdrop = 0 if xdrop is None else int(xdrop)
    p.warmup = int(warmup)
    p.traceback = 1 if traceback else 0
    return p


def fold(x, min_loop=3, xdrop=None, warmup=15, traceback=True) -> dict:
    """Nussinov fold of one RNA (codes A=0 C=1 G=2 U=3), optionally under the
    X-drop transfer of Sec. 9.5: score, status, end cell, cells and the partner
    of every base (-1 unpaired)."""
    p = make_fold_params(min_loop, xdrop, warmup, traceback)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint8))
    res = FoldResult()
    partner = np.full(max(x.shape[0], 1), -1, dtype=np.int32)
    rc = lib().orc_fold(C.byref(p), x.ctypes.data, x.shape[0], C.byref(res), partner.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dict(score=res.score, i_end=res.i_end, j_end=res.j_end, status=res.status,
                cells=res.cells, last_k=res.last_k, partner=partner[: x.shape[0]].copy())


def fold_batch(seq, off, lens, nthreads: int | None = None, **kw):
    """fold() over concatenated sequences; returns (results, partners)."""
    p = make_fold_params(**kw)
    n = int(len(lens))
    res = np.zeros(n, dtype=FOLD_RESULT_DTYPE)
    seq = np.ascontiguousarray(seq, dtype=np.uint8)
    off = np.ascontiguousarray(off, dtype=np.uint64)
    lens = np.ascontiguousarray(lens, dtype=np.uint32)
    partner = np.full(max(int(seq.shape[0]), 1), -1, dtype=np.int32)
    rc = lib().orc_fold_batch(C.byref(p), n, seq.ctypes.data, off.ctypes.data, lens.ctypes.data,
                              res.ctypes.data, partner.ctypes.data,
                              int(nthreads or os.cpu_count() or 1))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return res, partner
