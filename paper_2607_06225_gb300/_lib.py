"""ctypes binding of libfiltr.so: the C-ABI names, argument marshalling only.

Every computation happens in the library's CUDA kernels; nothing here falls
back to the CPU.  If the library has not been built this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfiltr.so")

OK = 0
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_BUSY, ERR_CIGAR_CAP, ERR_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7)
GLOBAL, LOCAL = 0, 1
ALPHA_DNA, ALPHA_PROTEIN = 4, 20
PRUNE_BAND, PRUNE_XDROP, PRUNE_BAND_LITERAL, PRUNE_ZDROP, PRUNE_XDROP_RUNNING = 1, 2, 4, 8, 16
AFFINE_MID = 2  # FILTR_AFFINE_MID: Table 1's M/I/D form
PREC_AUTO, PREC_I32, PREC_I16X2 = 0, 1, 2
XDROP_INF = 0x7FFFFFFF
ST_OK, ST_DROPPED, ST_UNREACHABLE, ST_EMPTY, ST_TOO_WIDE = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "OK", -1: "ERR_INVALID", -2: "ERR_NOMEM", -3: "ERR_CUDA", -4: "ERR_TIMEOUT",
                -5: "ERR_BUSY", -6: "ERR_CIGAR_CAP", -7: "ERR_UNSUPPORTED"}


class FiltrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("mode", C.c_int32), ("alphabet", C.c_int32), ("affine", C.c_int32),
                ("gap_open", C.c_int32), ("gap_extend", C.c_int32),
                ("subst", C.POINTER(C.c_int8)), ("prune", C.c_uint32), ("band", C.c_int32),
                ("xdrop", C.c_int32), ("traceback", C.c_int32), ("precision", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("score", C.c_int32), ("q_begin", C.c_int32), ("q_end", C.c_int32),
                ("r_begin", C.c_int32), ("r_end", C.c_int32), ("status", C.c_int32),
                ("cigar_len", C.c_uint32), ("reserved", C.c_uint32), ("cigar_off", C.c_uint64),
                ("cells", C.c_uint64)]


class SearchParams(C.Structure):
    _fields_ = [("traceback", C.c_int32), ("band", C.c_int32), ("adapt_min_len", C.c_int32),
                ("adapt_max_dist", C.c_int32), ("alphabet", C.c_int32)]


def make_search_params(traceback=True, band=None, adapt=None, alphabet=0) -> SearchParams:
    """filtr_search_params: band=None for none; adapt=(min_len, max_dist) turns
    WFA-Adapt on; alphabet=4 for DNA codes 0..3 (held two bits each)."""
    p = SearchParams()
    p.alphabet = int(alphabet)
    p.traceback = 1 if traceback else 0
    p.band = -1 if band is None else int(band)
    p.adapt_min_len, p.adapt_max_dist = (0, 0) if adapt is None else (int(adapt[0]),
                                                                      int(adapt[1]))
    return p


class FoldParams(C.Structure):
    _fields_ = [("min_loop", C.c_int32), ("use_xdrop", C.c_int32), ("xdrop", C.c_int32),
                ("warmup", C.c_int32), ("traceback", C.c_int32)]


FOLD_RESULT_DTYPE = np.dtype([("score", np.int32), ("i_end", np.int32), ("j_end", np.int32),
                              ("status", np.int32), ("cells", np.uint64)])


def make_fold_params(min_loop=3, xdrop=None, warmup=15, traceback=True) -> FoldParams:
    """filtr_fold_params: xdrop=None folds unpruned."""
    p = FoldParams()
    p.min_loop = int(min_loop)
    p.use_xdrop = 0 if xdrop is None else 1
    p.xdrop = 0 if xdrop is None else int(xdrop)
    p.warmup = int(warmup)
    p.traceback = 1 if traceback else 0
    return p


class Stats(C.Structure):
    _fields_ = [("ms_validate", C.c_double), ("ms_forward", C.c_double), ("ms_walk", C.c_double),
                ("ms_place", C.c_double), ("ms_total", C.c_double), ("launches", C.c_uint32),
                ("waves", C.c_uint32), ("cells_planned", C.c_uint64),
                ("pairs_i16x2", C.c_uint32), ("device_plan", C.c_uint32),
                ("ms_host_wait", C.c_double), ("ms_host_plan", C.c_double),
                ("cells_i16x2", C.c_uint64), ("pairs_xd16", C.c_uint32),
                ("pairs_xd16_rerun", C.c_uint32)]


# the eight tiled shapes in the order filtr_autotune reports them
TUNE_SHAPES = [("i32", 32), ("i32", 24), ("i32", 16), ("i32", 8)] + [
    ("i16x2", R) for R in range(32, 7, -2)]
TUNE_MAX_SHAPES = 24
# the antidiagonal sweep's candidates (X-drop / Z-drop parameters), in report order
TUNE_SWEEP = [("i16x2", 1), ("i32", 1), ("i16x2", 2), ("i32", 2)]


class TuneReport(C.Structure):
    _fields_ = [("n_shapes", C.c_int32), ("rows_per_lane", C.c_int32 * TUNE_MAX_SHAPES),
                ("packed", C.c_int32 * TUNE_MAX_SHAPES),
                ("ns_per_warp_step", C.c_double * TUNE_MAX_SHAPES)]


RESULT_DTYPE = np.dtype([("score", np.int32), ("q_begin", np.int32), ("q_end", np.int32),
                         ("r_begin", np.int32), ("r_end", np.int32), ("status", np.int32),
                         ("cigar_len", np.uint32), ("reserved", np.uint32),
                         ("cigar_off", np.uint64), ("cells", np.uint64)])
assert RESULT_DTYPE.itemsize == C.sizeof(Result) == 48

_lib = None
_P = C.c_void_p
_U8P = C.c_void_p


def lib():
    """Load libfiltr.so (built by paper_2607_06225_gb300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfiltr.so is not built; run paper_2607_06225_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        i32 = C.c_int
        L.filtr_last_error.restype = C.c_char_p
        L.filtr_version.restype = C.c_char_p
        L.filtr_params_check.restype = i32
        L.filtr_params_check.argtypes = [C.POINTER(Params)]
        L.filtr_ctx_create.restype = i32
        L.filtr_ctx_create.argtypes = [i32, C.c_size_t, C.POINTER(C.c_void_p)]
        L.filtr_ctx_destroy.restype = i32
        L.filtr_ctx_destroy.argtypes = [C.c_void_p]
        L.filtr_pack.restype = i32
        L.filtr_pack.argtypes = [_P, C.c_uint64, C.c_int32, _P, _P, _P]
        batch_args = [C.c_void_p, C.POINTER(Params), C.c_uint32, _P, _P, _P, _P, _P, _P, _P, _P,
                      C.c_uint64]
        L.filtr_fold_batch.restype = i32
        L.filtr_fold_batch.argtypes = [C.c_void_p, C.POINTER(FoldParams), C.c_uint32, _P, _P, _P,
                                       _P, _P, C.c_void_p]
        L.filtr_search_batch.restype = i32
        L.filtr_search_batch.argtypes = [C.c_void_p, C.POINTER(SearchParams), C.c_uint32, _P, _P,
                                         _P, _P, _P, _P, _P, _P, C.c_uint64, C.c_void_p]
        for name in ("filtr_align_batch", "filtr_align_batch_plain"):
            f = getattr(L, name)
            f.restype = i32
            f.argtypes = batch_args + [_P]
        L.filtr_align_batch_noalloc.restype = i32
        L.filtr_align_batch_noalloc.argtypes = [C.POINTER(Params), C.c_uint32, _P, _P, _P, _P, _P,
                                                _P, C.c_uint32, C.c_uint32, _P, _P]
        L.filtr_align_batch_host.restype = i32
        L.filtr_align_batch_host.argtypes = batch_args
        L.filtr_align_long.restype = i32
        L.filtr_align_long.argtypes = [C.c_void_p, C.POINTER(Params), _P, C.c_uint32, _P,
                                       C.c_uint32, _P, _P, C.c_uint64, _P]
        L.filtr_ctx_set_timing.restype = i32
        L.filtr_ctx_set_timing.argtypes = [C.c_void_p, i32]
        L.filtr_ctx_last_stats.restype = i32
        L.filtr_ctx_last_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.filtr_autotune.restype = i32
        L.filtr_autotune.argtypes = [C.c_void_p, C.POINTER(Params), C.POINTER(TuneReport)]
        L.filtr_tune_apply.restype = i32
        L.filtr_tune_apply.argtypes = [C.c_void_p, C.POINTER(Params), C.POINTER(TuneReport)]
        L.filtr_probe_int_peak.restype = i32
        L.filtr_probe_int_peak.argtypes = [C.c_void_p, C.POINTER(C.c_double * 5)]
        L.filtr_test_long_timeout.restype = i32
        L.filtr_test_long_timeout.argtypes = [C.c_void_p, C.POINTER(Params), _P, C.c_uint32, _P,
                                              C.c_uint32, C.c_uint64]
        L.filtr_test_set_checkpoint.restype = i32
        L.filtr_test_set_checkpoint.argtypes = [C.c_void_p, C.c_int32]
        L.filtr_test_force_recompute.restype = i32
        L.filtr_test_force_recompute.argtypes = [C.c_void_p, C.c_int32]
        L.filtr_test_set_first_width.restype = i32
        L.filtr_test_set_first_width.argtypes = [C.c_void_p, C.c_int32]
        L.filtr_test_set_device_plan.restype = i32
        L.filtr_test_set_device_plan.argtypes = [C.c_void_p, C.c_int32]
        L.filtr_test_set_search_ring.restype = i32
        L.filtr_test_set_search_ring.argtypes = [C.c_void_p, C.c_int32]
        L.filtr_test_set_packed_sweep.restype = i32
        L.filtr_test_set_packed_sweep.argtypes = [C.c_void_p, C.c_int32]
        L.filtr_test_plan_host.restype = i32
        L.filtr_test_plan_host.argtypes = [C.POINTER(Params), C.c_uint32, _P, _P, C.c_uint64, _P, _P,
                                           _P, _P, _P, _P, _P]
        L.filtr_graph_create.restype = i32
        L.filtr_graph_create.argtypes = [C.c_void_p, C.POINTER(Params), C.c_uint32, C.c_uint32,
                                         C.c_size_t, C.POINTER(C.c_void_p)]
        L.filtr_graph_launch.restype = i32
        L.filtr_graph_launch.argtypes = [C.c_void_p, C.c_uint32, _P, _P, _P, _P, _P, _P, _P, _P,
                                         C.c_uint64, _P]
        L.filtr_graph_status.restype = i32
        L.filtr_graph_status.argtypes = [C.c_void_p]
        L.filtr_graph_destroy.restype = i32
        L.filtr_graph_destroy.argtypes = [C.c_void_p]
        L.filtr_serve_create.restype = i32
        L.filtr_serve_create.argtypes = [C.c_void_p, C.c_size_t, C.c_uint32, C.POINTER(C.c_void_p)]
        L.filtr_serve_submit.restype = i32
        L.filtr_serve_submit.argtypes = [C.c_void_p, C.POINTER(Params), _P, C.c_uint32, _P,
                                         C.c_uint32, C.POINTER(C.c_uint64)]
        L.filtr_serve_poll.restype = i32
        L.filtr_serve_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(Result), _P, C.c_uint64, _P]
        L.filtr_serve_wait.restype = i32
        L.filtr_serve_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_int64, C.POINTER(Result), _P,
                                       C.c_uint64, _P]
        L.filtr_serve_destroy.restype = i32
        L.filtr_serve_destroy.argtypes = [C.c_void_p]
        _lib = L
    return _lib


def last_error() -> str:
    return lib().filtr_last_error().decode()


def check(rc: int, what: str = ""):
    if rc != OK:
        raise FiltrError(rc, f"{what}: {last_error()}" if what else last_error())
    return rc


def make_params(subst, mode="global", affine=True, gap_open=0, gap_extend=1, band=None,
                band_literal=False, xdrop=None, zdrop=None, traceback=False, precision=PREC_AUTO,
                xdrop_running=False, mid=False, **_ignored) -> Params:
    """Build a filtr_params block; the substitution table is kept alive on it."""
    s = np.ascontiguousarray(np.asarray(subst, dtype=np.int8))
    p = Params()
    p.mode = LOCAL if mode in ("local", LOCAL) else GLOBAL
    p.alphabet = int(s.shape[0])
    p.affine = (AFFINE_MID if mid else 1) if affine else 0
    p.gap_open = int(gap_open)
    p.gap_extend = int(gap_extend)
    p.subst = s.ctypes.data_as(C.POINTER(C.c_int8))
    prune = 0
    if band is not None:
        prune |= PRUNE_BAND_LITERAL if band_literal else PRUNE_BAND
    if xdrop is not None and zdrop is not None:
        raise ValueError("xdrop and zdrop exclude each other")
    if xdrop is not None:
        prune |= PRUNE_XDROP
    if zdrop is not None:
        prune |= PRUNE_ZDROP
    if xdrop_running:
        prune |= PRUNE_XDROP_RUNNING
    thr = xdrop if zdrop is None else zdrop
    p.prune = prune
    p.band = 0 if band is None else int(band)
    p.xdrop = 0 if thr is None else int(min(int(thr), XDROP_INF))
    p.traceback = 1 if traceback else 0
    p.precision = int(precision)
    p._keep = s
    return p


class Context:
    """One filtr_ctx on one device."""

    def __init__(self, device: int = 0, workspace_bytes: int = 0):
        h = C.c_void_p()
        check(lib().filtr_ctx_create(int(device), int(workspace_bytes), C.byref(h)),
              "filtr_ctx_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().filtr_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- raw calls: device pointers as ints ---------------------------------
    def align_batch_ptr(self, params: Params, n: int, q_seq, q_off, q_len, r_seq, r_off, r_len,
                        out, cigar, cigar_cap: int, stream: int = 0, plain: bool = False) -> int:
        f = lib().filtr_align_batch_plain if plain else lib().filtr_align_batch
        return f(self.handle, C.byref(params), int(n), q_seq, q_off, q_len, r_seq, r_off, r_len,
                 out, cigar, int(cigar_cap), C.c_void_p(int(stream)) if stream else None)

    def search_batch_ptr(self, params: SearchParams, n: int, q_seq, q_off, q_len, r_seq, r_off,
                         r_len, out, cigar, cigar_cap: int, stream: int = 0) -> int:
        return lib().filtr_search_batch(self.handle, C.byref(params), int(n), q_seq, q_off, q_len,
                                        r_seq, r_off, r_len, out, cigar, int(cigar_cap),
                                        C.c_void_p(int(stream)) if stream else None)

    def fold_batch_ptr(self, params: FoldParams, n: int, seq, off, lens, out, partner,
                       stream: int = 0) -> int:
        return lib().filtr_fold_batch(self.handle, C.byref(params), int(n), seq, off, lens, out,
                                      partner, C.c_void_p(int(stream)) if stream else None)

    def align_batch_host_ptr(self, params: Params, n: int, q_seq, q_off, q_len, r_seq, r_off,
                             r_len, out, cigar, cigar_cap: int) -> int:
        return lib().filtr_align_batch_host(self.handle, C.byref(params), int(n), q_seq, q_off,
                                            q_len, r_seq, r_off, r_len, out, cigar, int(cigar_cap))

    def align_long_ptr(self, params: Params, q, M: int, r, N: int, out, cigar, cap: int,
                       stream: int = 0) -> int:
        return lib().filtr_align_long(self.handle, C.byref(params), q, int(M), r, int(N), out,
                                      cigar, int(cap),
                                      C.c_void_p(int(stream)) if stream else None)

    def set_timing(self, on: bool):
        check(lib().filtr_ctx_set_timing(self.handle, 1 if on else 0), "filtr_ctx_set_timing")

    def last_stats(self) -> dict:
        st = Stats()
        check(lib().filtr_ctx_last_stats(self.handle, C.byref(st)), "filtr_ctx_last_stats")
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def autotune(self, params) -> dict:
        """Time the tiled kernel shapes for this recurrence kind (filtr_autotune);
        returns {"i32 R=32": ns per warp step, ...} for the shapes timed, or for
        X-drop / Z-drop parameters {"sweep i16x2 W=1": ns per cell, ...} for the
        sweep candidates timed."""
        rep = TuneReport()
        check(lib().filtr_autotune(self.handle, C.byref(params), C.byref(rep)), "filtr_autotune")
        sweep = bool(params.prune & (PRUNE_XDROP | PRUNE_ZDROP)) or params.affine == AFFINE_MID
        out = {}
        for k in range(rep.n_shapes):
            if rep.ns_per_warp_step[k] > 0:
                kind = "i16x2" if rep.packed[k] else "i32"
                key = (f"sweep {kind} W={rep.rows_per_lane[k]}" if sweep
                       else f"{kind} R={rep.rows_per_lane[k]}")
                out[key] = rep.ns_per_warp_step[k]
        return out

    def tune_apply(self, params, table: dict):
        """Install costs from an earlier autotune() table (filtr_tune_apply);
        shapes missing from the table keep the scaled built-in cost."""
        rep = TuneReport()
        if params.prune & (PRUNE_XDROP | PRUNE_ZDROP) or params.affine == AFFINE_MID:
            rep.n_shapes = len(TUNE_SWEEP)
            for k, (kind, W) in enumerate(TUNE_SWEEP):
                rep.rows_per_lane[k] = W
                rep.packed[k] = 1 if kind == "i16x2" else 0
                rep.ns_per_warp_step[k] = float(table.get(f"sweep {kind} W={W}", 0.0))
            check(lib().filtr_tune_apply(self.handle, C.byref(params), C.byref(rep)),
                  "filtr_tune_apply")
            return
        rep.n_shapes = len(TUNE_SHAPES)
        for k, (kind, R) in enumerate(TUNE_SHAPES):
            rep.rows_per_lane[k] = R
            rep.packed[k] = 1 if kind == "i16x2" else 0
            rep.ns_per_warp_step[k] = float(table.get(f"{kind} R={R}", 0.0))
        check(lib().filtr_tune_apply(self.handle, C.byref(params), C.byref(rep)),
              "filtr_tune_apply")

    def probe(self):
        arr = (C.c_double * 5)()
        check(lib().filtr_probe_int_peak(self.handle, C.byref(arr)), "filtr_probe_int_peak")
        return dict(int_ops=arr[0], viaddmax=arr[1], vimax3=arr[2], viaddmax_s16x2_lanes=arr[3],
                    sm_hz=arr[4])


class Graph:
    """The batched tiled pipeline captured as a CUDA graph (filtr_graph_*)."""

    def __init__(self, ctx: "Context", params: Params, max_pairs: int, max_len: int,
                 workspace_bytes: int):
        h = C.c_void_p()
        check(lib().filtr_graph_create(ctx.handle, C.byref(params), int(max_pairs), int(max_len),
                                       int(workspace_bytes), C.byref(h)), "filtr_graph_create")
        self.handle = h
        self.params = params
        self.max_pairs = int(max_pairs)

    def launch_ptr(self, n: int, q_seq, q_off, q_len, r_seq, r_off, r_len, out, cigar,
                   cigar_cap: int, stream: int = 0) -> int:
        return lib().filtr_graph_launch(self.handle, int(n), q_seq, q_off, q_len, r_seq, r_off,
                                        r_len, out, cigar, int(cigar_cap),
                                        C.c_void_p(int(stream)) if stream else None)

    def status(self) -> int:
        return lib().filtr_graph_status(self.handle)

    def close(self):
        if self.handle:
            lib().filtr_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
