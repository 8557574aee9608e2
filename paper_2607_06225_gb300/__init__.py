"""GB300 pairwise alignment (NW / SW, linear and affine gaps -- Gotoh H/E/F or
Table 1's M/I/D --, band, X-drop and Z-drop pruning, CIGAR traceback), edit
distance by the search traversal (with WFA-Adapt) and Nussinov RNA folding with
X-drop, behind the C ABI in include/filtr.h.

This package is the thin Python face of libfiltr.so: it marshals numpy / torch
buffers into C-ABI calls.  PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import numpy as np

from ._lib import (ALPHA_DNA, ALPHA_PROTEIN, ERR_CIGAR_CAP, ERR_INVALID, ERR_NOMEM, ERR_UNSUPPORTED,
                   GLOBAL,
                   LOCAL, OK, PREC_AUTO, PREC_I16X2, PREC_I32, PRUNE_BAND, PRUNE_BAND_LITERAL,
                   PRUNE_XDROP, PRUNE_ZDROP, RESULT_DTYPE, ST_DROPPED, ST_EMPTY, ST_OK, ST_TOO_WIDE,
                   ST_UNREACHABLE, TUNE_SHAPES, XDROP_INF, Context, FiltrError, Graph, Params,
                   FOLD_RESULT_DTYPE, FoldParams, SearchParams, check, last_error, lib,
                   make_fold_params, make_params, make_search_params)

__all__ = ["Context", "FiltrError", "Params", "make_params", "DeviceBatch", "align_batch",
           "align_batch_host", "align_long", "RESULT_DTYPE", "lib", "last_error", "SearchParams",
           "make_search_params", "search_batch", "FoldParams", "make_fold_params", "fold_batch"]


class DeviceBatch:
    """A batch resident on the device (torch tensors), in the C-ABI layout."""

    def __init__(self, batch, device="cuda"):
        import torch

        def t(x, dt):
            return torch.from_numpy(np.ascontiguousarray(x).astype(dt, copy=False)).to(device)

        self.n = int(batch.q_len.shape[0])
        self.q_seq = t(batch.q_seq if batch.q_seq.size else np.zeros(1, np.uint8), np.uint8)
        self.r_seq = t(batch.r_seq if batch.r_seq.size else np.zeros(1, np.uint8), np.uint8)
        self.q_off = t(batch.q_off.view(np.int64), np.int64)
        self.r_off = t(batch.r_off.view(np.int64), np.int64)
        self.q_len = t(batch.q_len.view(np.int32), np.int32)
        self.r_len = t(batch.r_len.view(np.int32), np.int32)
        self.cigar_upper = int(batch.q_len.astype(np.int64).sum() + batch.r_len.astype(np.int64).sum())

    def ptrs(self):
        return (self.q_seq.data_ptr(), self.q_off.data_ptr(), self.q_len.data_ptr(),
                self.r_seq.data_ptr(), self.r_off.data_ptr(), self.r_len.data_ptr())


def alloc_outputs(n: int, cigar_cap: int, device="cuda"):
    import torch

    out = torch.empty(max(n, 1) * RESULT_DTYPE.itemsize, dtype=torch.uint8, device=device)
    cig = torch.empty(max(cigar_cap, 1), dtype=torch.int32, device=device)
    return out, cig


def results_to_numpy(out_t, n: int):
    return out_t[: n * RESULT_DTYPE.itemsize].cpu().numpy().view(RESULT_DTYPE).copy()


def align_batch(ctx: Context, params: Params, batch, stream=None, plain: bool = False,
                cigar_cap: int | None = None, device="cuda", raise_on_error=True):
    """Align a synth.Batch (host numpy) or a DeviceBatch on the device.

    Returns (results structured array, cigar ops uint32 array, status code)."""
    import torch

    db = batch if isinstance(batch, DeviceBatch) else DeviceBatch(batch, device)
    cap = db.cigar_upper if cigar_cap is None else int(cigar_cap)
    out_t, cig_t = alloc_outputs(db.n, cap, device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = ctx.align_batch_ptr(params, db.n, *db.ptrs(), out_t.data_ptr(),
                             cig_t.data_ptr() if params.traceback else None, cap if params.traceback else 0,
                             stream=s.cuda_stream, plain=plain)
    if rc not in (OK, ERR_CIGAR_CAP) and raise_on_error:
        check(rc, "filtr_align_batch")
    s.synchronize()
    res = results_to_numpy(out_t, db.n)
    cig = cig_t.cpu().numpy().view(np.uint32).copy() if params.traceback else np.zeros(0, np.uint32)
    return res, cig, rc


def search_batch(ctx: Context, params: SearchParams, batch, stream=None,
                 cigar_cap: int | None = None, device="cuda", raise_on_error=True):
    """Edit distance of every pair of a synth.Batch or DeviceBatch by the search
    traversal (filtr_search_batch).  Returns (results, cigar ops, status code);
    results' score is minus the distance found."""
    import torch

    db = batch if isinstance(batch, DeviceBatch) else DeviceBatch(batch, device)
    cap = db.cigar_upper + db.n if cigar_cap is None else int(cigar_cap)
    out_t, cig_t = alloc_outputs(db.n, cap, device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = ctx.search_batch_ptr(params, db.n, *db.ptrs(), out_t.data_ptr(),
                              cig_t.data_ptr() if params.traceback else None,
                              cap if params.traceback else 0, stream=s.cuda_stream)
    if rc not in (OK, ERR_CIGAR_CAP) and raise_on_error:
        check(rc, "filtr_search_batch")
    s.synchronize()
    res = results_to_numpy(out_t, db.n)
    cig = cig_t.cpu().numpy().view(np.uint32).copy() if params.traceback else np.zeros(0, np.uint32)
    return res, cig, rc


def fold_batch(ctx: Context, params: FoldParams, seq, off, lens, stream=None, device="cuda",
               raise_on_error=True):
    """Fold RNAs (host numpy codes, offsets, lengths) with filtr_fold_batch.
    Returns (results structured array, partner int32 array in seq's layout,
    status code)."""
    import torch

    n = int(len(lens))
    seq_t = torch.from_numpy(np.ascontiguousarray(seq, dtype=np.uint8)
                             if len(seq) else np.zeros(1, np.uint8)).to(device)
    off_t = torch.from_numpy(np.ascontiguousarray(off, dtype=np.uint64).view(np.int64)).to(device)
    len_t = torch.from_numpy(np.ascontiguousarray(lens, dtype=np.uint32).view(np.int32)).to(device)
    out_t = torch.empty(max(n, 1) * FOLD_RESULT_DTYPE.itemsize, dtype=torch.uint8, device=device)
    part_t = torch.full((max(int(len(seq)), 1),), -1, dtype=torch.int32, device=device)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = ctx.fold_batch_ptr(params, n, seq_t.data_ptr(), off_t.data_ptr(), len_t.data_ptr(),
                            out_t.data_ptr(), part_t.data_ptr() if params.traceback else None,
                            stream=s.cuda_stream)
    if rc != OK and raise_on_error:
        check(rc, "filtr_fold_batch")
    s.synchronize()
    res = out_t[: n * FOLD_RESULT_DTYPE.itemsize].cpu().numpy().view(FOLD_RESULT_DTYPE).copy()
    return res, part_t.cpu().numpy()[: int(len(seq))].copy(), rc


def graph_align(graph: Graph, batch, stream=None, cigar_cap: int | None = None, device="cuda"):
    """One launch of a captured pipeline over a synth.Batch or DeviceBatch; waits
    for it and returns (results, cigar ops, the launch's filtr_graph_status)."""
    import torch

    db = batch if isinstance(batch, DeviceBatch) else DeviceBatch(batch, device)
    cap = db.cigar_upper if cigar_cap is None else int(cigar_cap)
    out_t, cig_t = alloc_outputs(db.n, cap, device)
    s = stream if stream is not None else torch.cuda.current_stream()
    tb = bool(graph.params.traceback)
    rc = graph.launch_ptr(db.n, *db.ptrs(), out_t.data_ptr(), cig_t.data_ptr() if tb else None,
                          cap if tb else 0, stream=s.cuda_stream)
    check(rc, "filtr_graph_launch")
    s.synchronize()
    status = graph.status() if db.n else OK
    res = results_to_numpy(out_t, db.n)
    cig = cig_t.cpu().numpy().view(np.uint32).copy() if tb else np.zeros(0, np.uint32)
    return res, cig, status


def align_batch_host(ctx: Context, params: Params, batch, cigar_cap: int | None = None):
    """Host-buffer entry point: every array in host memory (numpy)."""
    n = int(batch.q_len.shape[0])
    cap = int(batch.q_len.astype(np.int64).sum() + batch.r_len.astype(np.int64).sum()) \
        if cigar_cap is None else int(cigar_cap)
    out = np.zeros(max(n, 1), dtype=RESULT_DTYPE)
    cig = np.zeros(max(cap, 1), dtype=np.uint32)
    arrs = [np.ascontiguousarray(x) for x in (batch.q_seq, batch.q_off, batch.q_len, batch.r_seq,
                                              batch.r_off, batch.r_len)]
    rc = ctx.align_batch_host_ptr(params, n, *[a.ctypes.data for a in arrs], out.ctypes.data,
                                  cig.ctypes.data if params.traceback else None,
                                  cap if params.traceback else 0)
    if rc not in (OK, ERR_CIGAR_CAP):
        check(rc, "filtr_align_batch_host")
    return out[:n], cig, rc


def align_long(ctx: Context, params: Params, q: np.ndarray, r: np.ndarray, device="cuda"):
    """One long pair with every SM on it; returns (result row, cigar ops, status)."""
    import torch

    qd = torch.from_numpy(np.ascontiguousarray(q, dtype=np.uint8) if q.size else np.zeros(1, np.uint8)).to(device)
    rd = torch.from_numpy(np.ascontiguousarray(r, dtype=np.uint8) if r.size else np.zeros(1, np.uint8)).to(device)
    cap = int(q.shape[0] + r.shape[0] + 1)
    out_t, cig_t = alloc_outputs(1, cap, device)
    s = torch.cuda.current_stream()
    rc = ctx.align_long_ptr(params, qd.data_ptr(), int(q.shape[0]), rd.data_ptr(), int(r.shape[0]),
                            out_t.data_ptr(), cig_t.data_ptr(), cap, stream=s.cuda_stream)
    if rc not in (OK, ERR_CIGAR_CAP):
        check(rc, "filtr_align_long")
    s.synchronize()
    res = results_to_numpy(out_t, 1)[0]
    cig = cig_t.cpu().numpy().view(np.uint32)
    return res, cig[int(res["cigar_off"]):int(res["cigar_off"]) + int(res["cigar_len"])].copy(), rc


def cigar_of(res_row, cig) -> np.ndarray:
    o, n = int(res_row["cigar_off"]), int(res_row["cigar_len"])
    return cig[o:o + n]


class Server:
    """Continuous-batching server (filtr_serve_*): submit single pairs from any
    thread, poll or wait for results."""

    def __init__(self, ctx: Context, mem_budget: int, max_inflight: int = 4):
        import ctypes as C

        h = C.c_void_p()
        check(lib().filtr_serve_create(ctx.handle, int(mem_budget), int(max_inflight), C.byref(h)),
              "filtr_serve_create")
        self.handle = h
        self._keep = {}

    def submit(self, params: Params, q: np.ndarray, r: np.ndarray) -> int:
        import ctypes as C

        q = np.ascontiguousarray(q, dtype=np.uint8)
        r = np.ascontiguousarray(r, dtype=np.uint8)
        t = C.c_uint64()
        rc = lib().filtr_serve_submit(self.handle, C.byref(params), q.ctypes.data, int(q.shape[0]),
                                      r.ctypes.data, int(r.shape[0]), C.byref(t))
        check(rc, "filtr_serve_submit")
        return int(t.value)

    def wait(self, ticket: int, timeout_us: int = -1, cap: int = 1 << 22):
        """Returns (result row, cigar ops, (t_submit, t_launch, t_done) in ns)."""
        import ctypes as C

        from ._lib import Result

        res = Result()
        cig = np.zeros(max(cap, 1), dtype=np.uint32)
        times = np.zeros(3, dtype=np.uint64)
        rc = lib().filtr_serve_wait(self.handle, int(ticket), int(timeout_us), C.byref(res),
                                    cig.ctypes.data, int(cap), times.ctypes.data)
        check(rc, "filtr_serve_wait")
        row = np.zeros(1, dtype=RESULT_DTYPE)
        for k, _ in Result._fields_:
            row[k] = getattr(res, k)
        return row[0], cig[: int(res.cigar_len)].copy(), tuple(int(x) for x in times)

    def poll(self, ticket: int, cap: int = 1 << 22):
        """None while running, else like wait()."""
        import ctypes as C

        from ._lib import ERR_BUSY, Result

        res = Result()
        cig = np.zeros(max(cap, 1), dtype=np.uint32)
        times = np.zeros(3, dtype=np.uint64)
        rc = lib().filtr_serve_poll(self.handle, int(ticket), C.byref(res), cig.ctypes.data,
                                    int(cap), times.ctypes.data)
        if rc == ERR_BUSY:
            return None
        check(rc, "filtr_serve_poll")
        row = np.zeros(1, dtype=RESULT_DTYPE)
        for k, _ in Result._fields_:
            row[k] = getattr(res, k)
        return row[0], cig[: int(res.cigar_len)].copy(), tuple(int(x) for x in times)

    def close(self):
        if self.handle:
            lib().filtr_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
