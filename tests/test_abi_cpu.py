"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, exports every function include/filtr.h declares, and rejects bad
parameters on the host; plus the host planner's cell-count formula."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2607_06225_gb300 import build

    build.build()
    import paper_2607_06225_gb300._lib as lib

    return lib


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(filtr_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    lib = L.lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_string(L):
    assert b"sm_103a" in L.lib().filtr_version()
    assert isinstance(L.last_error(), str)


def test_params_check(L):
    S = np.zeros((4, 4), np.int8)
    ok = L.make_params(S, gap_open=4, gap_extend=2)
    assert L.lib().filtr_params_check(C.byref(ok)) == L.OK
    for bad in [dict(gap_open=-1), dict(gap_extend=-2), dict(band=-3), dict(xdrop=-1),
                dict(zdrop=-1), dict(precision=7)]:
        p = L.make_params(S, **{**dict(gap_open=4, gap_extend=2), **bad})
        assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_INVALID, bad
    p = L.make_params(np.zeros((5, 5), np.int8))
    assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_INVALID  # alphabet 5
    p = L.make_params(S)
    p.mode = 3
    assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_INVALID
    p = L.make_params(S)
    p.subst = C.POINTER(C.c_int8)()
    assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_INVALID
    assert L.lib().filtr_params_check(None) == L.ERR_INVALID
    # X-drop and Z-drop exclude each other
    with pytest.raises(ValueError):
        L.make_params(S, xdrop=3, zdrop=3)
    p = L.make_params(S, zdrop=3)
    assert L.lib().filtr_params_check(C.byref(p)) == L.OK
    p.prune |= L.PRUNE_XDROP
    assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_INVALID
    # the running threshold needs X-drop or Z-drop
    for kw in (dict(xdrop=3), dict(zdrop=3)):
        p = L.make_params(S, xdrop_running=True, **kw)
        assert L.lib().filtr_params_check(C.byref(p)) == L.OK, kw
    p = L.make_params(S, xdrop_running=True)
    assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_INVALID
    # Table 1's M/I/D form: plain, X-drop or widened band; not Z-drop or the literal band
    for kw in (dict(), dict(xdrop=5), dict(band=8), dict(xdrop=5, xdrop_running=True)):
        p = L.make_params(S, gap_open=4, gap_extend=2, mid=True, **kw)
        assert p.affine == 2
        assert L.lib().filtr_params_check(C.byref(p)) == L.OK, kw
    for kw in (dict(zdrop=5), dict(band=8, band_literal=True)):
        p = L.make_params(S, gap_open=4, gap_extend=2, mid=True, **kw)
        assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_UNSUPPORTED, kw
    p = L.make_params(S)
    p.affine = 3
    assert L.lib().filtr_params_check(C.byref(p)) == L.ERR_INVALID


def test_ctx_create_without_gpu_fails_cleanly(L):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = L.lib().filtr_ctx_create(0, 1 << 20, C.byref(h))
    assert rc in (L.ERR_CUDA, L.ERR_INVALID)
    assert not h.value


def test_tune_apply_rejects_on_host(L):
    """filtr_tune_apply validates its arguments before touching the context."""
    S = np.zeros((4, 4), np.int8)
    p = L.make_params(S, gap_open=4, gap_extend=2)
    rep = L.TuneReport()
    rep.n_shapes = len(L.TUNE_SHAPES)
    for k, (kind, R) in enumerate(L.TUNE_SHAPES):
        rep.rows_per_lane[k] = R
        rep.packed[k] = int(kind == "i16x2")
        rep.ns_per_warp_step[k] = 0.5
    lib = L.lib()
    assert lib.filtr_tune_apply(None, C.byref(p), C.byref(rep)) == L.ERR_INVALID
    assert lib.filtr_tune_apply(None, C.byref(p), None) == L.ERR_INVALID
    assert lib.filtr_tune_apply(None, None, C.byref(rep)) == L.ERR_INVALID
    assert "NULL" in L.last_error()


def test_graph_rejects_on_host(L):
    lib = L.lib()
    S = np.zeros((4, 4), np.int8)
    p = L.make_params(S, gap_open=4, gap_extend=2)
    h = C.c_void_p()
    assert lib.filtr_graph_create(None, C.byref(p), 10, 100, 1 << 26, C.byref(h)) == L.ERR_INVALID
    assert lib.filtr_graph_create(None, C.byref(p), 10, 100, 1 << 26, None) == L.ERR_INVALID
    assert lib.filtr_graph_launch(None, 1, None, None, None, None, None, None, None, None, 0,
                                  None) == L.ERR_INVALID
    assert lib.filtr_graph_status(None) == L.ERR_INVALID
    assert lib.filtr_graph_destroy(None) == L.OK


def test_search_rejects_on_host(L):
    """filtr_search_batch argument checks that need no device."""
    lib = L.lib()
    p = L.make_search_params(traceback=True)
    assert lib.filtr_search_batch(None, C.byref(p), 1, None, None, None, None, None, None, None,
                                  None, 0, None) == L.ERR_INVALID
    assert "NULL" in L.last_error()
    assert p.band == -1 and (p.adapt_min_len, p.adapt_max_dist) == (0, 0)
    q = L.make_search_params(traceback=False, band=7, adapt=(100, 20))
    assert (q.traceback, q.band, q.adapt_min_len, q.adapt_max_dist) == (0, 7, 100, 20)


def test_search_ring_hook_rejects_on_host(L):
    lib = L.lib()
    assert lib.filtr_test_set_search_ring(None, 256) == L.ERR_INVALID


def test_fold_rejects_on_host(L):
    lib = L.lib()
    p = L.make_fold_params(xdrop=2)
    assert (p.min_loop, p.use_xdrop, p.xdrop, p.warmup, p.traceback) == (3, 1, 2, 15, 1)
    assert lib.filtr_fold_batch(None, C.byref(p), 1, None, None, None, None, None,
                                None) == L.ERR_INVALID
    assert L.FOLD_RESULT_DTYPE.itemsize == 24
