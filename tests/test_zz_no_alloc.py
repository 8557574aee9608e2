"""filtr_align_batch_noalloc: the score-only batched alignment whose scratch is a
fixed device array inside the library, for callers that cannot allocate device
memory (a host framework that owns it, or a path that cannot take cudaMalloc's
device-wide synchronisation).  Called through the C ABI twice in a row on
different batches; each result must equal the oracle's and filtr_align_batch's
exactly (integer outputs, tolerance 0).  A pair longer than the limits the call
was given comes back FILTR_ST_TOO_WIDE while the others are computed as usual.
This file is collected last."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FIELDS = ("score", "q_begin", "q_end", "r_begin", "r_end", "status", "cells")
ORACLE_FIELDS = ("score", "q_end", "r_end", "status", "cells")


@pytest.fixture(scope="module")
def F():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_06225_gb300 as F

    return F


def noalloc(F, params, batch, max_q=None, max_r=None):
    import torch

    db = F.DeviceBatch(batch)
    out = torch.zeros(batch.n * F.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    max_q = int(batch.q_len.max()) if max_q is None else int(max_q)
    max_r = int(batch.r_len.max()) if max_r is None else int(max_r)
    rc = F.lib().filtr_align_batch_noalloc(
        C.byref(params), batch.n, *db.ptrs(), max_q, max_r, out.data_ptr(),
        C.c_void_p(s.cuda_stream))
    s.synchronize()
    return rc, F.results_to_numpy(out, batch.n)


def test_matches_align_batch_twice(F):
    ctx = F.Context(0, 1 << 30)
    P = synth.protein_pairs(n=400, lmin=50, lmax=1200, seed=31)
    D = synth.short_dna_pairs(n=300, length=700, seed=32)
    calls = [(P, dict(P.scoring, traceback=False)),
             (D, dict(D.scoring, band=40, traceback=False))]
    for batch, sc in calls:  # two calls in a row, different batches and modes
        params = F.make_params(batch.subst, **sc)
        rc, got = noalloc(F, params, batch)
        assert rc == 0, F.last_error()
        ores = oracle.align_batch(batch, **sc)[0]
        for f in ORACLE_FIELDS:
            assert np.array_equal(got[f].astype(np.int64), ores[f].astype(np.int64)), f
        want, _, rc2 = F.align_batch(ctx, params, batch)
        assert rc2 == 0
        for f in FIELDS:
            assert np.array_equal(got[f], want[f]), f
    ctx.close()


def test_pairs_beyond_the_given_limits(F):
    """Limits below some pairs' lengths: those pairs (and only those) come back
    FILTR_ST_TOO_WIDE; every other pair equals the oracle exactly."""
    P = synth.protein_pairs(n=300, lmin=50, lmax=900, seed=34)
    sc = dict(P.scoring, traceback=False)
    params = F.make_params(P.subst, **sc)
    max_q, max_r = 700, 600
    rc, got = noalloc(F, params, P, max_q=max_q, max_r=max_r)
    assert rc == 0, F.last_error()
    over = (P.q_len > max_q) | (P.r_len > max_r)
    assert over.any() and (~over).any()
    assert (got["status"][over] == F.ST_TOO_WIDE).all()
    ores = oracle.align_batch(P, **sc)[0]
    for f in ORACLE_FIELDS:
        assert np.array_equal(got[f][~over].astype(np.int64), ores[f][~over].astype(np.int64)), f


def test_rejects_what_it_cannot_hold(F):
    b = synth.short_dna_pairs(n=4, seed=33)
    db = F.DeviceBatch(b)
    import torch

    out = torch.zeros(4 * F.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    p = F.make_params(b.subst, **dict(b.scoring, traceback=True))
    rc = F.lib().filtr_align_batch_noalloc(C.byref(p), 4, *db.ptrs(), 200, 200, out.data_ptr(), None)
    assert rc == F.ERR_UNSUPPORTED
    p = F.make_params(b.subst, **dict(b.scoring, traceback=False))
    rc = F.lib().filtr_align_batch_noalloc(C.byref(p), 4, *db.ptrs(), 200, 3_000_000,
                                           out.data_ptr(), None)
    assert rc == F.ERR_UNSUPPORTED
