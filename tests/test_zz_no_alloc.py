"""filtr_align_batch_noalloc: the score-only batched alignment whose scratch is a
fixed device array inside the library, for callers that cannot allocate device
memory (a host framework that owns it, or a path that cannot take cudaMalloc's
device-wide synchronisation).  Called through the C ABI twice in a row on
different batches; each result must equal filtr_align_batch's exactly
(integer outputs, tolerance 0).  This file is collected last."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FIELDS = ("score", "q_begin", "q_end", "r_begin", "r_end", "status", "cells")


@pytest.fixture(scope="module")
def F():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_06225_gb300 as F

    return F


def noalloc(F, params, batch):
    import torch

    db = F.DeviceBatch(batch)
    out = torch.zeros(batch.n * F.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    rc = F.lib().filtr_align_batch_noalloc(
        C.byref(params), batch.n, *db.ptrs(), int(batch.q_len.max()), int(batch.r_len.max()),
        out.data_ptr(), C.c_void_p(s.cuda_stream))
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
        want, _, rc2 = F.align_batch(ctx, params, batch)
        assert rc2 == 0
        for f in FIELDS:
            assert np.array_equal(got[f], want[f]), f
    ctx.close()


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
