"""Serving (continuous batching): every request's result equals the oracle's and
is identical whether the request ran alone or in a mix of concurrent requests
of every kind (exact integers: tolerance 0)."""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

KINDS = {
    "sw_protein": dict(mode="local", affine=True, gap_open=11, gap_extend=1, traceback=True),
    "band_dna": dict(mode="global", affine=True, gap_open=4, gap_extend=2, band=256, traceback=True),
    "xdrop_dna": dict(mode="global", affine=True, gap_open=4, gap_extend=2, xdrop=400, traceback=True),
}


@pytest.fixture(scope="module")
def F():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_06225_gb300 as F

    return F


def requests(n, seed):
    reqs, psub = synth.serve_mix(n, rate_hz=1000.0, seed=seed, median=600.0, lmax=4000)
    return reqs, psub


def params_for(F, kind, psub):
    S = psub if kind == "sw_protein" else synth.dna_subst(2, -4)
    return F.make_params(S, **KINDS[kind]), S


def test_mix_equals_alone_equals_oracle(F):
    ctx = F.Context(0, 1 << 28)
    srv = F.Server(ctx, 4 << 30, max_inflight=4)
    reqs, psub = requests(60, seed=4)
    P = {k: params_for(F, k, psub) for k in KINDS}
    # the mix: submitted from two threads at once
    tickets = [None] * len(reqs)

    def submit(lo, hi):
        for k in range(lo, hi):
            tickets[k] = srv.submit(P[reqs[k].kind][0], reqs[k].q, reqs[k].r)

    th = [threading.Thread(target=submit, args=(0, 30)), threading.Thread(target=submit, args=(30, 60))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    mixed = [srv.wait(t) for t in tickets]
    # alone: one at a time
    alone = []
    for rq in reqs:
        t = srv.submit(P[rq.kind][0], rq.q, rq.r)
        alone.append(srv.wait(t))
    for k, rq in enumerate(reqs):
        (a, ca, ta), (b, cb, tb) = mixed[k], alone[k]
        assert np.array_equal(np.asarray(a), np.asarray(b)) or all(
            int(a[f]) == int(b[f]) for f in ("score", "q_begin", "q_end", "r_begin", "r_end", "status", "cells"))
        assert np.array_equal(ca, cb)
        assert ta[0] <= ta[1] <= ta[2]
        o = oracle.align(rq.q, rq.r, P[rq.kind][1], **KINDS[rq.kind])
        for f in ("score", "q_begin", "q_end", "r_begin", "r_end", "status", "cells"):
            assert int(a[f]) == int(o[f]), (k, rq.kind, f)
        assert np.array_equal(ca, o["cigar"]), (k, rq.kind)
    srv.close()
    ctx.close()


def test_poll_and_errors(F):
    ctx = F.Context(0, 1 << 28)
    srv = F.Server(ctx, 2 << 30, max_inflight=2)
    psub = synth.protein_subst(np.random.default_rng(2))
    p = F.make_params(psub, **KINDS["sw_protein"])
    rng = np.random.default_rng(1)
    q = rng.integers(0, 20, 300).astype(np.uint8)
    t = srv.submit(p, q, q)
    out = None
    for _ in range(200000):
        out = srv.poll(t)
        if out is not None:
            break
    assert out is not None and int(out[0]["score"]) == int(sum(int(psub[c, c]) for c in q))
    with pytest.raises(F.FiltrError):
        srv.poll(t)  # retrieved tickets are forgotten
    bad = q.copy()
    bad[0] = 25
    with pytest.raises(F.FiltrError):
        srv.submit(p, bad, q)
    srv.close()
    ctx.close()


def test_large_request_route_and_budget_refusal(F):
    """A request above 2^22 cells (a 8200 x 8300 protein pair, local, traceback)
    runs alone on the intra-pair kernel and equals the oracle; a request whose
    traceback exceeds a lane's share of the budget is refused with
    FILTR_ERR_BUSY at submission, and the server keeps serving afterwards."""
    from paper_2607_06225_gb300._lib import ERR_BUSY

    psub = synth.protein_subst(np.random.default_rng(2))
    p = F.make_params(psub, **KINDS["sw_protein"])
    rng = np.random.default_rng(44)
    r = rng.integers(0, 20, 8300).astype(np.uint8)
    q = np.concatenate([rng.integers(0, 20, 3000).astype(np.uint8), r[2000:7200]])
    assert q.shape[0] * r.shape[0] > 1 << 22
    ctx = F.Context(0, 1 << 28)
    srv = F.Server(ctx, 2 << 30, max_inflight=2)
    try:
        t = srv.submit(p, q, r)
        res, cig, _ = srv.wait(t)
        o = oracle.align(q, r, psub, **KINDS["sw_protein"])
        for f in ("score", "q_begin", "q_end", "r_begin", "r_end", "status", "cells"):
            assert int(res[f]) == int(o[f]), f
        assert np.array_equal(cig, o["cigar"])
    finally:
        srv.close()
    # 192 MB over two lanes: 16 MB of I/O buffer and 80 MB of workspace a lane,
    # of which a micro-batch may use 64 MB -- less than the traceback alone of a
    # 12000 x 12000 pair (half a byte per cell, about 72 MB)
    srv = F.Server(ctx, 192 << 20, max_inflight=2)
    try:
        big = rng.integers(0, 20, 12000).astype(np.uint8)
        with pytest.raises(F.FiltrError) as ei:
            srv.submit(p, big, big)
        assert ei.value.code == ERR_BUSY
        small = rng.integers(0, 20, 400).astype(np.uint8)
        res, cig, _ = srv.wait(srv.submit(p, small, small))
        assert int(res["score"]) == int(sum(int(psub[c, c]) for c in small))
    finally:
        srv.close()
        ctx.close()
