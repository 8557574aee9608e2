"""filtr_align_long: one pair across the whole GPU.  Multi-strip full-matrix and
banded pairs (cooperative strip kernel with release/acquire progress words)
and long X-drop pairs against the oracle, bit-exact; the megabase pair checked
by properties that hold at any size; and the bounded strip wait, made to run
out by a producer that never publishes."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from pins import rescore_cigar

pytestmark = pytest.mark.gpu

DNA_S = synth.dna_subst(2, -4)


@pytest.fixture(scope="module")
def F():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_06225_gb300 as F

    return F


@pytest.fixture(scope="module")
def ctx(F):
    c = F.Context(0, 8 << 30)
    yield c
    c.close()


def check_pair(F, ctx, q, r, S, sc):
    params = F.make_params(S, **sc)
    res, cig, rc = F.align_long(ctx, params, q, r)
    assert rc == 0, F.last_error()
    o = oracle.align(q, r, S, **sc)
    for f in ("score", "q_end", "r_end", "status", "cells"):
        assert int(res[f]) == int(o[f]), (f, int(res[f]), int(o[f]))
    if sc.get("traceback"):
        assert (int(res["q_begin"]), int(res["r_begin"])) == (o["q_begin"], o["r_begin"])
        assert np.array_equal(cig, o["cigar"])


@pytest.mark.parametrize("mode", ["global", "local"])
@pytest.mark.parametrize("tb", [False, True])
def test_full_multi_strip(F, ctx, mode, tb):
    rng = np.random.default_rng(3)
    r = rng.integers(0, 4, 2300).astype(np.uint8)
    q = synth.mutate(rng, r, 0.05, 0.02, 0.02, 0.7)[:3100]
    check_pair(F, ctx, q, r, DNA_S, dict(mode=mode, affine=True, gap_open=4, gap_extend=2,
                                         traceback=tb))


def test_protein_local(F, ctx):
    P = synth.protein_subst(np.random.default_rng(2))
    rng = np.random.default_rng(8)
    r = rng.integers(0, 20, 1800).astype(np.uint8)
    q = np.concatenate([rng.integers(0, 20, 700).astype(np.uint8), r[300:1500]])
    check_pair(F, ctx, q, r, P, dict(mode="local", affine=True, gap_open=11, gap_extend=1,
                                     traceback=True))


@pytest.mark.parametrize("literal", [False, True])
def test_banded_long(F, ctx, literal):
    rng = np.random.default_rng(4)
    r = rng.integers(0, 4, 20000).astype(np.uint8)
    q = synth.mutate(rng, r, 0.01, 0.02, 0.01, 0.7)
    check_pair(F, ctx, q, r, DNA_S, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                         band=64, band_literal=literal, traceback=True))


def test_banded_long_local(F, ctx):
    """A local alignment inside a long banded pair: a 12 kbp core at 3/1/1%
    sub/ins/del between random flanks, band 64 around the core's diagonal.  The
    best cell is reduced over every strip's warps, and the warp walk stops at the
    first H of 0 inside the banded tile."""
    rng = np.random.default_rng(21)
    core = rng.integers(0, 4, 12000).astype(np.uint8)
    flank = lambda n: rng.integers(0, 4, n).astype(np.uint8)
    r = np.concatenate([flank(1500), core, flank(800)])
    q = np.concatenate([flank(1500), synth.mutate(rng, core, 0.03, 0.01, 0.01, 0.7), flank(900)])
    check_pair(F, ctx, q, r, DNA_S, dict(mode="local", affine=True, gap_open=4, gap_extend=2,
                                         band=64, traceback=True))


def test_xdrop_long_scaled(F, ctx):
    """The megabase workload's shape at 30 kbp: 1% divergence plus a 300-base
    random insertion, X-drop 200."""
    b = synth.long_pair(length=30000, seg=300, seed=5, xdrop=200)
    q, r = b.pair(0)
    check_pair(F, ctx, q, r, DNA_S, dict(b.scoring))


def test_megabase_pair_properties(F, ctx):
    """The 1,000,000 bp pair (X-drop 1000): the CIGAR re-scores to the reported
    score and consumes exactly the reported spans; cells are reported."""
    b = synth.long_pair()
    q, r = b.pair(0)
    params = F.make_params(b.subst, **b.scoring)
    res, cig, rc = F.align_long(ctx, params, q, r)
    assert rc == 0, F.last_error()
    assert int(res["status"]) in (0, 1)
    sc, dq, dr = rescore_cigar(cig, q, r, b.subst, 4, 2, int(res["q_begin"]), int(res["r_begin"]))
    assert sc == int(res["score"])
    assert dq == int(res["q_end"]) - int(res["q_begin"])
    assert dr == int(res["r_end"]) - int(res["r_begin"])
    assert int(res["cells"]) > 0


def test_strip_wait_timeout_and_recovery(F, ctx):
    import torch

    rng = np.random.default_rng(9)
    q = rng.integers(0, 4, 2000).astype(np.uint8)
    r = rng.integers(0, 4, 1500).astype(np.uint8)
    qd = torch.from_numpy(q).cuda()
    rd = torch.from_numpy(r).cuda()
    params = F.make_params(DNA_S, mode="global", gap_open=4, gap_extend=2)
    rc = F.lib().filtr_test_long_timeout(ctx.handle, C.byref(params), qd.data_ptr(), 2000,
                                         rd.data_ptr(), 1500, 2_000_000)
    assert rc == F._lib.ERR_TIMEOUT
    # the context (and the GPU) stay usable
    check_pair(F, ctx, q, r, DNA_S, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                         traceback=True))


@pytest.mark.parametrize("interval", [7, 64, 1000])
@pytest.mark.parametrize("recompute", [False, True])
def test_checkpointed_traceback(F, ctx, interval, recompute):
    """Forcing the segmented X-drop sweep (state kept every `interval`
    antidiagonals) gives the oracle's result, including pairs that end DROPPED
    and local alignments, both in its single pass (every segment's traceback
    kept and walked once) and with the segments recomputed backwards."""
    cases = []
    b = synth.long_pair(length=6000, seg=150, seed=11, xdrop=120)
    cases.append((b.pair(0), b.subst, dict(b.scoring)))
    rng = np.random.default_rng(12)
    r = rng.integers(0, 4, 3000).astype(np.uint8)
    q = np.concatenate([r[:1500], rng.integers(0, 4, 900).astype(np.uint8)])
    cases.append(((q, r), DNA_S, dict(mode="global", affine=True, gap_open=4, gap_extend=2, xdrop=30,
                                       traceback=True)))
    cases.append(((q, r), DNA_S, dict(mode="local", affine=True, gap_open=4, gap_extend=2, xdrop=60,
                                       traceback=True)))
    assert F.lib().filtr_test_set_checkpoint(ctx.handle, interval) == 0
    assert F.lib().filtr_test_force_recompute(ctx.handle, int(recompute)) == 0
    try:
        for (qq, rr), S, sc in cases:
            check_pair(F, ctx, qq, rr, S, sc)
    finally:
        F.lib().filtr_test_set_checkpoint(ctx.handle, 0)
        F.lib().filtr_test_force_recompute(ctx.handle, 0)


def test_traceback_pool_exhausted_falls_back(F, ctx):
    """A context too small to keep a ~200 kb X-drop pair's whole traceback runs
    out of pool in the single pass and falls back to recomputing the segments;
    the result equals the single pass's in a large context."""
    b = synth.long_pair(length=200_000, seg=1000, seed=17, xdrop=400)
    q, r = b.pair(0)
    params = F.make_params(b.subst, **b.scoring)
    big, cig_big, rc = F.align_long(ctx, params, q, r)
    assert rc == 0, F.last_error()
    small = F.Context(0, 40 << 20)
    try:
        res, cig, rc = F.align_long(small, params, q, r)
        assert rc == 0, F.last_error()
    finally:
        small.close()
    assert np.array_equal(res, big)
    assert np.array_equal(cig, cig_big)
    assert int(res["status"]) in (0, 1)
