"""The packed (int16x2) antidiagonal sweep: X-drop and Z-drop pairs of affine
H/E/F alignments run two cells per register, values held relative to a base
score that follows the best.  Bit-exact against the oracle and against the
int32 sweep (tolerance 0: exact integers), including pairs whose scores leave
the 16-bit range when the base is never moved (filtr_test_set_packed_sweep
mode 2): those stop and are rerun by the int32 sweep, which the statistics
count."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare, oracle_batch

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
    c = F.Context(0, 4 << 30)
    c.set_timing(True)
    yield c
    c.close()


def run(F, ctx, batch, sc, mode=0):
    assert F.lib().filtr_test_set_packed_sweep(ctx.handle, mode) == 0
    try:
        params = F.make_params(batch.subst, **sc)
        res, cig, rc = F.align_batch(ctx, params, batch)
        assert rc == 0, F.last_error()
        st = ctx.last_stats()
    finally:
        F.lib().filtr_test_set_packed_sweep(ctx.handle, 0)
    return res, cig, st


def mixed(seed, n=100, lmax=700):
    qs, rs = synth.random_pairs(n, lmax, lmax, 4, seed=seed, related=0.7)
    rng = np.random.default_rng(seed)
    for M, N in [(1, 1), (0, 7), (7, 0), (1, 60), (60, 1), (3, 200), (260, 255)]:
        qs.append(rng.integers(0, 4, size=M).astype(np.uint8))
        rs.append(rng.integers(0, 4, size=N).astype(np.uint8))
    r = rng.integers(0, 4, size=400).astype(np.uint8)
    qs.append(r.copy())
    rs.append(r)
    return synth.pack(qs, rs, 4, DNA_S)


CASES = [
    dict(mode="global", xdrop=0), dict(mode="global", xdrop=7), dict(mode="global", xdrop=40),
    dict(mode="global", xdrop=400), dict(mode="local", xdrop=9), dict(mode="local", xdrop=60),
    dict(mode="global", zdrop=30), dict(mode="local", zdrop=50),
    dict(mode="global", xdrop=30, xdrop_running=True), dict(mode="global", zdrop=25, xdrop_running=True),
    dict(mode="global", xdrop=60, band=16), dict(mode="global", xdrop=60, band=20, band_literal=True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
@pytest.mark.parametrize("tb", [True, False])
def test_packed_equals_oracle_and_int32(F, ctx, case, tb):
    b = mixed(1000 + len(str(case)), n=90)
    sc = dict(affine=True, gap_open=4, gap_extend=2, traceback=tb, **case)
    res, cig, st = run(F, ctx, b, sc)
    assert st["pairs_xd16"] > 0
    ores, oops, ooff = oracle_batch(b, sc)
    compare(b, sc, res, cig, ores, oops, ooff, label=f"packed {case}")
    r32, c32, st32 = run(F, ctx, b, sc, mode=1)
    assert st32["pairs_xd16"] == 0
    assert np.array_equal(res, r32)
    if tb:
        used = int((res["cigar_off"] + res["cigar_len"]).max())
        assert np.array_equal(cig[:used], c32[:used])


WIDE = [dict(mode="global", xdrop=40), dict(mode="local", xdrop=60), dict(mode="global", zdrop=30),
        dict(mode="local", zdrop=50), dict(mode="global", xdrop=60, band=16),
        dict(mode="global", zdrop=25, xdrop_running=True)]


@pytest.mark.parametrize("case", WIDE, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
@pytest.mark.parametrize("width", [2, 4])
def test_packed_first_width(F, ctx, case, width):
    """The packed sweep started at a 512-slot window (one warp of 16-slot
    threads) or at 1024 slots (four warps of 8-slot threads): the same results
    and CIGARs as the oracle and as the default first width."""
    b = mixed(2000 + len(str(case)), n=60)
    sc = dict(affine=True, gap_open=4, gap_extend=2, traceback=True, **case)
    ref, rcig, _ = run(F, ctx, b, sc)
    assert F.lib().filtr_test_set_first_width(ctx.handle, width) == 0
    try:
        res, cig, st = run(F, ctx, b, sc)
    finally:
        F.lib().filtr_test_set_first_width(ctx.handle, 0)
    assert st["pairs_xd16"] > 0
    ores, oops, ooff = oracle_batch(b, sc)
    compare(b, sc, res, cig, ores, oops, ooff, label=f"first width {width} {case}")
    assert np.array_equal(res, ref)
    used = int((res["cigar_off"] + res["cigar_len"]).max())
    assert np.array_equal(cig[:used], rcig[:used])


def test_protein_scores_by_table(F, ctx):
    """A 20x20 matrix (scores looked up per cell pair, not by code comparison)."""
    P = synth.protein_pairs(n=60, lmin=30, lmax=600, seed=23)
    for mode in ("global", "local"):
        sc = dict(mode=mode, affine=True, gap_open=11, gap_extend=1, xdrop=45, traceback=True)
        res, cig, st = run(F, ctx, P, sc)
        assert st["pairs_xd16"] > 0
        ores, oops, ooff = oracle_batch(P, sc)
        compare(P, sc, res, cig, ores, oops, ooff, label=f"protein {mode}")


def test_long_reads_rebase(F, ctx):
    """Long reads whose global scores climb far past the 16-bit range: the base
    follows the best, nothing leaves the range, every pair equals the oracle."""
    b = synth.long_reads(n=8, lmin=18000, lmax=26000, seed=51)
    sc = dict(b.scoring)
    res, cig, st = run(F, ctx, b, sc)
    assert st["pairs_xd16"] == b.n and st["pairs_xd16_rerun"] == 0
    assert int(res["score"].max()) > 20000
    ores, oops, ooff = oracle_batch(b, sc)
    compare(b, sc, res, cig, ores, oops, ooff, label="rebase")


def test_overflow_rerun_in_int32(F, ctx):
    """With the base never moved, pairs whose scores drift past the 16-bit range
    stop in the packed sweep and are rerun by the int32 sweep (counted), while
    shorter pairs stay packed; every result equals the oracle."""
    long_b = synth.long_reads(n=6, lmin=18000, lmax=26000, seed=52)
    short_b = synth.long_reads(n=10, lmin=1000, lmax=3000, seed=53)
    qs = [long_b.pair(p)[0] for p in range(long_b.n)] + [short_b.pair(p)[0] for p in range(short_b.n)]
    rs = [long_b.pair(p)[1] for p in range(long_b.n)] + [short_b.pair(p)[1] for p in range(short_b.n)]
    b = synth.pack(qs, rs, 4, DNA_S, dict(long_b.scoring))
    sc = dict(b.scoring)
    res, cig, st = run(F, ctx, b, sc, mode=2)
    assert st["pairs_xd16"] == b.n
    assert 1 <= st["pairs_xd16_rerun"] <= long_b.n
    ores, oops, ooff = oracle_batch(b, sc)
    compare(b, sc, res, cig, ores, oops, ooff, label="overflow rerun")


@pytest.mark.parametrize("interval,recompute", [(64, False), (64, True), (1000, True)])
@pytest.mark.parametrize("mode", [0, 2])
def test_long_pair_segmented(F, ctx, interval, recompute, mode):
    """filtr_align_long's segmented sweep in the packed form (checkpoints stored
    as int32 values and repacked on resume), and with the base never moved, where
    the pair leaves the range and the whole sweep reruns in int32."""
    b = synth.long_pair(length=24000, seg=300, seed=54, xdrop=300)
    q, r = b.pair(0)
    sc = dict(b.scoring)
    params = F.make_params(b.subst, **sc)
    lib = F.lib()
    assert lib.filtr_test_set_checkpoint(ctx.handle, interval) == 0
    assert lib.filtr_test_force_recompute(ctx.handle, int(recompute)) == 0
    assert lib.filtr_test_set_packed_sweep(ctx.handle, mode) == 0
    try:
        res, cig, rc = F.align_long(ctx, params, q, r)
    finally:
        lib.filtr_test_set_checkpoint(ctx.handle, 0)
        lib.filtr_test_force_recompute(ctx.handle, 0)
        lib.filtr_test_set_packed_sweep(ctx.handle, 0)
    assert rc == 0, F.last_error()
    o = oracle.align(q, r, b.subst, **sc)
    for f in ("score", "q_end", "r_end", "status", "cells"):
        assert int(res[f]) == int(o[f]), (f, int(res[f]), int(o[f]))
    assert np.array_equal(cig, o["cigar"])


def test_sweep_autotune_and_apply(F):
    """filtr_autotune with X-drop parameters times the int16x2 and int32 sweeps at
    a first width of one and two warps and keeps the fastest; filtr_tune_apply
    installs a saved choice.  Results never change: every choice equals the
    oracle; a table with only int32 candidates runs no pair packed."""
    b = synth.long_reads(n=40, lmin=2000, lmax=4000, seed=61)
    sc = dict(b.scoring)
    params = F.make_params(b.subst, **sc)
    ores, oops, ooff = oracle_batch(b, sc)
    c = F.Context(0, 4 << 30)
    try:
        table = c.autotune(params)
        assert set(table) <= {"sweep i16x2 W=1", "sweep i32 W=1", "sweep i16x2 W=2", "sweep i32 W=2"}
        assert "sweep i16x2 W=1" in table and "sweep i32 W=1" in table
        assert all(v > 0 for v in table.values())
        c.set_timing(True)
        res, cig, rc = F.align_batch(c, params, b)
        assert rc == 0, F.last_error()
        compare(b, sc, res, cig, ores, oops, ooff, label="tuned sweep")
        only32 = {k: v for k, v in table.items() if "i32" in k}
        c.tune_apply(params, only32)
        res, cig, rc = F.align_batch(c, params, b)
        assert rc == 0, F.last_error()
        assert c.last_stats()["pairs_xd16"] == 0
        compare(b, sc, res, cig, ores, oops, ooff, label="int32 sweep by tune table")
        c.tune_apply(params, {"sweep i16x2 W=2": 1.0})
        res, cig, rc = F.align_batch(c, params, b)
        assert rc == 0, F.last_error()
        assert c.last_stats()["pairs_xd16"] == b.n
        compare(b, sc, res, cig, ores, oops, ooff, label="packed sweep at two warps by tune table")
    finally:
        c.close()
