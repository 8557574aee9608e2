"""GPU parity of the X-drop antidiagonal kernel against the oracle (bit-exact):
thresholds from 0 (stops on antidiagonal 1) to infinity (whole matrix), with and
without a band, global and local, linear and affine, traceback on and off, the
running-maximum threshold (X-drop and Z-drop, batched and segmented long pairs),
windows that overflow and are rerun with wider groups, and long-read pairs."""
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
    yield c
    c.close()


def run_both(F, ctx, batch, sc):
    params = F.make_params(batch.subst, **sc)
    res, cig, rc = F.align_batch(ctx, params, batch)
    assert rc == 0, F.last_error()
    ores, oops, ooff = oracle_batch(batch, sc)
    compare(batch, sc, res, cig, ores, oops, ooff, label=str(sc))
    return res


def mixed_pairs(seed, n=120, lmax=600):
    qs, rs = synth.random_pairs(n, lmax, lmax, 4, seed=seed, related=0.7)
    rng = np.random.default_rng(seed)
    for M, N in [(1, 1), (1, 50), (50, 1), (3, 200), (200, 3), (257, 255)]:
        qs.append(rng.integers(0, 4, size=M).astype(np.uint8))
        rs.append(rng.integers(0, 4, size=N).astype(np.uint8))
    r = rng.integers(0, 4, size=300).astype(np.uint8)
    qs.append(r.copy())
    rs.append(r)
    return synth.pack(qs, rs, 4, DNA_S)


@pytest.mark.parametrize("X", [0, 5, 12, 40, 400])
@pytest.mark.parametrize("tb", [False, True])
def test_global_affine(F, ctx, X, tb):
    b = mixed_pairs(100 + X)
    run_both(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2, xdrop=X,
                             traceback=tb))


@pytest.mark.parametrize("X", [3, 30])
@pytest.mark.parametrize("mode", ["global", "local"])
@pytest.mark.parametrize("affine", [False, True])
def test_modes(F, ctx, X, mode, affine):
    b = mixed_pairs(7 + X, n=80)
    run_both(F, ctx, b, dict(mode=mode, affine=affine, gap_open=3 if affine else 0, gap_extend=1,
                             xdrop=X, traceback=True))


@pytest.mark.parametrize("band,literal", [(2, False), (16, False), (16, True), (100, False)])
def test_band_and_xdrop(F, ctx, band, literal):
    b = mixed_pairs(31 + band, n=80)
    run_both(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2, xdrop=60,
                             band=band, band_literal=literal, traceback=True))


def test_protein_xdrop(F, ctx):
    P = synth.protein_pairs(n=60, lmin=30, lmax=500, seed=21)
    run_both(F, ctx, P, dict(mode="global", affine=True, gap_open=11, gap_extend=1, xdrop=50,
                             traceback=True))


def test_window_overflow_rerun(F, ctx):
    """X = infinity keeps every cell: the live region grows to the full
    antidiagonal, outgrows the 256-, 1024- and 4096-slot windows and is rerun
    with wider groups."""
    rng = np.random.default_rng(5)
    qs = [rng.integers(0, 4, size=M).astype(np.uint8) for M in (300, 1500, 2500, 5200)]
    rs = [rng.integers(0, 4, size=N).astype(np.uint8) for N in (280, 1400, 2600, 5000)]
    b = synth.pack(qs, rs, 4, DNA_S)
    res = run_both(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                   xdrop=oracle.INF, traceback=True))
    full = oracle_batch(b, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                traceback=True))[0]
    assert np.array_equal(res["score"].astype(np.int64), full["score"])


def test_too_wide_reported(F, ctx):
    """A live region wider than the widest window (8192 cells) is reported, not
    computed wrongly."""
    rng = np.random.default_rng(6)
    q = rng.integers(0, 4, size=9000).astype(np.uint8)
    r = rng.integers(0, 4, size=9000).astype(np.uint8)
    b = synth.pack([q], [r], 4, DNA_S)
    params = F.make_params(DNA_S, mode="global", gap_open=4, gap_extend=2, xdrop=2**31 - 1,
                           traceback=False)
    res, _, rc = F.align_batch(ctx, params, b)
    assert rc == 0 and int(res[0]["status"]) == F.ST_TOO_WIDE


def test_long_reads_sampled(F, ctx):
    """Long noisy reads (band 256 widened to hold both corners, X-drop 400):
    a 300-pair batch of the long-read model with lengths U[2k, 6k], all pairs
    checked against the oracle."""
    b = synth.long_reads(n=300, lmin=2000, lmax=6000, seed=3)
    run_both(F, ctx, b, dict(b.scoring))


def test_plain_equals_batched_xdrop(F, ctx):
    """One launch (and one walk) per pair gives the batched call's results,
    including pairs that outgrow the one-warp window and are rerun wider."""
    b = synth.long_reads(n=12, lmin=1500, lmax=3000, seed=13)
    params = F.make_params(b.subst, **b.scoring)
    r1, c1, rc1 = F.align_batch(ctx, params, b)
    r2, c2, rc2 = F.align_batch(ctx, params, b, plain=True)
    assert rc1 == 0 and rc2 == 0, F.last_error()
    assert np.array_equal(r1, r2)
    used = int((r1["cigar_off"] + r1["cigar_len"]).max())
    assert np.array_equal(c1[:used], c2[:used])
    ores, oops, ooff = oracle_batch(b, dict(b.scoring))
    compare(b, dict(b.scoring), r1, c1, ores, oops, ooff, label="plain")


@pytest.mark.parametrize("kind", ["xdrop", "zdrop"])
@pytest.mark.parametrize("X", [0, 6, 40])
@pytest.mark.parametrize("mode", ["global", "local"])
def test_running_threshold(F, ctx, kind, X, mode):
    """FILTR_PRUNE_XDROP_RUNNING (the threshold follows the best of every
    antidiagonal so far): bit-exact against the oracle's running variant, X-drop
    and Z-drop, with traceback, including pairs whose window is rerun wider."""
    b = mixed_pairs(200 + X, n=100)
    run_both(F, ctx, b, {"mode": mode, "affine": True, "gap_open": 4, "gap_extend": 2,
                         kind: X, "xdrop_running": True, "traceback": True})


def test_running_long_reads(F, ctx):
    b = synth.long_reads(n=60, lmin=2000, lmax=5000, seed=32)
    for kind in ("xdrop", "zdrop"):
        sc = dict(b.scoring, xdrop=None, xdrop_running=True)
        sc[kind] = 400
        run_both(F, ctx, b, sc)


@pytest.mark.parametrize("recompute", [False, True])
def test_running_long_pair_segmented(F, ctx, recompute):
    """filtr_align_long with the running threshold through the segmented sweep
    (the running best and its diagonal carried across checkpoints)."""
    b = synth.long_pair(length=5000, seg=150, seed=33, xdrop=120)
    q, r = b.pair(0)
    for kind, X in (("xdrop", 100), ("zdrop", 60)):
        sc = dict(b.scoring, xdrop=None, xdrop_running=True)
        sc[kind] = X
        params = F.make_params(b.subst, **sc)
        assert F.lib().filtr_test_set_checkpoint(ctx.handle, 64) == 0
        assert F.lib().filtr_test_force_recompute(ctx.handle, int(recompute)) == 0
        try:
            res, cig, rc = F.align_long(ctx, params, q, r)
        finally:
            F.lib().filtr_test_set_checkpoint(ctx.handle, 0)
            F.lib().filtr_test_force_recompute(ctx.handle, 0)
        assert rc == 0, F.last_error()
        o = oracle.align(q, r, b.subst, **sc)
        for f in ("score", "q_end", "r_end", "status", "cells"):
            assert int(res[f]) == int(o[f]), (kind, f, int(res[f]), int(o[f]))
        assert np.array_equal(cig, o["cigar"])


@pytest.mark.parametrize("X", [None, 6, 40])
@pytest.mark.parametrize("mode", ["global", "local"])
@pytest.mark.parametrize("band", [None, 16])
def test_mid_form(F, ctx, X, mode, band):
    """Table 1's M/I/D recurrence (FILTR_AFFINE_MID) on the antidiagonal sweep,
    with and without an X-drop threshold and a band: bit-exact against the
    oracle's M/I/D form, CIGARs included (unpruned pairs outgrow the first window
    and are rerun wider)."""
    b = mixed_pairs(300 + (X or 0), n=90)
    run_both(F, ctx, b, dict(mode=mode, affine=True, gap_open=4, gap_extend=2, xdrop=X,
                             band=band, mid=True, traceback=True))


@pytest.mark.parametrize("mode", ["global", "local"])
def test_mid_protein(F, ctx, mode):
    """Protein scores with cheap gaps (open 0, extend 1, mismatches down to -4),
    where an insertion next to a deletion beats a mismatch, so the M/I/D and
    H/E/F forms part ways: the GPU follows the M/I/D oracle, with and without the
    running X-drop threshold."""
    P = synth.protein_pairs(n=60, lmin=30, lmax=400, seed=22)
    for extra in (dict(), dict(xdrop=30, xdrop_running=True)):
        sc = dict(mode=mode, affine=True, gap_open=0, gap_extend=1, mid=True, traceback=True,
                  **extra)
        res = run_both(F, ctx, P, sc)
        if not extra:
            plain = res
    hef = oracle_batch(P, dict(mode=mode, affine=True, gap_open=0, gap_extend=1, traceback=False))[0]
    res = plain
    if mode == "global":
        assert (hef["score"] != res["score"].astype(np.int64)).any()
