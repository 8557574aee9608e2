"""GPU parity of Z-drop pruning (Sec. 9.3: a cell is pruned when
best(k-1) - H > Z + |diag - diag_best(k-1)|) against the oracle, bit-exact:
thresholds from 0 to infinity, global and local, linear and affine, with and
without a band and traceback, windows that outgrow their group and are rerun
wider, long reads, and long pairs through the segmented sweep (single pass and
recomputed segments)."""
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


def mixed_pairs(seed, n=100, lmax=500):
    qs, rs = synth.random_pairs(n, lmax, lmax, 4, seed=seed, related=0.7)
    rng = np.random.default_rng(seed)
    for M, N in [(1, 1), (1, 40), (40, 1), (3, 150), (150, 3), (257, 255)]:
        qs.append(rng.integers(0, 4, size=M).astype(np.uint8))
        rs.append(rng.integers(0, 4, size=N).astype(np.uint8))
    # long gaps: a related pair with a 60-base insertion, where the distance
    # term keeps cells X-drop would prune
    r = rng.integers(0, 4, size=400).astype(np.uint8)
    q = np.concatenate([r[:200], rng.integers(0, 4, size=60).astype(np.uint8), r[200:]])
    qs.append(q)
    rs.append(r)
    return synth.pack(qs, rs, 4, DNA_S)


@pytest.mark.parametrize("Z", [0, 5, 20, 60, 400])
@pytest.mark.parametrize("tb", [False, True])
def test_global_affine(F, ctx, Z, tb):
    b = mixed_pairs(200 + Z)
    run_both(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2, zdrop=Z,
                             traceback=tb))


@pytest.mark.parametrize("Z", [2, 30])
@pytest.mark.parametrize("mode", ["global", "local"])
@pytest.mark.parametrize("affine", [False, True])
def test_modes(F, ctx, Z, mode, affine):
    b = mixed_pairs(17 + Z, n=70)
    run_both(F, ctx, b, dict(mode=mode, affine=affine, gap_open=3 if affine else 0, gap_extend=1,
                             zdrop=Z, traceback=True))


@pytest.mark.parametrize("band", [3, 40])
def test_band_and_zdrop(F, ctx, band):
    b = mixed_pairs(61 + band, n=70)
    run_both(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2, zdrop=40,
                             band=band, traceback=True))


def test_protein_zdrop(F, ctx):
    P = synth.protein_pairs(n=50, lmin=30, lmax=500, seed=23)
    run_both(F, ctx, P, dict(mode="global", affine=True, gap_open=11, gap_extend=1, zdrop=40,
                             traceback=True))


def test_window_overflow_rerun(F, ctx):
    """Z = infinity keeps every cell: windows overflow and rerun wider, and the
    result is the unpruned alignment."""
    rng = np.random.default_rng(8)
    qs = [rng.integers(0, 4, size=M).astype(np.uint8) for M in (300, 1500, 2600)]
    rs = [rng.integers(0, 4, size=N).astype(np.uint8) for N in (280, 1400, 2500)]
    b = synth.pack(qs, rs, 4, DNA_S)
    res = run_both(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                   zdrop=oracle.INF, traceback=True))
    full = oracle_batch(b, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                traceback=True))[0]
    assert np.array_equal(res["score"].astype(np.int64), full["score"])


def test_long_reads_zdrop(F, ctx):
    b = synth.long_reads(n=40, lmin=2000, lmax=5000, seed=31)
    sc = dict(b.scoring, xdrop=None, zdrop=400)  # xdrop=None overrides the generator's
    run_both(F, ctx, b, sc)


@pytest.mark.parametrize("recompute", [False, True])
def test_long_pair_segmented(F, ctx, recompute):
    """filtr_align_long over a pair with a 150-base insertion, forced through
    the segmented sweep (checkpoint every 64 antidiagonals)."""
    b = synth.long_pair(length=5000, seg=150, seed=29, xdrop=120)
    q, r = b.pair(0)
    sc = dict(b.scoring, xdrop=None, zdrop=60)
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
        assert int(res[f]) == int(o[f]), (f, int(res[f]), int(o[f]))
    assert (int(res["q_begin"]), int(res["r_begin"])) == (o["q_begin"], o["r_begin"])
    assert np.array_equal(cig, o["cigar"])

