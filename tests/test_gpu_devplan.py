"""GPU checks of the device planner: the same batch planned on the host and on
the device gives identical results and CIGARs, the same shape for every pair
(same int16x2 count) and the same cell estimate; device-planned batches match
the oracle; a batch whose traceback needs several waves falls back to the host
planner; X-drop batches stay on the host."""
import numpy as np
import pytest

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
    c = F.Context(0, 2 << 30)
    yield c
    c.close()


def with_empty(qs, rs, rng, alpha):
    """Add pairs with an empty side at scattered positions."""
    for pos, (M, N) in zip((0, 7, 300, 301), [(0, 40), (35, 0), (0, 0), (1, 1)]):
        pos = min(pos, len(qs))
        qs.insert(pos, rng.integers(0, alpha, size=M).astype(np.uint8))
        rs.insert(pos, rng.integers(0, alpha, size=N).astype(np.uint8))
    return qs, rs


def run_mode(F, ctx, batch, sc, mode):
    F.lib().filtr_test_set_device_plan(ctx.handle, mode)
    try:
        params = F.make_params(batch.subst, **sc)
        ctx.set_timing(True)
        res, cig, rc = F.align_batch(ctx, params, batch)
        assert rc == 0, F.last_error()
        st = ctx.last_stats()
        ctx.set_timing(False)
    finally:
        F.lib().filtr_test_set_device_plan(ctx.handle, 0)
    return res, cig, st


def host_vs_device(F, ctx, batch, sc, expect_device=1):
    r1, c1, s1 = run_mode(F, ctx, batch, sc, 1)
    r2, c2, s2 = run_mode(F, ctx, batch, sc, 2)
    assert s1["device_plan"] == 0
    assert s2["device_plan"] == expect_device, s2
    assert np.array_equal(r1, r2)
    if sc.get("traceback"):
        used = int((r1["cigar_off"] + r1["cigar_len"]).max())
        assert np.array_equal(c1[:used], c2[:used])
    assert s1["pairs_i16x2"] == s2["pairs_i16x2"]
    assert s1["cells_planned"] == s2["cells_planned"]
    return r2, c2, s2


@pytest.mark.parametrize("mode", ["global", "local"])
@pytest.mark.parametrize("tb", [True, False])
def test_protein_host_equals_device(F, ctx, mode, tb):
    b0 = synth.protein_pairs(n=600, lmin=1, lmax=1500, seed=41)
    rng = np.random.default_rng(41)
    qs, rs = with_empty([b0.pair(p)[0] for p in range(b0.n)], [b0.pair(p)[1] for p in range(b0.n)],
                        rng, 20)
    b = synth.pack(qs, rs, 20, b0.subst)
    host_vs_device(F, ctx, b, dict(mode=mode, affine=True, gap_open=11, gap_extend=1, traceback=tb))


@pytest.mark.parametrize("prec", ["I32", "I16X2"])
def test_precision_and_band(F, ctx, prec):
    qs, rs = synth.random_pairs(500, 700, 700, 4, seed=43, related=0.7)
    qs, rs = with_empty(qs, rs, np.random.default_rng(43), 4)
    b = synth.pack(qs, rs, 4, DNA_S)
    p = getattr(F, "PREC_" + prec)
    host_vs_device(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                   traceback=True, precision=p))
    host_vs_device(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                   traceback=True, band=24, precision=p))


def test_device_plan_matches_oracle(F, ctx):
    """Forced device plan on sizes spanning several tile heights, empty sides,
    one-residue pairs: bit-exact against the oracle."""
    qs, rs = synth.random_pairs(300, 1200, 900, 4, seed=44, related=0.6)
    qs, rs = with_empty(qs, rs, np.random.default_rng(44), 4)
    b = synth.pack(qs, rs, 4, DNA_S)
    for sc in (dict(mode="local", affine=True, gap_open=4, gap_extend=2, traceback=True),
               dict(mode="global", affine=False, gap_open=0, gap_extend=3, traceback=True,
                    band=30)):
        res, cig, st = run_mode(F, ctx, b, sc, 2)
        assert st["device_plan"] == 1
        ores, oops, ooff = oracle_batch(b, sc)
        compare(b, sc, res, cig, ores, oops, ooff, label=str(sc))


def test_default_threshold(F, ctx):
    """By default a batch of a few pairs is planned on the host and a batch of
    a few hundred on the device."""
    small = synth.protein_pairs(n=20, lmin=50, lmax=200, seed=45)
    big = synth.protein_pairs(n=400, lmin=50, lmax=200, seed=45)
    for b, want in ((small, 0), (big, 1)):
        params = F.make_params(b.subst, **b.scoring)
        ctx.set_timing(True)
        _, _, rc = F.align_batch(ctx, params, b)
        assert rc == 0, F.last_error()
        assert ctx.last_stats()["device_plan"] == want
        ctx.set_timing(False)


def test_multi_wave_falls_back(F):
    """A workspace too small for one wave of traceback: the device plan's total
    exceeds it and the host planner cuts waves; results equal the host plan in
    a large workspace."""
    b = synth.protein_pairs(n=700, lmin=300, lmax=1000, seed=46)
    sc = dict(b.scoring)
    big = F.Context(0, 2 << 30)
    try:
        r1, c1, s1 = run_mode(F, big, b, sc, 1)
        assert s1["waves"] == 1
    finally:
        big.close()
    small = F.Context(0, 96 << 20)
    try:
        r2, c2, s2 = run_mode(F, small, b, sc, 2)
        assert s2["device_plan"] == 0 and s2["waves"] > 1, s2
    finally:
        small.close()
    assert np.array_equal(r1, r2)
    used = int((r1["cigar_off"] + r1["cigar_len"]).max())
    assert np.array_equal(c1[:used], c2[:used])


def test_xdrop_stays_on_host(F, ctx):
    qs, rs = synth.random_pairs(300, 400, 400, 4, seed=47, related=0.8)
    b = synth.pack(qs, rs, 4, DNA_S)
    _, _, st = run_mode(F, ctx, b, dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                                        xdrop=30, traceback=True), 2)
    assert st["device_plan"] == 0


def test_host_buffers_device_plan(F, ctx):
    """The host-buffer entry point (lengths on the host, validated on the
    device) also plans on the device and gives the device-buffer results."""
    b = synth.protein_pairs(n=500, lmin=20, lmax=900, seed=48)
    params = F.make_params(b.subst, **b.scoring)
    r1, c1, rc = F.align_batch(ctx, params, b)
    assert rc == 0, F.last_error()
    ctx.set_timing(True)
    r2, c2, rc = F.align_batch_host(ctx, params, b)
    assert rc == 0, F.last_error()
    assert ctx.last_stats()["device_plan"] == 1
    ctx.set_timing(False)
    assert np.array_equal(r1, r2)
    used = int((r1["cigar_off"] + r1["cigar_len"]).max())
    assert np.array_equal(c1[:used], c2[:used])
