"""GPU checks of the captured batch pipeline (filtr_graph_*): results equal to
filtr_align_batch and to the oracle, one graph replayed over batches of
different sizes, and the checks that run inside the graph (bad residues,
lengths over the bound, traceback over the budget, CIGAR capacity) reported by
filtr_graph_status without disturbing the next launch."""
import re

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


def same(F, ctx, g, params, b):
    r1, c1, rc = F.align_batch(ctx, params, b)
    assert rc == 0, F.last_error()
    r2, c2, st = F.graph_align(g, b)
    assert st == 0, F.last_error()
    assert np.array_equal(r1, r2)
    if params.traceback:
        used = int((r1["cigar_off"] + r1["cigar_len"]).max()) if b.n else 0
        assert np.array_equal(c1[:used], c2[:used])
    return r2, c2


def with_empty(b, alpha, seed):
    rng = np.random.default_rng(seed)
    qs = [b.pair(p)[0] for p in range(b.n)]
    rs = [b.pair(p)[1] for p in range(b.n)]
    for pos, (M, N) in zip((0, 5, 40), [(0, 30), (25, 0), (0, 0)]):
        qs.insert(pos, rng.integers(0, alpha, size=M).astype(np.uint8))
        rs.insert(pos, rng.integers(0, alpha, size=N).astype(np.uint8))
    return synth.pack(qs, rs, alpha, b.subst)


def test_protein_replays(F, ctx):
    """One graph, several batches of different sizes and contents."""
    b0 = synth.protein_pairs(n=10, seed=61)
    params = F.make_params(b0.subst, **b0.scoring)
    g = F.Graph(ctx, params, max_pairs=700, max_len=1300, workspace_bytes=1 << 30)
    try:
        for n, seed in ((600, 62), (37, 63), (700, 64), (1, 65)):
            b = synth.protein_pairs(n=n, lmin=1, lmax=1200, seed=seed)
            if n > 3:
                b = synth.pack([b.pair(p)[0] for p in range(b.n - 3)],
                               [b.pair(p)[1] for p in range(b.n - 3)], 20, b0.subst)
                b = with_empty(b, 20, seed)
            same(F, ctx, g, params, b)
    finally:
        g.close()


@pytest.mark.parametrize("kind", ["global_notb", "band", "i32", "linear_local"])
def test_kinds(F, ctx, kind):
    qs, rs = synth.random_pairs(300, 900, 900, 4, seed=66, related=0.7)
    b = with_empty(synth.pack(qs, rs, 4, DNA_S), 4, 66)
    sc = {"global_notb": dict(mode="global", affine=True, gap_open=4, gap_extend=2, traceback=False),
          "band": dict(mode="global", affine=True, gap_open=4, gap_extend=2, traceback=True, band=40),
          "i32": dict(mode="local", affine=True, gap_open=4, gap_extend=2, traceback=True,
                      precision=F.PREC_I32),
          "linear_local": dict(mode="local", affine=False, gap_open=0, gap_extend=3,
                               traceback=True)}[kind]
    params = F.make_params(b.subst, **sc)
    g = F.Graph(ctx, params, max_pairs=b.n, max_len=900, workspace_bytes=1 << 30)
    try:
        res, cig = same(F, ctx, g, params, b)
    finally:
        g.close()
    ores, oops, ooff = oracle_batch(b, {k: v for k, v in sc.items() if k != "precision"})
    compare(b, sc, res, cig, ores, oops, ooff, label=kind)


def test_deferred_errors(F, ctx):
    b = synth.protein_pairs(n=200, lmin=50, lmax=400, seed=67)
    params = F.make_params(b.subst, **b.scoring)
    g = F.Graph(ctx, params, max_pairs=300, max_len=400, workspace_bytes=1 << 28)
    try:
        same(F, ctx, g, params, b)
        # a residue code >= 20
        bad = synth.pack([b.pair(p)[0] for p in range(b.n)], [b.pair(p)[1] for p in range(b.n)],
                         20, b.subst)
        bad.q_seq[5] = 25
        _, _, st = F.graph_align(g, bad)
        assert st == F.ERR_INVALID
        # a sequence longer than max_len
        qs = [b.pair(p)[0] for p in range(b.n)]
        rs = [b.pair(p)[1] for p in range(b.n)]
        qs[3] = np.concatenate([qs[3], qs[3]])[:401]
        _, _, st = F.graph_align(g, synth.pack(qs, rs, 20, b.subst))
        assert st == F.ERR_INVALID
        # CIGAR capacity too small: results still right, status CIGAR_CAP
        r_ok, _, _ = F.align_batch(ctx, params, b)
        res, _, st = F.graph_align(g, b, cigar_cap=100)
        assert st == F.ERR_CIGAR_CAP
        for f in ("score", "q_end", "r_end", "status", "cigar_len"):
            assert np.array_equal(res[f], r_ok[f]), f
        # and the next launch is clean
        same(F, ctx, g, params, b)
        with pytest.raises(F.FiltrError):
            F.graph_align(g, synth.protein_pairs(n=301, lmin=50, lmax=60, seed=68))
    finally:
        g.close()


def test_traceback_budget(F, ctx):
    """A workspace whose traceback area holds a small batch but not a large one."""
    small = synth.protein_pairs(n=20, lmin=100, lmax=300, seed=69)
    big = synth.protein_pairs(n=400, lmin=300, lmax=400, seed=70)
    params = F.make_params(small.subst, **small.scoring)
    # the fixed parts depend on the device's occupancy: read them from the
    # refusal, then leave ~24 MB of traceback area (400 pairs of ~350^2 cells
    # need ~42 MB, 20 pairs of ~200^2 about 1 MB)
    with pytest.raises(F.FiltrError) as ei:
        F.Graph(ctx, params, max_pairs=400, max_len=450, workspace_bytes=1 << 20)
    fixed = int(re.search(r"need (\d+)", str(ei.value)).group(1))
    g = F.Graph(ctx, params, max_pairs=400, max_len=450, workspace_bytes=fixed + (24 << 20))
    try:
        same(F, ctx, g, params, small)
        _, _, st = F.graph_align(g, big)
        assert st == F.ERR_NOMEM
        same(F, ctx, g, params, small)
    finally:
        g.close()


def test_create_rejects(F, ctx):
    S = DNA_S
    with pytest.raises(F.FiltrError):
        F.Graph(ctx, F.make_params(S, xdrop=20), 10, 100, 1 << 26)
    with pytest.raises(F.FiltrError):
        F.Graph(ctx, F.make_params(S), 10, 100, 1 << 10)  # below the fixed parts
    with pytest.raises(F.FiltrError):
        F.Graph(ctx, F.make_params(S), 0, 100, 1 << 26)
