"""GPU parity of the search traversal (filtr_search_batch, Sec. 6.3) against the
oracle's search: distance, wavefront cells, end coordinates and CIGAR, bit for
bit, exact and with the band and WFA-Adapt options; the edit-distance
workloads of the search-versus-antidiagonal comparison (500 / 2000 / 4000
residues at 1 / 5 / 30% divergence) in full on samples of pairs and on the
batch sizes the benchmark times; cross-checked against the antidiagonal kernels'
unit-cost global score; edge cases (empty sides, identical pairs, a pair across
many score levels), a CIGAR buffer too small, the length limit, and a
workspace small enough to need several traceback waves."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


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


def compare_search(b, res, cig, ores, oops, ooff, tb, idx=None, label=""):
    pairs = range(b.n) if idx is None else idx
    bad = []
    for row, p in enumerate(pairs):
        o = ores[row] if idx is not None else ores[p]
        g = res[p]
        M, N = int(b.q_len[p]), int(b.r_len[p])
        want = dict(score=-int(o["distance"]), cells=int(o["cells"]), q_begin=0, q_end=M,
                    r_begin=0, r_end=N, status=0)
        for f, v in want.items():
            if int(g[f]) != v:
                bad.append((p, f, int(g[f]), v))
        if tb:
            got = cig[int(g["cigar_off"]):int(g["cigar_off"]) + int(g["cigar_len"])]
            oo = int(ooff[row if idx is not None else p])
            exp = oops[oo:oo + int(o["n_ops"])]
            if not np.array_equal(got, exp):
                bad.append((p, "cigar", oracle.cigar_str(got)[:60], oracle.cigar_str(exp)[:60]))
        if len(bad) > 8:
            break
    assert not bad, f"{label}: {len(bad)} mismatches, first: {bad[:8]}"


def run(F, ctx, b, tb=True, band=None, adapt=None, alphabet=0):
    prm = F.make_search_params(traceback=tb, band=band, adapt=adapt, alphabet=alphabet)
    res, cig, rc = F.search_batch(ctx, prm, b)
    assert rc == 0, F.last_error()
    return res, cig


def check(F, ctx, b, tb=True, band=None, adapt=None, label="", alphabet=0):
    res, cig = run(F, ctx, b, tb, band, adapt, alphabet)
    ores, oops, ooff = oracle.search_batch(b, traceback=tb, band=band, adapt=adapt)
    compare_search(b, res, cig, ores, oops, ooff, tb, label=label)
    return res


def with_edges(qs, rs, rng, alpha):
    for pos, (M, N) in zip((0, 5, 17, 40, 41), [(0, 30), (25, 0), (0, 0), (1, 1), (1, 2)]):
        pos = min(pos, len(qs))
        qs.insert(pos, rng.integers(0, alpha, size=M).astype(np.uint8))
        rs.insert(pos, rng.integers(0, alpha, size=N).astype(np.uint8))
    same = rng.integers(0, alpha, size=333).astype(np.uint8)
    qs.append(same)
    rs.append(same.copy())
    return qs, rs


@pytest.mark.parametrize("alpha,packed", [(4, False), (4, True), (20, False)])
@pytest.mark.parametrize("tb", [True, False])
def test_small_exact(F, ctx, alpha, packed, tb):
    qs, rs = synth.random_pairs(300, 300, 300, alpha, seed=61 + alpha, related=0.7)
    qs, rs = with_edges(qs, rs, np.random.default_rng(61), alpha)
    b = synth.pack(qs, rs, alpha, np.zeros((alpha, alpha), np.int8))
    check(F, ctx, b, tb=tb, label=f"alpha {alpha} tb {tb}", alphabet=4 if packed else 0)


def test_packed_rejects_codes(F, ctx):
    """Alphabet 4 checks every code: a 4 anywhere fails the call before the search."""
    qs, rs = synth.random_pairs(20, 50, 50, 4, seed=69)
    rs[7] = rs[7].copy()
    rs[7][3] = 4
    b = synth.pack(qs, rs, 5, np.zeros((5, 5), np.int8))
    prm = F.make_search_params(traceback=False, alphabet=4)
    _, _, rc = F.search_batch(ctx, prm, b, raise_on_error=False)
    assert rc == F.ERR_INVALID
    _, _, rc = F.search_batch(ctx, F.make_search_params(traceback=False), b)
    assert rc == 0


@pytest.mark.parametrize("band", [0, 5, 40])
def test_band(F, ctx, band):
    qs, rs = synth.random_pairs(200, 250, 250, 4, seed=62, related=0.8)
    qs, rs = with_edges(qs, rs, np.random.default_rng(62), 4)
    b = synth.pack(qs, rs, 4, np.zeros((4, 4), np.int8))
    check(F, ctx, b, band=band, label=f"band {band}")


@pytest.mark.parametrize("adapt", [(1, 0), (10, 5), (64, 50)])
def test_adapt(F, ctx, adapt):
    qs, rs = synth.random_pairs(200, 400, 400, 4, seed=63, related=0.9)
    qs, rs = with_edges(qs, rs, np.random.default_rng(63), 4)
    b = synth.pack(qs, rs, 4, np.zeros((4, 4), np.int8))
    check(F, ctx, b, adapt=adapt, label=f"adapt {adapt}")


@pytest.mark.parametrize("length", [500, 2000, 4000])
@pytest.mark.parametrize("div", [0.01, 0.05, 0.30])
def test_table_workloads(F, ctx, length, div):
    """Full-length pairs of each cell of the comparison table, traceback on, all
    pairs against the oracle; the score-only run agrees; the antidiagonal
    kernels' unit-cost global score is minus the same distance."""
    b = synth.edit_pairs(48, length, div, seed=64)
    res = check(F, ctx, b, tb=True, label=f"{length} {div}", alphabet=4)
    for alphabet in (0, 4):
        res0, _ = run(F, ctx, b, tb=False, alphabet=alphabet)
        assert np.array_equal(res0["score"], res["score"])
        assert np.array_equal(res0["cells"], res["cells"])
    params = F.make_params(b.subst, **b.scoring)
    ares, _, rc = F.align_batch(ctx, params, b)
    assert rc == 0, F.last_error()
    assert np.array_equal(ares["score"], res["score"])


@pytest.mark.parametrize("length,div,n", [(500, 0.05, 20000), (4000, 0.30, 2000)])
def test_bench_batches_sampled(F, ctx, length, div, n):
    """The batch sizes the benchmark times, sampled pairs against the oracle."""
    b = synth.edit_pairs(n, length, div, seed=6)
    res, _ = run(F, ctx, b, tb=False, alphabet=4)
    idx = np.random.default_rng(65).choice(b.n, size=40, replace=False)
    sub = synth.pack([b.pair(int(p))[0] for p in idx], [b.pair(int(p))[1] for p in idx], 4,
                     b.subst)
    ores, _, _ = oracle.search_batch(sub, traceback=False)
    compare_search(b, res, None, ores, None, None, False, idx=idx, label="sampled")


def test_long_pair_many_levels(F, ctx):
    rng = np.random.default_rng(66)
    r = rng.integers(0, 4, size=9000).astype(np.uint8)
    q = synth.mutate(rng, r, 0.004, 0.003, 0.003, None)
    u = rng.integers(0, 4, size=1500).astype(np.uint8)  # two unrelated sequences too
    v = rng.integers(0, 4, size=1400).astype(np.uint8)
    b = synth.pack([q, u], [r, v], 4, np.zeros((4, 4), np.int8))
    check(F, ctx, b, label="long")


def test_cigar_cap(F, ctx):
    qs, rs = synth.random_pairs(50, 100, 100, 4, seed=67, related=0.5)
    b = synth.pack(qs, rs, 4, np.zeros((4, 4), np.int8))
    full, _ = run(F, ctx, b)
    prm = F.make_search_params(traceback=True)
    res, _, rc = F.search_batch(ctx, prm, b, cigar_cap=10, raise_on_error=False)
    assert rc == F.ERR_CIGAR_CAP
    assert np.array_equal(res["cigar_len"], full["cigar_len"])
    assert np.array_equal(res["score"], full["score"])


def test_length_limit(F, ctx):
    big = np.zeros(100_000, np.uint8)
    b = synth.pack([big], [big.copy()], 4, np.zeros((4, 4), np.int8))
    prm = F.make_search_params(traceback=False)
    _, _, rc = F.search_batch(ctx, prm, b, raise_on_error=False)
    assert rc == F.ERR_UNSUPPORTED


def test_traceback_waves(F):
    """A workspace that holds a few pairs' wavefronts at a time: several
    traceback waves, same results as one."""
    b = synth.edit_pairs(60, 2000, 0.30, seed=68)  # about 1.1 MB of wavefronts per pair
    small = F.Context(0, 40 << 20)
    try:
        prm = F.make_search_params(traceback=True)
        res, cig, rc = F.search_batch(small, prm, b)
        assert rc == 0, F.last_error()
        assert small.last_stats()["waves"] > 1
    finally:
        small.close()
    ores, oops, ooff = oracle.search_batch(b)
    compare_search(b, res, cig, ores, oops, ooff, True, label="waves")
