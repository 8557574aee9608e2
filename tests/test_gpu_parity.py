"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by
element, bit-exact (integer scores, coordinates, status, cell counts, CIGARs).

Sizes span several strips of the tiled kernel (256 / 512 rows) with ragged
tails; edge cases cover empty and one-residue sequences, M >> N, N >> M,
identical and all-mismatch pairs, strip boundaries +-1, bands wider than the
matrix and the literal band that misses the corner."""
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


def run_both(F, ctx, batch, sc, plain=False):
    params = F.make_params(batch.subst, **sc)
    res, cig, rc = F.align_batch(ctx, params, batch, plain=plain)
    assert rc == 0, F.last_error()
    ores, oops, ooff = oracle_batch(batch, sc)
    compare(batch, sc, res, cig, ores, oops, ooff, label=str(sc))
    return res, cig


def edge_pairs(alpha, rng):
    qs, rs = [], []
    spec = [(0, 0), (0, 5), (5, 0), (1, 1), (1, 40), (40, 1), (300, 7), (7, 300), (255, 255),
            (256, 256), (257, 257), (511, 300), (512, 90), (513, 513), (1030, 60), (60, 1030)]
    for M, N in spec:
        qs.append(rng.integers(0, alpha, size=M).astype(np.uint8))
        rs.append(rng.integers(0, alpha, size=N).astype(np.uint8))
    same = rng.integers(0, alpha, size=200).astype(np.uint8)
    qs.append(same)
    rs.append(same.copy())
    a = np.zeros(150, np.uint8)
    qs.append(a)
    rs.append(np.full(170, 1, np.uint8))  # all mismatches
    return qs, rs


MODES = [
    dict(mode="global", affine=True, gap_open=4, gap_extend=2),
    dict(mode="local", affine=True, gap_open=4, gap_extend=2),
    dict(mode="global", affine=False, gap_extend=3),
    dict(mode="local", affine=False, gap_extend=1),
]


@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("sc", MODES, ids=lambda s: f"{s['mode']}-{'aff' if s['affine'] else 'lin'}")
def test_dna_random_and_edges(F, ctx, sc, tb):
    rng = np.random.default_rng(101)
    qs, rs = synth.random_pairs(120, 700, 700, 4, seed=5)
    eq, er = edge_pairs(4, rng)
    batch = synth.pack(qs + eq, rs + er, 4, DNA_S)
    run_both(F, ctx, batch, dict(sc, traceback=tb))


@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("mode", ["global", "local"])
def test_protein(F, ctx, mode, tb):
    P = synth.protein_subst(np.random.default_rng(2))
    qs, rs = synth.random_pairs(150, 900, 900, 20, seed=7, mmin=1, nmin=1)
    eq, er = edge_pairs(20, np.random.default_rng(3))
    batch = synth.pack(qs + eq, rs + er, 20, P)
    run_both(F, ctx, batch, dict(mode=mode, affine=True, gap_open=11, gap_extend=1, traceback=tb))


@pytest.mark.parametrize("literal", [False, True])
@pytest.mark.parametrize("B", [0, 3, 40, 5000])
@pytest.mark.parametrize("mode", ["global", "local"])
def test_band(F, ctx, mode, B, literal):
    qs, rs = synth.random_pairs(80, 800, 800, 4, seed=11 + B)
    eq, er = edge_pairs(4, np.random.default_rng(B))
    batch = synth.pack(qs + eq, rs + er, 4, DNA_S)
    run_both(F, ctx, batch, dict(mode=mode, affine=True, gap_open=4, gap_extend=2, band=B,
                                  band_literal=literal, traceback=True))


def test_short_dna_workload_full(F, ctx):
    """The 1000-pair short-read workload at its full size (score only)."""
    b = synth.short_dna_pairs()
    run_both(F, ctx, b, dict(b.scoring))
    run_both(F, ctx, b, dict(b.scoring, traceback=True))


def test_plain_equals_batched(F, ctx):
    P = synth.protein_pairs(n=60, lmin=50, lmax=600, seed=9)
    sc = dict(P.scoring)
    params = F.make_params(P.subst, **sc)
    a, ca, _ = F.align_batch(ctx, params, P)
    b, cb, _ = F.align_batch(ctx, params, P, plain=True)
    assert np.array_equal(a, b)
    assert np.array_equal(ca[: int(a["cigar_off"][-1] + a["cigar_len"][-1])],
                          cb[: int(b["cigar_off"][-1] + b["cigar_len"][-1])])


def test_host_entry_point(F, ctx):
    P = synth.protein_pairs(n=40, lmin=10, lmax=400, seed=12)
    params = F.make_params(P.subst, **P.scoring)
    a, ca, _ = F.align_batch(ctx, params, P)
    h, ch, rc = F.align_batch_host(ctx, params, P)
    assert rc == 0
    assert np.array_equal(a, h)
    tot = int(a["cigar_off"][-1] + a["cigar_len"][-1])
    assert np.array_equal(ca[:tot], ch[:tot])


def test_cigar_cap_too_small(F, ctx):
    b = synth.short_dna_pairs(n=30, seed=4)
    params = F.make_params(b.subst, **dict(b.scoring, traceback=True))
    res, cig, rc = F.align_batch(ctx, params, b, cigar_cap=10, raise_on_error=False)
    assert rc == F.ERR_CIGAR_CAP
    ores, _, _ = oracle_batch(b, dict(b.scoring, traceback=True))
    assert np.array_equal(res["cigar_len"].astype(np.int64), ores["n_ops"])


def test_invalid_codes_rejected(F, ctx):
    b = synth.short_dna_pairs(n=5, seed=4)
    b.q_seq = b.q_seq.copy()
    b.q_seq[3] = 9
    params = F.make_params(b.subst, **b.scoring)
    with pytest.raises(F.FiltrError) as ei:
        F.align_batch(ctx, params, b)
    assert ei.value.code == F.ERR_INVALID


def test_protein_workload_sampled(F, ctx):
    """The 100,000-pair protein workload at full size in the benchmark's launch
    configuration; 400 sampled pairs are checked one by one against the oracle
    and every CIGAR is checked for consistency with its coordinates."""
    P = synth.protein_pairs()
    sc = dict(P.scoring)
    params = F.make_params(P.subst, **sc)
    res, cig, rc = F.align_batch(ctx, params, P)
    assert rc == 0
    idx = np.random.default_rng(0).choice(P.n, size=400, replace=False)
    sub = P.subset(idx)
    ores, oops, ooff = oracle_batch(sub, sc)
    compare(P, sc, res, cig, ores, oops, ooff, idx=list(idx), label="protein-100k")
    # consumed lengths of every CIGAR equal the reported spans
    ops = cig[: int(res["cigar_off"][-1] + res["cigar_len"][-1])]
    ln, op = ops >> 4, ops & 15
    consq = np.where((op == 7) | (op == 8) | (op == 1), ln, 0).astype(np.int64)
    consr = np.where((op == 7) | (op == 8) | (op == 2), ln, 0).astype(np.int64)
    starts = res["cigar_off"].astype(np.int64)
    cq = np.add.reduceat(consq, starts[res["cigar_len"] > 0]) if len(ops) else np.zeros(0)
    cr = np.add.reduceat(consr, starts[res["cigar_len"] > 0]) if len(ops) else np.zeros(0)
    nz = res[res["cigar_len"] > 0]
    assert np.array_equal(cq, (nz["q_end"] - nz["q_begin"]).astype(np.int64))
    assert np.array_equal(cr, (nz["r_end"] - nz["r_begin"]).astype(np.int64))
    assert int(res["cells"].sum()) == P.cells_full()
