"""GPU parity of the int16x2 tiled kernel (two 16-bit cells per register)
against the oracle, bit-exact, and against the int32 kernel on the same pairs.

precision=I16X2 sends every pair whose score range fits 15 bits to the packed
kernel; the stats report how many did.  Sizes cover the packed staircase's
edge-only strips (N < 64: every step masked), one and several strips of
512 and 1024 rows with ragged tails, rows past M in either half of a lane's
registers, one-residue sequences, and pairs whose bound does not fit (they run
in int32 and give identical results).  Also the residue packer (filtr_pack,
16 codes per vector load) against a host packer."""
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
    c = F.Context(0, 4 << 30)
    yield c
    c.close()


def sized_pairs(alpha, seed):
    rng = np.random.default_rng(seed)
    spec = [(1, 1), (1, 70), (70, 1), (2, 63), (9, 62), (16, 64), (17, 65), (40, 200),
            (200, 40), (255, 130), (257, 300), (300, 257), (511, 100), (512, 512), (513, 77),
            (520, 600), (1023, 90), (1024, 1024), (1025, 333), (1500, 1400), (2100, 700)]
    qs, rs = [], []
    for M, N in spec:
        r = rng.integers(0, alpha, size=N).astype(np.uint8)
        q = rng.integers(0, alpha, size=M).astype(np.uint8)
        # make about half of the pairs related so that alignments carry gaps
        if rng.random() < 0.5:
            L = min(M, N)
            keep = rng.random(L) < 0.8
            q[:L] = np.where(keep, r[:L], q[:L])
        qs.append(q)
        rs.append(r)
    return qs, rs


def run_checked(F, ctx, batch, sc, expect_packed=None):
    params = F.make_params(batch.subst, **sc)
    ctx.set_timing(True)
    res, cig, rc = F.align_batch(ctx, params, batch)
    assert rc == 0, F.last_error()
    st = ctx.last_stats()
    ctx.set_timing(False)
    ores, oops, ooff = oracle_batch(batch, {k: v for k, v in sc.items() if k != "precision"})
    compare(batch, sc, res, cig, ores, oops, ooff, label=str(sc))
    if expect_packed is not None:
        assert st["pairs_i16x2"] == expect_packed, st
    return res, cig, st


@pytest.mark.parametrize("mode", ["global", "local"])
@pytest.mark.parametrize("affine", [True, False])
@pytest.mark.parametrize("tb", [True, False])
def test_dna_sizes(F, ctx, mode, affine, tb):
    qs, rs = sized_pairs(4, 11)
    b = synth.pack(qs, rs, 4, DNA_S)
    sc = dict(mode=mode, affine=affine, gap_open=4 if affine else 0, gap_extend=2, traceback=tb,
              precision=F.PREC_I16X2)
    run_checked(F, ctx, b, sc, expect_packed=b.n)


@pytest.mark.parametrize("mode", ["global", "local"])
def test_protein_sizes(F, ctx, mode):
    qs, rs = sized_pairs(20, 12)
    P = synth.protein_pairs(n=2, seed=3)
    b = synth.pack(qs, rs, 20, P.subst)
    sc = dict(mode=mode, affine=True, gap_open=11, gap_extend=1, traceback=True,
              precision=F.PREC_I16X2)
    run_checked(F, ctx, b, sc, expect_packed=b.n)


def test_protein_workload_sample(F, ctx):
    """The protein workload's generator (related pairs, indels), local affine
    with traceback: packed and int32 give the oracle's results."""
    b = synth.protein_pairs(n=300, lmin=100, lmax=1000, seed=2)
    sc = dict(b.scoring, precision=F.PREC_I16X2)
    run_checked(F, ctx, b, sc, expect_packed=b.n)
    sc32 = dict(b.scoring, precision=F.PREC_I32)
    run_checked(F, ctx, b, sc32, expect_packed=0)


def test_auto_matches_int32(F, ctx):
    b = synth.protein_pairs(n=200, lmin=20, lmax=1300, seed=8)
    outs = []
    for prec in (F.PREC_AUTO, F.PREC_I32, F.PREC_I16X2):
        params = F.make_params(b.subst, **dict(b.scoring, precision=prec))
        res, cig, rc = F.align_batch(ctx, params, b)
        assert rc == 0, F.last_error()
        used = int((res["cigar_off"] + res["cigar_len"]).max())
        outs.append((res, cig[:used].copy()))
    for res, cig in outs[1:]:
        assert np.array_equal(res, outs[0][0])
        assert np.array_equal(cig, outs[0][1])


def test_out_of_range_runs_int32(F, ctx):
    """Pairs whose 16-bit bound does not hold (scores beyond [-64, 63], or a
    global alignment whose gap costs reach 2^15) are kept in int32 even under
    precision=I16X2, with the oracle's results."""
    rng = np.random.default_rng(4)
    big = np.array([[90, -70], [-70, 90]], dtype=np.int8)
    qs = [rng.integers(0, 2, size=n).astype(np.uint8) for n in (50, 300)]
    rs = [rng.integers(0, 2, size=n).astype(np.uint8) for n in (60, 280)]
    b = synth.pack(qs, rs, 4, np.pad(big, ((0, 2), (0, 2))))
    sc = dict(mode="local", affine=True, gap_open=5, gap_extend=3, traceback=True,
              precision=F.PREC_I16X2)
    run_checked(F, ctx, b, sc, expect_packed=0)
    q = rng.integers(0, 4, size=3000).astype(np.uint8)
    r = rng.integers(0, 4, size=3100).astype(np.uint8)
    b2 = synth.pack([q, q[:100]], [r, r[:120]], 4, DNA_S)
    sc2 = dict(mode="global", affine=True, gap_open=20, gap_extend=5, traceback=True,
               precision=F.PREC_I16X2)
    run_checked(F, ctx, b2, sc2, expect_packed=1)


def test_plain_equals_batched(F, ctx):
    b = synth.protein_pairs(n=40, lmin=30, lmax=900, seed=15)
    params = F.make_params(b.subst, **dict(b.scoring, precision=F.PREC_I16X2))
    r1, c1, _ = F.align_batch(ctx, params, b)
    r2, c2, _ = F.align_batch(ctx, params, b, plain=True)
    assert np.array_equal(r1, r2)
    used = int((r1["cigar_off"] + r1["cigar_len"]).max())
    assert np.array_equal(c1[:used], c2[:used])


def test_autotune_keeps_results(F):
    """filtr_autotune times every allowed shape and only changes which shape a
    pair runs in: results before and after tuning are identical."""
    c = F.Context(0, 2 << 30)
    try:
        b = synth.protein_pairs(n=150, lmin=40, lmax=1100, seed=21)
        params = F.make_params(b.subst, **b.scoring)
        r0, c0, rc = F.align_batch(c, params, b)
        assert rc == 0, F.last_error()
        table = c.autotune(params)
        assert {"i32 R=32", "i32 R=24", "i32 R=16", "i32 R=8"} | {
            f"i16x2 R={R}" for R in (32, 28, 24, 20, 16, 12, 8)} <= set(table)
        assert all(v > 0 for v in table.values())
        r1, c1, rc = F.align_batch(c, params, b)
        assert rc == 0, F.last_error()
        assert np.array_equal(r0, r1)
        used = int((r0["cigar_off"] + r0["cigar_len"]).max())
        assert np.array_equal(c0[:used], c1[:used])
    finally:
        c.close()


def test_tune_apply_reproduces_plan(F):
    """A table saved from filtr_autotune, installed with filtr_tune_apply in a
    fresh context, plans the same shapes (same packed count); a table that
    prices the packed tile out sends no pair to it; results never change."""
    b = synth.protein_pairs(n=120, lmin=40, lmax=1100, seed=27)
    params = F.make_params(b.subst, **b.scoring)
    c1 = F.Context(0, 2 << 30)
    try:
        table = c1.autotune(params)
        c1.set_timing(True)
        r1, g1, rc = F.align_batch(c1, params, b)
        assert rc == 0, F.last_error()
        n1 = c1.last_stats()["pairs_i16x2"]
    finally:
        c1.close()
    c2 = F.Context(0, 2 << 30)
    try:
        c2.tune_apply(params, table)
        c2.set_timing(True)
        r2, g2, rc = F.align_batch(c2, params, b)
        assert rc == 0, F.last_error()
        assert c2.last_stats()["pairs_i16x2"] == n1
        assert np.array_equal(r1, r2)
        used = int((r1["cigar_off"] + r1["cigar_len"]).max())
        assert np.array_equal(g1[:used], g2[:used])
        dear = {k: (v * 100 if k.startswith("i16x2") else v) for k, v in table.items()}
        c2.tune_apply(params, dear)
        r3, g3, rc = F.align_batch(c2, params, b)
        assert rc == 0, F.last_error()
        assert c2.last_stats()["pairs_i16x2"] == 0
        assert np.array_equal(r1, r3)
        assert np.array_equal(g1[:used], g3[:used])
        with pytest.raises(F.FiltrError):
            c2.tune_apply(params, {"i32 R=32": -1.0})
    finally:
        c2.close()


@pytest.mark.parametrize("R", list(range(8, 33, 2)))
@pytest.mark.parametrize("mode", ["global", "local"])
def test_each_packed_height(F, R, mode):
    """Every packed tile height, forced by a tune table that prices the other
    shapes out: bit-exact against the oracle over sizes that span several
    strips of that height, ragged tails and one-residue pairs."""
    c = F.Context(0, 2 << 30)
    try:
        qs, rs = sized_pairs(4, 50 + R)
        b = synth.pack(qs, rs, 4, DNA_S)
        sc = dict(mode=mode, affine=True, gap_open=4, gap_extend=2, traceback=True)
        params = F.make_params(b.subst, **sc)
        table = {f"{kind} R={r}": 1000.0 for kind, r in F.TUNE_SHAPES}
        table[f"i16x2 R={R}"] = 0.001
        c.tune_apply(params, table)
        run_checked(F, c, b, sc, expect_packed=b.n)
    finally:
        c.close()


@pytest.mark.parametrize("alphabet", [4, 20])
@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 1000, 65536 + 7])
def test_filtr_pack_against_host_packer(F, alphabet, n):
    """filtr_pack (one 16-byte load per thread) against a numpy packer: DNA two
    bits per code (code t at bits 2*(t % 16) of word t / 16), protein one byte
    per code; codes >= alphabet are counted (and packed by their low bits)."""
    import ctypes as C

    import torch

    rng = np.random.default_rng(n + alphabet)
    codes = rng.integers(0, alphabet, size=n).astype(np.uint8)
    bad_at = rng.choice(n, size=min(n, 5), replace=False) if n else []
    for t in bad_at:
        codes[t] = alphabet + int(rng.integers(0, 50))
    bits, per = (2, 16) if alphabet == 4 else (8, 4)
    words = (n * bits + 31) // 32
    want = np.zeros(max(words, 1), dtype=np.uint64)
    for t in range(n):
        want[t // per] |= (int(codes[t]) & ((1 << bits) - 1)) << (bits * (t % per))
    d_codes = torch.from_numpy(codes if n else np.zeros(1, np.uint8)).cuda()
    d_packed = torch.zeros(max(words, 1), dtype=torch.int32, device="cuda")
    d_bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = F.lib().filtr_pack(C.c_void_p(d_codes.data_ptr()), n, alphabet, C.c_void_p(d_packed.data_ptr()),
                            C.c_void_p(d_bad.data_ptr()), None)
    torch.cuda.synchronize()
    assert rc == 0, F.last_error()
    got = d_packed.cpu().numpy().view(np.uint32).astype(np.uint64)
    assert np.array_equal(got[:words], want[:words])
    assert int(d_bad.item()) == len(bad_at)


def test_filtr_pack_rejects_misaligned_codes(F):
    import ctypes as C

    import torch

    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.int32, device="cuda")
    bad = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = F.lib().filtr_pack(C.c_void_p(d.data_ptr() + 1), 32, 4, C.c_void_p(out.data_ptr()),
                            C.c_void_p(bad.data_ptr()), None)
    assert rc == F.ERR_INVALID
