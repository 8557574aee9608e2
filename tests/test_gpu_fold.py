"""GPU parity of the folding kernel (filtr_fold_batch: Nussinov, Table 1, with
the X-drop transfer of Sec. 9.5) against the oracle: score, end cell, status,
cells and the fold, bit for bit, unpruned and under several thresholds and
warm-ups, on random and structured RNAs of 0 to 500 bases (Sec. 9.5's range),
plus several table waves in a small workspace and the argument checks."""
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
    c = F.Context(0, 2 << 30)
    yield c
    c.close()


def check(F, ctx, seq, off, lens, label, **kw):
    res, part, rc = F.fold_batch(ctx, F.make_fold_params(**kw), seq, off, lens)
    assert rc == 0, F.last_error()
    ores, opart = oracle.fold_batch(seq, off, lens, **kw)
    bad = []
    for p in range(len(lens)):
        for f in ("score", "i_end", "j_end", "status", "cells"):
            if int(res[p][f]) != int(ores[p][f]):
                bad.append((p, f, int(res[p][f]), int(ores[p][f])))
        a, n = int(off[p]), int(lens[p])
        if kw.get("traceback", True) and not np.array_equal(part[a:a + n], opart[a:a + n]):
            bad.append((p, "fold"))
        if len(bad) > 8:
            break
    assert not bad, f"{label}: {bad[:8]}"
    return res


def random_rna(n, lmax, seed):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, lmax + 1, size=n).astype(np.uint32)
    lens[:4] = [0, 1, 2, 5]
    off = np.zeros(n, np.uint64)
    off[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    return rng.integers(0, 4, size=int(lens.sum())).astype(np.uint8), off, lens


@pytest.mark.parametrize("min_loop", [0, 3])
@pytest.mark.parametrize("cfg", [None, (0, 0), (2, 15), (5, 5)])
def test_random(F, ctx, min_loop, cfg):
    seq, off, lens = random_rna(150, 120, 71 + min_loop)
    kw = dict(min_loop=min_loop)
    if cfg:
        kw.update(xdrop=cfg[0], warmup=cfg[1])
    check(F, ctx, seq, off, lens, str(kw), **kw)


@pytest.mark.parametrize("length", [76, 120, 300, 500])
def test_structured(F, ctx, length):
    """Sec. 9.5's lengths on structured RNAs: unpruned and X = 2, 8 with the
    15-span warm-up; the pruned folds never have more pairs."""
    seq, off, lens = synth.rna_structured(24, length, seed=72)
    base = check(F, ctx, seq, off, lens, "unpruned")
    for X in (2, 8):
        res = check(F, ctx, seq, off, lens, f"X {X}", xdrop=X, warmup=15)
        assert (res["score"] <= base["score"]).all()


def test_score_only(F, ctx):
    seq, off, lens = synth.rna_structured(16, 200, seed=73)
    check(F, ctx, seq, off, lens, "score only", traceback=False, xdrop=3)


def test_rejects(F, ctx):
    seq = np.array([0, 1, 4, 2], np.uint8)
    off = np.zeros(1, np.uint64)
    lens = np.array([4], np.uint32)
    _, _, rc = F.fold_batch(ctx, F.make_fold_params(), seq, off, lens, raise_on_error=False)
    assert rc == F.ERR_INVALID
    big = np.zeros(5000, np.uint8)
    _, _, rc = F.fold_batch(ctx, F.make_fold_params(), big, off, np.array([5000], np.uint32),
                            raise_on_error=False)
    assert rc == F.ERR_UNSUPPORTED


def test_table_waves(F):
    """A workspace that holds a few hundred 300-base triangles at a time: the
    call runs in several waves with the same results as one."""
    seq, off, lens = synth.rna_structured(600, 300, seed=74)
    small = F.Context(0, 40 << 20)  # about 0.18 MB of table per sequence
    try:
        res, part, rc = F.fold_batch(small, F.make_fold_params(xdrop=2), seq, off, lens)
        assert rc == 0, F.last_error()
        assert small.last_stats()["waves"] > 1
    finally:
        small.close()
    ores, opart = oracle.fold_batch(seq, off, lens, xdrop=2)
    assert np.array_equal(res["score"].astype(np.int64), ores["score"])
    assert np.array_equal(res["cells"].astype(np.int64), ores["cells"])
    assert np.array_equal(part, opart[: len(seq)])
