"""Pins for the folding oracle (oracle/fold.c: Nussinov, Table 1, with the X-drop
transfer of Sec. 9.5): checks against what the mathematics fixes.

  * the score equals the largest pair count over every secondary structure
    (explicit enumeration, n <= 10) for min_loop 0..3;
  * the reported fold is a valid secondary structure with exactly that many
    pairs;
  * unpruned runs evaluate the whole triangle, n(n+1)/2 cells;
  * X = infinity, or a warm-up covering every span, reproduces the unpruned
    run; a pruned run never reports more pairs nor more cells;
  * hand-worked cases (tests/golden/fold_hand_worked.json).
The X-drop transfer's domain and DROPPED end are readings the paper does not fix.
"""
import json
import os

import numpy as np
import pytest

import oracle
from pins import brute_fold, check_structure

HERE = os.path.dirname(os.path.abspath(__file__))
CODE = {"A": 0, "C": 1, "G": 2, "U": 3}


def structure(partner):
    return "".join("(" if p > i else (")" if p >= 0 else ".") for i, p in enumerate(partner))


@pytest.mark.parametrize("min_loop", [0, 1, 3])
def test_brute_force(min_loop, oracle_lib):
    rng = np.random.default_rng(51 + min_loop)
    for _ in range(120):
        n = int(rng.integers(0, 11))
        x = rng.integers(0, 4, size=n).astype(np.uint8)
        r = oracle.fold(x, min_loop=min_loop)
        want = brute_fold(x.tolist(), min_loop) if n else 0
        assert r["score"] == want, (x, min_loop)
        assert check_structure(x.tolist(), r["partner"], min_loop) == r["score"]
        assert r["cells"] == n * (n + 1) // 2


def test_xdrop_inactive_is_unpruned(oracle_lib):
    rng = np.random.default_rng(52)
    for _ in range(40):
        n = int(rng.integers(1, 80))
        x = rng.integers(0, 4, size=n).astype(np.uint8)
        u = oracle.fold(x)
        for kw in (dict(xdrop=10**9, warmup=0), dict(xdrop=0, warmup=n)):
            r = oracle.fold(x, **kw)
            assert (r["score"], r["cells"], r["status"]) == (u["score"], u["cells"], u["status"])
            assert np.array_equal(r["partner"], u["partner"])


def test_pruned_never_more(oracle_lib):
    rng = np.random.default_rng(53)
    pruned = 0
    for _ in range(40):
        n = int(rng.integers(20, 120))
        x = rng.integers(0, 4, size=n).astype(np.uint8)
        u = oracle.fold(x)
        for X, w in ((0, 0), (1, 5), (2, 15), (5, 15)):
            r = oracle.fold(x, xdrop=X, warmup=w)
            assert r["score"] <= u["score"] and r["cells"] <= u["cells"]
            pruned += r["cells"] < u["cells"]
            got = check_structure(x.tolist(), r["partner"], 3)
            assert got == r["score"]
            if r["status"] == 0:
                assert (r["i_end"], r["j_end"]) == (0, n - 1)
    assert pruned > 0


def _golden():
    with open(os.path.join(HERE, "golden", "fold_hand_worked.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_hand_worked(case, oracle_lib):
    x = np.array([CODE[c] for c in case["x"]], np.uint8)
    r = oracle.fold(x, min_loop=case["min_loop"], xdrop=case.get("xdrop"),
                    warmup=case.get("warmup", 15))
    assert (r["score"], r["status"], r["cells"]) == (case["score"], case["status"], case["cells"])
    if "structure" in case:
        assert structure(r["partner"]) == case["structure"]


def test_batch_matches_single(oracle_lib):
    rng = np.random.default_rng(54)
    lens = rng.integers(0, 60, size=25).astype(np.uint32)
    off = np.zeros(25, np.uint64)
    off[1:] = np.cumsum(lens[:-1])
    seq = rng.integers(0, 4, size=int(lens.sum())).astype(np.uint8)
    res, partner = oracle.fold_batch(seq, off, lens, nthreads=3, xdrop=1, warmup=4)
    for p in range(25):
        a, n = int(off[p]), int(lens[p])
        one = oracle.fold(seq[a:a + n], xdrop=1, warmup=4)
        assert (res[p]["score"], res[p]["cells"], res[p]["status"]) == (
            one["score"], one["cells"], one["status"])
        assert np.array_equal(partner[a:a + n], one["partner"])


def test_invalid_arguments(oracle_lib):
    with pytest.raises(ValueError):
        oracle.fold([0, 4, 1])
    with pytest.raises(ValueError):
        oracle.fold([0, 1], min_loop=-1)
