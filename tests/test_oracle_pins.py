"""Pins for the CPU oracle: checks against facts the paper and the mathematics
fix, none of which is the oracle restating itself.

  * brute force over every alignment path (Delannoy enumeration) for M, N <= 6;
  * unit-cost global alignment equals minus the Levenshtein distance (Sec. 2's
    edit-distance recurrence is exactly that special case);
  * self-alignment scores the sum of the diagonal substitution scores;
  * a band at least as wide as the matrix reproduces the unpruned run; the
    banded domain in (k, m) coordinates matches the closed form of Sec. 7.1;
    a banded score is the best path that stays inside the band (brute force);
  * X-drop with X = infinity reproduces the unpruned run;
  * row-major and antidiagonal evaluation agree in every output (Sec. 6:
    ordering rewrites preserve values and traceback);
  * hand-worked examples (tests/golden/hand_worked.json);
  * every CIGAR re-scores to the reported score and spans the reported range.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from pins import (brute_global, brute_global_band, brute_global_mid, brute_local, brute_local_band,
                  brute_local_mid, cigar_from_str,
                  levenshtein, mid_ok, rescore_cigar)

HERE = os.path.dirname(os.path.abspath(__file__))
DNA_S = np.array([[2, -4, -4, -4], [-4, 2, -4, -4], [-4, -4, 2, -4], [-4, -4, -4, 2]], np.int8)


def _asym(rng, a):
    S = rng.integers(-5, 6, size=(a, a)).astype(np.int8)
    return S


SCORINGS = [
    # (name, alphabet, subst maker, affine, o, e)
    ("dna_affine", 4, lambda rng: DNA_S, True, 4, 2),
    ("dna_linear", 4, lambda rng: DNA_S, False, 0, 2),
    ("asym5_affine", 5, lambda rng: _asym(rng, 5), True, 3, 1),
    ("asym5_affine_o0", 5, lambda rng: _asym(rng, 5), True, 0, 2),
    ("asym3_linear", 3, lambda rng: _asym(rng, 3), False, 0, 1),
]


def _check_cigar(res, q, r, S, o, e):
    sc, dq, dr = rescore_cigar(res["cigar"], q, r, S, o, e, res["q_begin"], res["r_begin"])
    assert sc == res["score"]
    assert dq == res["q_end"] - res["q_begin"]
    assert dr == res["r_end"] - res["r_begin"]


@pytest.mark.parametrize("name,alpha,mk,affine,o,e", SCORINGS)
@pytest.mark.parametrize("mode", ["global", "local"])
def test_brute_force(name, alpha, mk, affine, o, e, mode, oracle_lib):
    rng = np.random.default_rng(abs(hash((name, mode))) % 2**32)
    S = mk(rng)
    oo = o if affine else 0
    ncase = 14 if mode == "global" else 8
    maxl = 6 if mode == "global" else 4
    for _ in range(ncase):
        M, N = int(rng.integers(0, maxl + 1)), int(rng.integers(0, maxl + 1))
        q = rng.integers(0, alpha, size=M).astype(np.uint8)
        r = rng.integers(0, alpha, size=N).astype(np.uint8)
        res = oracle.align(q, r, S, mode=mode, affine=affine, gap_open=o, gap_extend=e)
        if mode == "global":
            want = brute_global(q.tolist(), r.tolist(), S, oo, e)
            assert res["score"] == want, (q, r)
            assert res["status"] == 0
            assert (res["q_end"], res["r_end"]) == (M, N)
            assert res["cells"] == M * N
        else:
            want = brute_local(q.tolist(), r.tolist(), S, oo, e)
            assert res["score"] == want, (q, r)
            assert res["status"] == (3 if want == 0 else 0)
        if res["status"] == 0:
            _check_cigar(res, q, r, S, oo, e)


def test_levenshtein(oracle_lib):
    rng = np.random.default_rng(11)
    S = np.where(np.eye(4, dtype=bool), 0, -1).astype(np.int8)
    for _ in range(60):
        M, N = int(rng.integers(0, 40)), int(rng.integers(0, 40))
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        res = oracle.align(q, r, S, mode="global", affine=False, gap_extend=1)
        assert res["score"] == -levenshtein(q.tolist(), r.tolist())
        _check_cigar(res, q, r, S, 0, 1)


@pytest.mark.parametrize("mode", ["global", "local"])
def test_self_alignment(mode, oracle_lib):
    import synth

    rng = np.random.default_rng(5)
    P = synth.protein_subst(np.random.default_rng(2))
    for S, alpha, o, e in [(DNA_S, 4, 4, 2), (P, 20, 11, 1)]:
        for L in [1, 7, 50, 131]:
            q = rng.integers(0, alpha, size=L).astype(np.uint8)
            res = oracle.align(q, q, S, mode=mode, affine=True, gap_open=o, gap_extend=e)
            assert res["score"] == int(sum(int(S[c, c]) for c in q))
            assert oracle.cigar_str(res["cigar"]) == f"{L}="
            assert (res["q_begin"], res["q_end"], res["r_begin"], res["r_end"]) == (0, L, 0, L)


@pytest.mark.parametrize("mode", ["global", "local"])
def test_wide_band_equals_unpruned(mode, oracle_lib):
    rng = np.random.default_rng(7)
    for _ in range(25):
        M, N = int(rng.integers(0, 30)), int(rng.integers(0, 30))
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        full = oracle.align(q, r, DNA_S, mode=mode, gap_open=4, gap_extend=2)
        for literal in (False, True):
            b = oracle.align(q, r, DNA_S, mode=mode, gap_open=4, gap_extend=2,
                             band=max(M, N), band_literal=literal)
            assert b["score"] == full["score"] and b["cells"] == full["cells"] == M * N
            assert np.array_equal(b["cigar"], full["cigar"])
            assert (b["q_begin"], b["r_begin"], b["q_end"], b["r_end"]) == (
                full["q_begin"], full["r_begin"], full["q_end"], full["r_end"])


def test_band_closed_form(oracle_lib):
    """Sec. 7.1: under shear(k = antidiag(i,j), m = j) the band -B <= diag <= B
    becomes max(0, k-M, ceil((k-B)/2)) <= m <= min(N, k, floor((k+B)/2))."""
    rng = np.random.default_rng(3)
    for M, N, B in [(9, 9, 2), (12, 7, 3), (5, 14, 0), (20, 20, 6), (3, 3, 10)]:
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        ij, alive = oracle.domain(q, r, DNA_S, mode="global", gap_open=4, gap_extend=2,
                                  band=B, band_literal=True)
        got = {(int(i), int(j)) for i, j in ij}
        want = set()
        for k in range(M + N + 1):
            lo = max(0, k - M, math.ceil((k - B) / 2))
            hi = min(N, k, math.floor((k + B) / 2))
            for m in range(lo, hi + 1):
                want.add((k - m, m))
        assert got == want
        res = oracle.align(q, r, DNA_S, mode="global", gap_open=4, gap_extend=2, band=B,
                           band_literal=True)
        assert res["cells"] == sum(1 for (i, j) in want if i >= 1 and j >= 1)
        assert res["status"] == (0 if abs(N - M) <= B else 2)


@pytest.mark.parametrize("affine,o", [(True, 4), (False, 0)])
@pytest.mark.parametrize("mode", ["global", "local"])
def test_band_brute_force(mode, affine, o, oracle_lib):
    """Sec. 7.1: a banded alignment scores the best path (in local mode, the best
    path between any two cells, or 0) whose every cell lies inside the band --
    brute force over every path of tiny pairs, literal and widened bands.  A
    global pair whose band holds no path from (0,0) to (M,N) is unreachable."""
    rng = np.random.default_rng(31 if affine else 32)
    seen_unreachable = seen_clipped = False
    for t in range(48):
        M, N = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        if t % 3 == 1:  # a related pair: substitutions of the reference, then cut to M
            q = np.where(rng.random(max(M, N)) < 0.2, rng.integers(0, 4, size=max(M, N)),
                         np.resize(r, max(M, N)))[:M].astype(np.uint8)
        elif t % 3 == 2:  # the reference behind 1-2 extra residues: its diagonal is -s
            s = int(rng.integers(1, 3))
            q = np.concatenate([rng.integers(0, 4, size=s), r])[:max(M, s + 1)].astype(np.uint8)
            M = len(q)
        else:
            q = rng.integers(0, 4, size=M).astype(np.uint8)
        B = int(rng.integers(0, 3))
        for literal in (False, True):
            if literal:
                lo, hi = -B, B
            else:  # widened to hold both corners
                lo, hi = min(0, N - M) - B, max(0, N - M) + B
            res = oracle.align(q, r, DNA_S, mode=mode, affine=affine, gap_open=o, gap_extend=2,
                               band=B, band_literal=literal)
            unbanded = oracle.align(q, r, DNA_S, mode=mode, affine=affine, gap_open=o,
                                    gap_extend=2)
            if mode == "global":
                want = brute_global_band(q, r, DNA_S, o, 2, lo, hi)
                if want is None:
                    seen_unreachable = True
                    assert res["status"] == 2
                    continue
                assert res["status"] == 0 and res["score"] == want
            else:
                want = brute_local_band(q, r, DNA_S, o, 2, lo, hi)
                assert res["score"] == want
                if want == 0:
                    continue
            seen_clipped |= want < unbanded["score"]
            _check_cigar(res, q, r, DNA_S, o, 2)
    assert seen_clipped  # some band cut off the unbanded optimum
    if mode == "global":
        assert seen_unreachable  # some literal band missed the far corner


def test_widened_band_holds_both_corners(oracle_lib):
    rng = np.random.default_rng(4)
    for M, N, B in [(30, 10, 2), (8, 25, 0), (15, 15, 1)]:
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        res = oracle.align(q, r, DNA_S, mode="global", gap_open=4, gap_extend=2, band=B)
        assert res["status"] == 0 and (res["q_end"], res["r_end"]) == (M, N)
        ij, _ = oracle.domain(q, r, DNA_S, mode="global", band=B)
        d = ij[:, 1] - ij[:, 0]
        assert d.min() == min(0, N - M) - B or d.min() == -M
        _check_cigar(res, q, r, DNA_S, 4, 2)


@pytest.mark.parametrize("mode", ["global", "local"])
def test_xdrop_infinite_equals_unpruned(mode, oracle_lib):
    rng = np.random.default_rng(9)
    for _ in range(25):
        M, N = int(rng.integers(0, 25)), int(rng.integers(0, 25))
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        full = oracle.align(q, r, DNA_S, mode=mode, gap_open=4, gap_extend=2)
        x = oracle.align(q, r, DNA_S, mode=mode, gap_open=4, gap_extend=2, xdrop=oracle.INF)
        for key in ("score", "q_begin", "q_end", "r_begin", "r_end", "status", "cells"):
            assert x[key] == full[key]
        assert np.array_equal(x["cigar"], full["cigar"])


@pytest.mark.parametrize("mode", ["global", "local"])
def test_zdrop_infinite_equals_unpruned(mode, oracle_lib):
    """Sec. 9.3 Z-drop with Z = infinity prunes nothing: the unpruned result."""
    rng = np.random.default_rng(19)
    for _ in range(25):
        M, N = int(rng.integers(0, 25)), int(rng.integers(0, 25))
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        full = oracle.align(q, r, DNA_S, mode=mode, gap_open=4, gap_extend=2)
        z = oracle.align(q, r, DNA_S, mode=mode, gap_open=4, gap_extend=2, zdrop=oracle.INF)
        for key in ("score", "q_begin", "q_end", "r_begin", "r_end", "status", "cells"):
            assert z[key] == full[key]
        assert np.array_equal(z["cigar"], full["cigar"])


@pytest.mark.parametrize("band", [None, 3])
@pytest.mark.parametrize("mode", ["global", "local"])
def test_schedule_invariance(mode, band, oracle_lib):
    """Sec. 6: row-major and antidiagonal orders give identical values and
    traceback."""
    rng = np.random.default_rng(13)
    S = _asym(rng, 4)
    for _ in range(20):
        M, N = int(rng.integers(0, 30)), int(rng.integers(0, 30))
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = rng.integers(0, 4, size=N).astype(np.uint8)
        a = oracle.align(q, r, S, mode=mode, gap_open=3, gap_extend=1, band=band, order=0)
        b = oracle.align(q, r, S, mode=mode, gap_open=3, gap_extend=1, band=band, order=1)
        assert {k: v for k, v in a.items() if k != "cigar"} == {k: v for k, v in b.items() if k != "cigar"}
        assert np.array_equal(a["cigar"], b["cigar"])


def test_linear_equals_affine_open0(oracle_lib):
    rng = np.random.default_rng(17)
    S = _asym(rng, 4)
    for mode in ("global", "local"):
        for _ in range(20):
            M, N = int(rng.integers(0, 30)), int(rng.integers(0, 30))
            q = rng.integers(0, 4, size=M).astype(np.uint8)
            r = rng.integers(0, 4, size=N).astype(np.uint8)
            a = oracle.align(q, r, S, mode=mode, affine=False, gap_extend=2)
            b = oracle.align(q, r, S, mode=mode, affine=True, gap_open=0, gap_extend=2)
            assert a["score"] == b["score"] and np.array_equal(a["cigar"], b["cigar"])


def _golden():
    with open(os.path.join(HERE, "golden", "hand_worked.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_hand_worked(case, oracle_lib):
    code = {"A": 0, "C": 1, "G": 2, "T": 3}
    q = np.array([code[c] for c in case["q"]], np.uint8)
    r = np.array([code[c] for c in case["r"]], np.uint8)
    S = np.full((4, 4), case["mismatch"], np.int8)
    np.fill_diagonal(S, case["match"])
    kw = dict(mode=case["mode"], affine=case["affine"], gap_open=case["gap_open"],
              gap_extend=case["gap_extend"], xdrop=case.get("xdrop"), zdrop=case.get("zdrop"),
              xdrop_running=case.get("running", False), mid=case.get("mid", False))
    res = oracle.align(q, r, S, **kw)
    assert res["score"] == case["score"]
    assert res["status"] == case["status"]
    assert res["cells"] == case["cells"]
    assert oracle.cigar_str(res["cigar"]) == case["cigar"]
    for key in ("q_begin", "q_end", "r_begin", "r_end", "last_k"):
        if key in case:
            assert res[key] == case[key], key
    if "alive" in case:
        ij, alive = oracle.domain(q, r, S, **kw)
        got_alive = {(int(i), int(j)) for (i, j), a in zip(ij, alive) if a}
        got_pruned = {(int(i), int(j)) for (i, j), a in zip(ij, alive) if not a}
        assert got_alive == {tuple(x) for x in case["alive"]}
        assert got_pruned == {tuple(x) for x in case["pruned"]}
    if "H" in case:
        # every row-major prefix: H of (i, j) equals the score of aligning q[:i] and r[:j] globally
        H = np.array(case["H"])
        for i in range(len(q) + 1):
            for j in range(len(r) + 1):
                sub = oracle.align(q[:i], r[:j], S, **kw)
                assert sub["score"] == H[i, j], (i, j)


def test_cigar_helpers():
    assert oracle.cigar_str(cigar_from_str("3=1X2I4D")) == "3=1X2I4D"


def test_batch_matches_single(oracle_lib):
    import synth

    b = synth.short_dna_pairs(n=20, seed=1)
    res, ops, off = oracle.align_batch(b, nthreads=3, traceback=True)
    for p in range(b.n):
        q, r = b.pair(p)
        one = oracle.align(q, r, b.subst, **dict(b.scoring, traceback=True))
        assert res[p]["score"] == one["score"] and res[p]["cells"] == one["cells"]
        n = int(res[p]["n_ops"])
        assert np.array_equal(ops[int(off[p]):int(off[p]) + n], one["cigar"])


def test_invalid_arguments(oracle_lib):
    with pytest.raises(ValueError):
        oracle.align(np.array([5], np.uint8), np.array([0], np.uint8), DNA_S)
    with pytest.raises(ValueError):
        oracle.align(np.array([0], np.uint8), np.array([0], np.uint8), DNA_S, gap_open=-1)


@pytest.mark.parametrize("zd", [False, True])
@pytest.mark.parametrize("mode", ["global", "local"])
def test_running_threshold(mode, zd, oracle_lib):
    """The running-maximum variant: with X = infinity it is the unpruned run.  For
    X-drop its threshold is never below the literal one, so it keeps a subset of
    the cells the literal run keeps (evaluated and alive); Z-drop's distance term
    is measured from another reference diagonal, so there only the CIGAR is
    checked."""
    rng = np.random.default_rng(31)
    S = np.where(np.eye(4, dtype=bool), 2, -3).astype(np.int8)
    for _ in range(40):
        M, N = int(rng.integers(1, 40)), int(rng.integers(1, 40))
        q = rng.integers(0, 4, size=M).astype(np.uint8)
        r = q[:N].copy() if rng.random() < 0.5 and N <= M else rng.integers(0, 4, size=N).astype(np.uint8)
        N = len(r)
        base = dict(mode=mode, affine=True, gap_open=2, gap_extend=1)
        key = "zdrop" if zd else "xdrop"
        inf = oracle.align(q, r, S, **base, **{key: oracle.INF}, xdrop_running=True)
        un = oracle.align(q, r, S, **base)
        assert (inf["score"], inf["q_end"], inf["r_end"]) == (un["score"], un["q_end"], un["r_end"])
        for X in (0, 3, 8):
            lit = oracle.align(q, r, S, **base, **{key: X})
            run = oracle.align(q, r, S, **base, **{key: X}, xdrop_running=True)
            if run["status"] == 0:
                _check_cigar(run, q, r, S, 2, 1)
            if zd:
                continue
            assert run["cells"] <= lit["cells"]
            ij_l, al_l = oracle.domain(q, r, S, **base, **{key: X})
            ij_r, al_r = oracle.domain(q, r, S, **base, **{key: X}, xdrop_running=True)
            lit_cells = {tuple(x) for x in ij_l.tolist()}
            lit_alive = {tuple(x) for x, a in zip(ij_l.tolist(), al_l) if a}
            assert {tuple(x) for x in ij_r.tolist()} <= lit_cells
            assert {tuple(x) for x, a in zip(ij_r.tolist(), al_r) if a} <= lit_alive


@pytest.mark.parametrize("mode", ["global", "local"])
def test_mid_brute_force(mode, oracle_lib):
    """Table 1's M/I/D form against every alignment path of its grammar (no
    insertion next to a deletion), asymmetric scores, M, N <= 5; the CIGAR obeys
    the grammar and re-scores to the score."""
    rng = np.random.default_rng(41)
    for t in range(60):
        S = _asym(rng, 3)
        o, e = int(rng.integers(0, 4)), int(rng.integers(1, 3))
        M, N = int(rng.integers(0 if mode == "global" else 1, 6)), int(rng.integers(1, 6))
        q = rng.integers(0, 3, size=M).astype(np.uint8)
        r = rng.integers(0, 3, size=N).astype(np.uint8)
        res = oracle.align(q, r, S, mode=mode, affine=True, gap_open=o, gap_extend=e, mid=True)
        want = (brute_global_mid if mode == "global" else brute_local_mid)(
            q.tolist(), r.tolist(), S, o, e)
        assert res["score"] == want, (t, q, r, o, e)
        if res["status"] == 0:
            _check_cigar(res, q, r, S, o, e)
            steps = "".join({1: "V", 2: "H", 7: "M", 8: "M"}[op & 15] * (op >> 4)
                            for op in res["cigar"].tolist())
            assert mid_ok(steps)


@pytest.mark.parametrize("mode", ["global", "local"])
def test_mid_brute_force_cheap_gaps(mode, oracle_lib):
    """Scores where a deletion beside an insertion would beat a mismatch (match 1,
    mismatch -5, open 0 or 1, extend 1): the M/I/D form must still keep them
    apart, and the H/E/F form must find the pairs that use them."""
    rng = np.random.default_rng(43)
    S = np.array([[1, -5, -5], [-5, 1, -5], [-5, -5, 1]], np.int8)
    differ = 0
    for t in range(200):
        o = int(rng.integers(0, 2))
        M, N = int(rng.integers(1, 5)), int(rng.integers(1, 5))
        q = rng.integers(0, 3, size=M).astype(np.uint8)
        r = rng.integers(0, 3, size=N).astype(np.uint8)
        res = oracle.align(q, r, S, mode=mode, affine=True, gap_open=o, gap_extend=1, mid=True)
        want = (brute_global_mid if mode == "global" else brute_local_mid)(
            q.tolist(), r.tolist(), S, o, 1)
        assert res["score"] == want, (t, q, r, o)
        if res["status"] == 0:
            _check_cigar(res, q, r, S, o, 1)
            steps = "".join({1: "V", 2: "H", 7: "M", 8: "M"}[op & 15] * (op >> 4)
                            for op in res["cigar"].tolist())
            assert mid_ok(steps), (t, oracle.cigar_str(res["cigar"]))
        hef = oracle.align(q, r, S, mode=mode, affine=True, gap_open=o, gap_extend=1)
        differ += hef["score"] != res["score"]
    if mode == "global":  # local alignments end before such regions anyway
        assert differ > 0


def test_mid_equals_hef_on_dna_scoring(oracle_lib):
    """With the DNA scoring of the workloads (+2/-4, open 4, extend 2) a deletion
    next to an insertion never beats a mismatch, so both forms score alike."""
    import synth
    S = synth.dna_subst(2, -4)
    qs, rs = synth.random_pairs(60, 80, 80, 4, seed=42, related=0.7)
    for q, r in zip(qs, rs):
        for mode in ("global", "local"):
            a = oracle.align(q, r, S, mode=mode, affine=True, gap_open=4, gap_extend=2)
            b = oracle.align(q, r, S, mode=mode, affine=True, gap_open=4, gap_extend=2, mid=True)
            assert a["score"] == b["score"]
