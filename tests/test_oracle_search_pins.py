"""Pins for the search-traversal oracle (oracle/search.c, Sec. 6.3): checks
against what the mathematics fixes, none of which is the oracle restating
itself.

  * the distance equals the textbook two-row Levenshtein distance, brute force
    over every alignment path for tiny inputs, and minus the unit-cost global
    score of the (separately pinned) alignment oracle;
  * a band: at least as wide as the matrix it changes nothing; otherwise the
    distance equals the unit-cost banded alignment score (both are the best path
    inside the same diagonals);
  * the cell count of an exact run follows the domain's closed form (one more
    diagonal on each side per score, clipped to the matrix and the band);
  * every CIGAR consumes both sequences, its '=' / 'X' agree with the residues
    and it costs exactly the reported distance;
  * WFA-Adapt with thresholds that cannot trigger reproduces the exact run's
    alignment; with any thresholds it never reports less than the edit distance;
  * hand-worked wavefronts (tests/golden/search_hand_worked.json).
The CIGAR's choice among equally short alignments and the WFA-Adapt trimming
rule beyond these properties are readings the paper does not fix.
"""
import json
import os

import numpy as np
import pytest

import oracle
from pins import all_paths, levenshtein, rescore_cigar

HERE = os.path.dirname(os.path.abspath(__file__))
UNIT4 = np.where(np.eye(4, dtype=bool), 0, -1).astype(np.int8)


def _pairs(seed, n, lmax, alpha, related=0.6):
    import synth
    return list(zip(*synth.random_pairs(n, lmax, lmax, alpha, seed=seed, related=related)))


def _unit(alpha):
    return np.where(np.eye(alpha, dtype=bool), 0, -1).astype(np.int8)


def _check_cigar(res, q, r):
    sc, qi, rj = rescore_cigar(res["cigar"], q, r, _unit(256), 0, 1, 0, 0)
    assert (qi, rj) == (len(q), len(r))
    assert -sc == res["distance"]


@pytest.mark.parametrize("alpha", [2, 4, 20])
def test_levenshtein(alpha, oracle_lib):
    for q, r in _pairs(21 + alpha, 60, 40, alpha):
        res = oracle.search(q, r)
        assert res["distance"] == levenshtein(q.tolist(), r.tolist())
        _check_cigar(res, q, r)


def test_brute_force(oracle_lib):
    rng = np.random.default_rng(22)
    for _ in range(150):
        M, N = int(rng.integers(0, 6)), int(rng.integers(0, 6))
        q = rng.integers(0, 3, size=M).astype(np.uint8)
        r = rng.integers(0, 3, size=N).astype(np.uint8)
        best = None
        for p in all_paths(M, N):
            i = j = cost = 0
            for mv in p:
                if mv == "M":
                    cost += int(q[i] != r[j])
                    i += 1
                    j += 1
                elif mv == "H":
                    cost += 1
                    j += 1
                else:
                    cost += 1
                    i += 1
            best = cost if best is None else min(best, cost)
        res = oracle.search(q, r)
        assert res["distance"] == best, (q, r)
        _check_cigar(res, q, r)


def test_equals_unit_cost_alignment(oracle_lib):
    for q, r in _pairs(23, 40, 300, 4, related=0.8):
        res = oracle.search(q, r)
        al = oracle.align(q, r, UNIT4, mode="global", affine=False, gap_extend=1, traceback=False)
        assert res["distance"] == -al["score"]


def _domain_cells(D, M, N, dlo, dhi):
    """Sum over s = 0..D of the width of [max(-s, dlo), min(s, dhi)]."""
    return sum(min(s, dhi) - max(-s, dlo) + 1 for s in range(D + 1))


@pytest.mark.parametrize("band", [None, 0, 3])
def test_cells_closed_form(band, oracle_lib):
    for q, r in _pairs(24, 40, 50, 4):
        M, N = len(q), len(r)
        res = oracle.search(q, r, band=band)
        dlo, dhi = -M, N
        if band is not None:
            dlo = max(dlo, min(0, N - M) - band)
            dhi = min(dhi, max(0, N - M) + band)
        assert res["cells"] == _domain_cells(res["distance"], M, N, dlo, dhi)


def test_band(oracle_lib):
    for q, r in _pairs(25, 40, 80, 4, related=0.8):
        M, N = len(q), len(r)
        exact = oracle.search(q, r)
        wide = oracle.search(q, r, band=M + N)
        assert (wide["distance"], wide["cells"]) == (exact["distance"], exact["cells"])
        assert np.array_equal(wide["cigar"], exact["cigar"])
        for B in (0, 2, 7):
            res = oracle.search(q, r, band=B)
            al = oracle.align(q, r, UNIT4, mode="global", affine=False, gap_extend=1, band=B,
                              traceback=False)
            assert res["distance"] == -al["score"]
            _check_cigar(res, q, r)
            lo, hi = min(0, N - M) - B, max(0, N - M) + B
            i = j = 0
            for op in res["cigar"].tolist():  # the path stays inside the band
                n, c = op >> 4, op & 15
                for _ in range(n):
                    i += c in (1, 7, 8)
                    j += c in (2, 7, 8)
                    assert lo <= j - i <= hi


def test_identical_and_empty(oracle_lib):
    rng = np.random.default_rng(26)
    q = rng.integers(0, 4, size=57).astype(np.uint8)
    res = oracle.search(q, q)
    assert (res["distance"], res["cells"], oracle.cigar_str(res["cigar"])) == (0, 1, "57=")
    e = np.zeros(0, np.uint8)
    assert oracle.search(e, q)["distance"] == 57
    assert oracle.cigar_str(oracle.search(e, q)["cigar"]) == "57D"
    assert oracle.cigar_str(oracle.search(q, e)["cigar"]) == "57I"
    assert oracle.search(e, e)["distance"] == 0


def test_adapt_inactive_is_exact(oracle_lib):
    """Never reaching min_len changes nothing; a max_dist no diagonal can exceed
    trims only unreached end diagonals, which feed nothing: same distance and
    CIGAR, no more cells."""
    for q, r in _pairs(27, 40, 80, 4):
        M, N = len(q), len(r)
        exact = oracle.search(q, r)
        res = oracle.search(q, r, adapt=(M + N + 2, 0))
        assert (res["distance"], res["cells"]) == (exact["distance"], exact["cells"])
        assert np.array_equal(res["cigar"], exact["cigar"])
        res = oracle.search(q, r, adapt=(1, M + N + 1))
        assert res["distance"] == exact["distance"] and res["cells"] <= exact["cells"]
        assert np.array_equal(res["cigar"], exact["cigar"])


def test_adapt_never_below_distance(oracle_lib):
    hits = 0
    for q, r in _pairs(28, 80, 120, 4, related=0.9):
        exact = oracle.search(q, r)["distance"]
        for adapt in ((1, 0), (4, 2), (10, 5)):
            res = oracle.search(q, r, adapt=adapt)
            assert res["distance"] >= exact
            hits += res["distance"] > exact
            _check_cigar(res, q, r)
    assert hits > 0  # the heuristic does trim on these inputs


def _golden():
    with open(os.path.join(HERE, "golden", "search_hand_worked.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden(), ids=lambda c: c["name"])
def test_hand_worked(case, oracle_lib):
    code = {"A": 0, "C": 1, "G": 2, "T": 3}
    q = np.array([code[c] for c in case["q"]], np.uint8)
    r = np.array([code[c] for c in case["r"]], np.uint8)
    res = oracle.search(q, r, band=case.get("band"), adapt=case.get("adapt"))
    assert res["distance"] == case["distance"]
    assert res["cells"] == case["cells"]
    assert oracle.cigar_str(res["cigar"]) == case["cigar"]


def test_batch_matches_single(oracle_lib):
    import synth
    qs, rs = synth.random_pairs(30, 70, 70, 4, seed=29, related=0.7)
    b = synth.pack(qs, rs, 4, UNIT4)
    res, ops, off = oracle.search_batch(b, nthreads=3, adapt=(6, 3))
    for p in range(b.n):
        q, r = b.pair(p)
        one = oracle.search(q, r, adapt=(6, 3))
        assert (res[p]["distance"], res[p]["cells"], res[p]["n_ops"]) == (
            one["distance"], one["cells"], one["n_ops"])
        assert np.array_equal(ops[int(off[p]):int(off[p]) + one["n_ops"]], one["cigar"])


def test_invalid_arguments(oracle_lib):
    q = np.zeros(3, np.uint8)
    with pytest.raises(ValueError):
        oracle.search(q, q, band=-1)
    with pytest.raises(ValueError):
        oracle.search(q, q, adapt=(-1, 0))
