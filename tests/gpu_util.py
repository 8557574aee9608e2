"""Helpers for the GPU parity tests: run a batch through the C ABI and through the
oracle, and compare every output field exactly (integer work: bit-exact)."""
from __future__ import annotations

import numpy as np

import oracle

FIELDS = ("score", "q_end", "r_end", "status", "cells")


def oracle_batch(batch, sc):
    return oracle.align_batch(batch, **sc)


def compare(batch, sc, res, cig, ores, oops, ooff, idx=None, label=""):
    """Assert exact equality of every pair (or of the pairs in idx, which index
    both `res` and the batch while `ores` rows follow idx order)."""
    pairs = range(batch.n) if idx is None else idx
    bad = []
    for row, p in enumerate(pairs):
        o = ores[row] if idx is not None else ores[p]
        g = res[p]
        for f in FIELDS:
            if int(g[f]) != int(o[f]):
                bad.append((p, f, int(g[f]), int(o[f])))
        if sc.get("traceback"):
            for f in ("q_begin", "r_begin"):
                if int(g[f]) != int(o[f]):
                    bad.append((p, f, int(g[f]), int(o[f])))
            got = cig[int(g["cigar_off"]):int(g["cigar_off"]) + int(g["cigar_len"])]
            want = oops[int(ooff[row if idx is not None else p]):int(ooff[row if idx is not None else p]) + int(o["n_ops"])]
            if not np.array_equal(got, want):
                bad.append((p, "cigar", oracle.cigar_str(got)[:80], oracle.cigar_str(want)[:80]))
        elif int(g["q_begin"]) != (-1 if sc.get("mode") == "local" and int(o["status"]) == 0 else 0):
            bad.append((p, "q_begin(score-only)", int(g["q_begin"]), None))
        if len(bad) > 8:
            break
    assert not bad, f"{label}: {len(bad)} mismatches, first: {bad[:8]}"
