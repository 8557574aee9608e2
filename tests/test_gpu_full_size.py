"""Parity at the configured sizes of the long workloads (bit-exact against the
oracle, tolerance 0: the arithmetic is exact integer).

* Long reads at their real lengths (10-50 kb, band 256 widened to hold both
  corners, X-drop 400, traceback): a seeded sample of 24 pairs of the
  10,000-pair workload, regenerated pair by pair, through the batched call.
* An X-drop batch cut into several traceback waves by a small workspace, with
  pairs that outgrow the one-warp window and are rerun wider in sub-waves.
* The megabase pair (X-drop 1000) through filtr_align_long against the oracle's
  result stored in tests/golden/long_pair_1mbp.json (written by
  tests/golden/make_long_pair_golden.py, which runs only the oracle).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import compare, oracle_batch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
DNA_S = synth.dna_subst(2, -4)


@pytest.fixture(scope="module")
def F():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_06225_gb300 as F

    return F


def test_long_reads_configured_lengths(F):
    """24 pairs drawn (seeded) from the 10,000-pair long-read workload, at its
    10-50 kb lengths: every field and every CIGAR equal to the oracle's."""
    idx = np.sort(np.random.default_rng(303).choice(10_000, size=24, replace=False))
    b = synth.long_reads(idx=idx)
    assert int(b.q_len.min()) >= 9_000 and int(b.r_len.max()) <= 50_000
    sc = dict(b.scoring)
    ctx = F.Context(0, 2 << 30)
    try:
        params = F.make_params(b.subst, **sc)
        res, cig, rc = F.align_batch(ctx, params, b)
        assert rc == 0, F.last_error()
    finally:
        ctx.close()
    ores, oops, ooff = oracle_batch(b, sc)
    compare(b, sc, res, cig, ores, oops, ooff, label="long reads 10-50 kb")
    assert (res["status"] == 0).all()


def test_xdrop_several_waves_and_reruns(F):
    """A 12 MB workspace holds the traceback of only a few pairs at a time, so
    the X-drop batch runs in several waves; with a large threshold the live
    region of most pairs outgrows the one-warp window and is rerun with wider
    groups, again in sub-waves that fit the workspace."""
    ctx = F.Context(0, 12 << 20)
    try:
        ctx.set_timing(True)
        b = synth.long_reads(n=40, lmin=1500, lmax=3000, seed=41)
        sc = dict(b.scoring)
        params = F.make_params(b.subst, **sc)
        res, cig, rc = F.align_batch(ctx, params, b)
        assert rc == 0, F.last_error()
        st = ctx.last_stats()
        assert st["waves"] >= 3, st
        ores, oops, ooff = oracle_batch(b, sc)
        compare(b, sc, res, cig, ores, oops, ooff, label="waves")

        qs, rs = synth.random_pairs(30, 1100, 1100, 4, seed=42, mmin=300, nmin=300, related=0.8)
        b2 = synth.pack(qs, rs, 4, DNA_S)
        sc2 = dict(mode="global", affine=True, gap_open=4, gap_extend=2, xdrop=1500, traceback=True)
        params = F.make_params(DNA_S, **sc2)
        res2, cig2, rc = F.align_batch(ctx, params, b2)
        assert rc == 0, F.last_error()
        st2 = ctx.last_stats()
        assert st2["waves"] >= 2, st2
        ores2, oops2, ooff2 = oracle_batch(b2, sc2)
        compare(b2, sc2, res2, cig2, ores2, oops2, ooff2, label="waves + reruns")
        # the reruns really happened: some pair's live region is wider than 256 cells
        widths = [oracle.domain(*b2.pair(p), DNA_S, **sc2)[0] for p in range(4)]
        assert max(int(np.bincount(ij[:, 0] + ij[:, 1]).max()) for ij in widths) > 256
    finally:
        ctx.close()


def test_megabase_pair_against_oracle_golden(F):
    """The 1,000,000 bp pair (1% divergence, one 5 kb inserted segment, X-drop
    1000) through filtr_align_long: score, end cell, status, cell count and the
    whole CIGAR (length and SHA-256) equal the oracle's stored result."""
    path = os.path.join(HERE, "golden", "long_pair_1mbp.json")
    with open(path) as f:
        g = json.load(f)
    b = synth.long_pair()
    q, r = b.pair(0)
    assert (int(q.shape[0]), int(r.shape[0])) == (g["M"], g["N"])
    ctx = F.Context(0, 8 << 30)
    try:
        params = F.make_params(b.subst, **b.scoring)
        res, cig, rc = F.align_long(ctx, params, q, r)
        assert rc == 0, F.last_error()
    finally:
        ctx.close()
    for f in ("score", "q_end", "r_end", "status", "cells"):
        assert int(res[f]) == int(g[f]), (f, int(res[f]), g[f])
    assert int(cig.shape[0]) == g["n_ops"]
    digest = hashlib.sha256(np.ascontiguousarray(cig, dtype="<u4").tobytes()).hexdigest()
    assert digest == g["cigar_sha256"]
