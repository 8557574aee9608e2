"""The seeded input generators (synth/) against the recipes they state: event
rates of the mutation model, the workloads' length distributions, matrices,
request mix and arrivals, and seeding (a workload and any sample of it come back
identical)."""
import numpy as np
import pytest

import synth


def test_mutate_event_rates():
    """Long-read model: per reference base an insertion event w.p. 0.042 and a
    deletion event w.p. 0.021, Geometric(0.7) lengths, so 6% inserted and about
    3% deleted bases; substitutions 1%, always to a different residue."""
    rng = np.random.default_rng(11)
    n = 400_000
    ref = rng.integers(0, 4, n).astype(np.uint8)
    q = synth.mutate(rng, ref, 0.01, 0.042, 0.021, 0.7, draw=lambda k: np.full(k, 9))
    ins = int((q == 9).sum())
    assert ins / n == pytest.approx(0.06, abs=0.002)
    kept = n - (len(q) - ins)
    assert kept / n == pytest.approx(0.03, abs=0.002)  # runs that overlap merge
    # substitutions alone (no indels): the query keeps every position
    q = synth.mutate(rng, ref, 0.01, 0.0, 0.0, 0.7)
    assert len(q) == n
    assert (q != ref).mean() == pytest.approx(0.01, abs=0.001)
    # single-base indels (geom_p None): each event moves one base
    q = synth.mutate(rng, ref, 0.0, 0.01, 0.0, None, draw=lambda k: np.full(k, 9))
    assert (q == 9).sum() == len(q) - n
    assert (q == 9).sum() / n == pytest.approx(0.01, abs=0.001)


def test_short_dna():
    b = synth.short_dna_pairs()
    assert b.n == 1000 and (b.r_len == 128).all()
    assert b.q_len.mean() == pytest.approx(128, abs=1.0)
    assert b.scoring == dict(mode="global", affine=True, gap_open=4, gap_extend=2,
                             traceback=False)
    assert (b.subst == synth.dna_subst(2, -4)).all()


def test_protein_pairs():
    b = synth.protein_pairs(n=3000)
    for L in (b.r_len, b.q_len.astype(np.int64)):
        assert L.min() >= 90 and L.max() <= 1100  # U[100, 1000], then 1% + 1% indels
    assert b.r_len.min() >= 100 and b.r_len.max() <= 1000
    assert b.r_len.mean() == pytest.approx(550, abs=15)
    S = b.subst.astype(int)
    assert (S == S.T).all()
    d = np.diag(S)
    off = S[~np.eye(20, dtype=bool)]
    assert d.min() >= 4 and d.max() <= 11 and off.min() >= -4 and off.max() <= 3
    assert b.q_seq.max() < 20 and b.r_seq.max() < 20
    rng = np.random.default_rng(2)  # the matrix, then the background, as the workload draws them
    assert (synth.protein_subst(rng) == b.subst).all()
    bg = synth.protein_background(rng)
    assert bg.min() > 0 and bg.sum() == pytest.approx(1.0)


def test_long_reads_and_samples():
    full = synth.long_reads(n=300)
    assert full.r_len.min() >= 10_000 and full.r_len.max() <= 50_000
    ratio = full.q_len.astype(np.float64) / full.r_len
    assert ratio.mean() == pytest.approx(1.03, abs=0.003)  # +6% inserted, -3% deleted
    idx = [0, 17, 299]
    part = synth.long_reads(n=300, idx=idx)
    for t, p in enumerate(idx):
        qa, ra = full.pair(p)
        qb, rb = part.pair(t)
        assert np.array_equal(qa, qb) and np.array_equal(ra, rb)
    assert full.scoring["band"] == 256 and full.scoring["xdrop"] == 400


def test_serve_mix():
    reqs, _ = synth.serve_mix(4000, 1000.0)
    kinds = [r.kind for r in reqs]
    for k, f in (("sw_protein", 0.4), ("band_dna", 0.4), ("xdrop_dna", 0.2)):
        assert kinds.count(k) / len(reqs) == pytest.approx(f, abs=0.03)
    lens = np.array([len(r.r) for r in reqs])
    assert lens.min() >= 100 and lens.max() <= 100_000
    assert np.median(lens) == pytest.approx(2000, rel=0.08)
    t = np.array([r.t_arrival for r in reqs])
    assert t[0] == 0.0 and (np.diff(t) >= 0).all()
    assert np.diff(t).mean() == pytest.approx(1e-3, rel=0.05)


def test_long_pair_shape():
    b = synth.long_pair(length=200_000, seg=1000)
    q, r = b.pair(0)
    assert len(r) == 200_000
    assert len(q) == pytest.approx(201_000, rel=0.002)  # single-base ins and del cancel
    assert b.scoring["xdrop"] == 1000


def test_edit_pairs_and_rna():
    b = synth.edit_pairs(32, 2000, 0.3)
    assert (b.r_len == 2000).all() and b.q_len.mean() == pytest.approx(2000, abs=20)
    assert (b.subst == np.where(np.eye(4, dtype=bool), 0, -1)).all()
    seq, off, lens = synth.rna_structured(8, 120)
    assert (lens == 120).all() and len(seq) == 960 and seq.max() < 4
    assert off.tolist() == [120 * i for i in range(8)]


def test_seeded():
    a, b = synth.short_dna_pairs(n=50), synth.short_dna_pairs(n=50)
    assert np.array_equal(a.q_seq, b.q_seq) and np.array_equal(a.r_seq, b.r_seq)
    c = synth.short_dna_pairs(n=50, seed=2)
    assert not np.array_equal(a.r_seq, c.r_seq)
