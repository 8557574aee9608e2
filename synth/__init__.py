"""Seeded synthetic workload generators.

This module is shared by the CPU oracle side (tests, CPU baseline) and the CUDA
path (tests, bench).  It draws sequences, substitution matrices and arrival
times only; it contains none of the alignment arithmetic.

Encodings: DNA residues are codes 0..3 (A C G T); protein residues are codes
0..19.  A batch is three parallel arrays per side, the layout the C ABI takes:
concatenated codes (uint8), start offsets (uint64) and lengths (uint32).

The paper measures only synthetic pairs with controlled divergence (Sec. 9.1,
"Experimental Methodology"); the shapes below follow the workloads this library
is benchmarked on (short DNA reads, protein pairs of uneven length, long noisy
reads, a serving mix and one megabase pair).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DNA = 4
PROT = 20


@dataclass
class Batch:
    """A batch of pairs in the C-ABI layout plus the scoring that goes with it."""

    q_seq: np.ndarray  # uint8 codes, all queries concatenated
    q_off: np.ndarray  # uint64 start of each query
    q_len: np.ndarray  # uint32 length of each query
    r_seq: np.ndarray
    r_off: np.ndarray
    r_len: np.ndarray
    alphabet: int  # 4 (DNA) or 20 (protein)
    subst: np.ndarray  # int8 [alphabet, alphabet], row = query code, col = reference code
    scoring: dict = field(default_factory=dict)  # mode / gap_open / gap_extend / band / xdrop ...
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.q_len.shape[0])

    def pair(self, p: int):
        qo, ql = int(self.q_off[p]), int(self.q_len[p])
        ro, rl = int(self.r_off[p]), int(self.r_len[p])
        return self.q_seq[qo:qo + ql], self.r_seq[ro:ro + rl]

    def cells_full(self) -> int:
        return int(np.sum(self.q_len.astype(np.int64) * self.r_len.astype(np.int64)))

    def subset(self, idx) -> "Batch":
        """A new batch holding pairs `idx` (in that order), repacked."""
        idx = np.asarray(idx, dtype=np.int64)
        qs = [self.pair(int(p))[0] for p in idx]
        rs = [self.pair(int(p))[1] for p in idx]
        return pack(qs, rs, self.alphabet, self.subst, dict(self.scoring), self.seed)


def pack(qs, rs, alphabet, subst, scoring=None, seed=0) -> Batch:
    """Concatenate per-pair code arrays into the C-ABI batch layout."""
    ql = np.array([len(x) for x in qs], dtype=np.uint32)
    rl = np.array([len(x) for x in rs], dtype=np.uint32)
    qo = np.zeros(len(qs), dtype=np.uint64)
    ro = np.zeros(len(rs), dtype=np.uint64)
    if len(qs):
        qo[1:] = np.cumsum(ql[:-1], dtype=np.uint64)
        ro[1:] = np.cumsum(rl[:-1], dtype=np.uint64)
    q = np.concatenate([np.asarray(x, dtype=np.uint8) for x in qs]) if len(qs) and ql.sum() else np.zeros(0, np.uint8)
    r = np.concatenate([np.asarray(x, dtype=np.uint8) for x in rs]) if len(rs) and rl.sum() else np.zeros(0, np.uint8)
    return Batch(q, qo, ql, r, ro, rl, alphabet, np.asarray(subst, dtype=np.int8),
                 dict(scoring or {}), seed)


# ---------------------------------------------------------------------------
# scoring tables
# ---------------------------------------------------------------------------

def dna_subst(match: int = 2, mismatch: int = -4) -> np.ndarray:
    s = np.full((DNA, DNA), mismatch, dtype=np.int8)
    np.fill_diagonal(s, match)
    return s


def protein_subst(rng: np.random.Generator) -> np.ndarray:
    """Seeded symmetric 20x20 integer matrix: diagonal U[4,11], off-diagonal U[-4,3]."""
    s = rng.integers(-4, 4, size=(PROT, PROT))  # high is exclusive: values -4..3
    s = np.triu(s, 1)
    s = s + s.T
    np.fill_diagonal(s, rng.integers(4, 12, size=PROT))
    return s.astype(np.int8)


def protein_background(rng: np.random.Generator) -> np.ndarray:
    """A fixed non-uniform residue frequency vector: 20 seeded U[1,10] weights, normalised."""
    w = rng.uniform(1.0, 10.0, size=PROT)
    return w / w.sum()


# ---------------------------------------------------------------------------
# mutation models
# ---------------------------------------------------------------------------

def _geom(rng, p, size):
    return rng.geometric(p, size=size).astype(np.int64)  # support 1, 2, ...


def mutate(rng: np.random.Generator, ref: np.ndarray, p_sub: float, p_ins: float,
           p_del: float, geom_p: float | None, alphabet: int = DNA,
           draw=None) -> np.ndarray:
    """Derive a query from `ref`.

    Each reference base draws at most one event: substitution (a different
    residue, uniform among the others), deletion (this base and, for geometric
    indels, the following ones are dropped) or insertion (new residues are placed
    before this base, which is kept).  `geom_p=None` gives single-base indels.
    `draw(n)` samples inserted residues (uniform by default).
    """
    n = ref.shape[0]
    if draw is None:
        def draw(k):
            return rng.integers(0, alphabet, size=k, dtype=np.int64)
    u = rng.random(n)
    is_sub = u < p_sub
    is_del = (u >= p_sub) & (u < p_sub + p_del)
    is_ins = (u >= p_sub + p_del) & (u < p_sub + p_del + p_ins)
    # substitution: add 1..alphabet-1 modulo alphabet
    shift = rng.integers(1, alphabet, size=n)
    base = ref.astype(np.int64)
    base = np.where(is_sub, (base + shift) % alphabet, base)
    # deletions (possibly runs)
    if geom_p is None:
        del_len = is_del.astype(np.int64)
    else:
        del_len = np.where(is_del, _geom(rng, geom_p, n), 0)
    diff = np.zeros(n + 1, dtype=np.int64)
    starts = np.nonzero(del_len)[0]
    np.add.at(diff, starts, 1)
    np.add.at(diff, np.minimum(starts + del_len[starts], n), -1)
    deleted = np.cumsum(diff[:n]) > 0
    # insertions
    if geom_p is None:
        ins_len = is_ins.astype(np.int64)
    else:
        ins_len = np.where(is_ins, _geom(rng, geom_p, n), 0)
    keep = (~deleted).astype(np.int64)
    counts = ins_len + keep
    total = int(counts.sum())
    out = np.zeros(total, dtype=np.int64)
    if total:
        start = np.cumsum(counts) - counts
        n_ins = int(ins_len.sum())
        if n_ins:
            ins_pos = np.repeat(start, ins_len) + (np.arange(n_ins) - np.repeat(np.cumsum(ins_len) - ins_len, ins_len))
            out[ins_pos] = draw(n_ins)
        kept = keep.astype(bool)
        out[(start + ins_len)[kept]] = base[kept]
    return out.astype(np.uint8)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

def short_dna_pairs(n: int = 1000, length: int = 128, err: float = 0.05, seed: int = 1) -> Batch:
    """Global NW affine, short DNA: reference uniform ACGT of `length`; query =
    reference with `err` errors split equally into substitution / insertion /
    deletion of single bases.  Scoring +2/-4, open 4, extend 2, int32, score only."""
    rng = np.random.default_rng(seed)
    qs, rs = [], []
    for _ in range(n):
        r = rng.integers(0, DNA, size=length).astype(np.uint8)
        q = mutate(rng, r, err / 3, err / 3, err / 3, None)
        qs.append(q)
        rs.append(r)
    return pack(qs, rs, DNA, dna_subst(2, -4),
                dict(mode="global", affine=True, gap_open=4, gap_extend=2, traceback=False), seed)


def protein_pairs(n: int = 100_000, lmin: int = 100, lmax: int = 1000, seed: int = 2,
                  indel_rate: float = 0.02) -> Batch:
    """Local SW affine protein pairs of uneven length.

    Reference length and query length are i.i.d. U[lmin, lmax]; the reference is
    drawn from the background vector.  For each query position p < len(ref) the
    residue copies ref[p] with probability t ~ U[0.3, 0.7] (per pair) and is drawn
    from the background otherwise; positions past the reference end are background.
    Then indel events (rate `indel_rate` per position, half insertions, half
    deletions, lengths geometric p=0.7) are applied so alignments contain gaps.
    Scoring: the seeded 20x20 matrix, open 11, extend 1, traceback on.
    """
    rng = np.random.default_rng(seed)
    subst = protein_subst(rng)
    bg = protein_background(rng)
    cdf = np.cumsum(bg)
    cdf[-1] = 1.0

    def draw(k):
        return np.searchsorted(cdf, rng.random(k), side="right").astype(np.int64)

    lr = rng.integers(lmin, lmax + 1, size=n)
    lq = rng.integers(lmin, lmax + 1, size=n)
    ident = rng.uniform(0.3, 0.7, size=n)
    qs, rs = [], []
    for p in range(n):
        r = draw(int(lr[p]))
        q = draw(int(lq[p]))
        m = min(int(lq[p]), int(lr[p]))
        copy = rng.random(m) < ident[p]
        q[:m] = np.where(copy, r[:m], q[:m])
        q = mutate(rng, q.astype(np.uint8), 0.0, indel_rate / 2, indel_rate / 2, 0.7, PROT, draw)
        if q.shape[0] == 0:
            q = draw(1).astype(np.uint8)
        rs.append(r.astype(np.uint8))
        qs.append(q)
    return pack(qs, rs, PROT, subst,
                dict(mode="local", affine=True, gap_open=11, gap_extend=1, traceback=True), seed)


def long_reads(n: int = 10_000, lmin: int = 10_000, lmax: int = 50_000, seed: int = 3,
               band: int = 256, xdrop: int = 400, idx=None) -> Batch:
    """Banded global alignment of simulated long reads.

    `idx` (optional) selects pairs of the n-pair workload: the batch then holds
    exactly those pairs, identical to the same rows of the full batch.

    Reference uniform ACGT of length U[lmin, lmax].  Query: per reference base an
    insertion event with probability 0.06*0.7, a deletion event 0.03*0.7, a
    substitution 0.01; indel lengths Geometric(0.7) on {1,2,...}, so the expected
    error bases are 6% / 3% / 1%.  Scoring +2/-4, open 4, extend 2, band
    half-width 256, X-drop 400, traceback on.
    """
    rng = np.random.default_rng(seed)
    lens = rng.integers(lmin, lmax + 1, size=n)
    qs, rs = [], []
    for p in (range(n) if idx is None else idx):
        # each pair draws from its own stream, so a sample of the workload can be
        # regenerated without the rest of it
        prng = np.random.default_rng((seed, int(p)))
        r = prng.integers(0, DNA, size=int(lens[p])).astype(np.uint8)
        q = mutate(prng, r, 0.01, 0.06 * 0.7, 0.03 * 0.7, 0.7)
        qs.append(q)
        rs.append(r)
    return pack(qs, rs, DNA, dna_subst(2, -4),
                dict(mode="global", affine=True, gap_open=4, gap_extend=2, band=band,
                     xdrop=xdrop, traceback=True), seed)


def long_pair(length: int = 1_000_000, div: float = 0.01, seg: int = 5000, seed: int = 5,
              xdrop: int = 1000) -> Batch:
    """One long pair: reference uniform ACGT; query = reference at `div` divergence
    (equal single-base substitution / insertion / deletion) plus one `seg`-base
    uniform random segment inserted at a seeded position in [25%, 75%] of the query.
    Global affine DNA with X-drop, traceback on."""
    rng = np.random.default_rng(seed)
    r = rng.integers(0, DNA, size=length).astype(np.uint8)
    q = mutate(rng, r, div / 3, div / 3, div / 3, None)
    if seg > 0:
        pos = int(rng.integers(len(q) // 4, 3 * len(q) // 4 + 1))
        q = np.concatenate([q[:pos], rng.integers(0, DNA, size=seg).astype(np.uint8), q[pos:]])
    return pack([q], [r], DNA, dna_subst(2, -4),
                dict(mode="global", affine=True, gap_open=4, gap_extend=2, xdrop=xdrop,
                     traceback=True), seed)


@dataclass
class ServeRequest:
    t_arrival: float  # seconds from the start of the run
    kind: str  # "sw_protein" | "band_dna" | "xdrop_dna"
    q: np.ndarray
    r: np.ndarray


def serve_mix(n_req: int, rate_hz: float, seed: int = 4, median: float = 2000.0,
              sigma: float = 1.0, lmin: int = 100, lmax: int = 100_000):
    """Poisson arrivals at `rate_hz`; each request one pair of log-normal length
    (median 2000, sigma 1.0, clipped to [100, 100000]); kind drawn 40% SW protein,
    40% banded NW DNA (band 256, no X-drop), 20% X-drop DNA (X = 400, no band).
    Protein queries follow the protein-pair model (identity U[0.3, 0.7], no
    indels); DNA queries follow the long-read error model."""
    rng = np.random.default_rng(seed)
    prng = np.random.default_rng(2)  # the same matrix and background as the protein batch
    psub = protein_subst(prng)
    bg = protein_background(prng)
    cdf = np.cumsum(bg)
    cdf[-1] = 1.0
    gaps = rng.exponential(1.0 / rate_hz, size=n_req)
    t = np.cumsum(gaps) - gaps[0]
    lens = np.clip(np.round(rng.lognormal(np.log(median), sigma, size=n_req)), lmin, lmax).astype(np.int64)
    kind_u = rng.random(n_req)
    out = []
    for k in range(n_req):
        L = int(lens[k])
        if kind_u[k] < 0.4:
            r = np.searchsorted(cdf, rng.random(L), side="right").astype(np.uint8)
            q = np.searchsorted(cdf, rng.random(L), side="right").astype(np.uint8)
            ident = rng.uniform(0.3, 0.7)
            copy = rng.random(L) < ident
            q = np.where(copy, r, q).astype(np.uint8)
            out.append(ServeRequest(float(t[k]), "sw_protein", q, r))
        else:
            r = rng.integers(0, DNA, size=L).astype(np.uint8)
            q = mutate(rng, r, 0.01, 0.06 * 0.7, 0.03 * 0.7, 0.7)
            if q.shape[0] == 0:
                q = rng.integers(0, DNA, size=1).astype(np.uint8)
            out.append(ServeRequest(float(t[k]), "band_dna" if kind_u[k] < 0.8 else "xdrop_dna", q, r))
    return out, psub


def edit_pairs(n: int, length: int, div: float, seed: int = 6) -> Batch:
    """Edit-distance pairs of the search-versus-antidiagonal comparison (Sec. 9.4's
    synthetic pairs at 1 / 5 / 30% divergence): reference uniform ACGT of
    `length`; query = reference with `div` divergence split equally into
    single-base substitutions, insertions and deletions.  The scoring given is
    unit-cost global alignment (match 0, mismatch -1, linear gap 1), whose
    score is minus the edit distance."""
    rng = np.random.default_rng(seed)
    qs, rs = [], []
    for _ in range(n):
        r = rng.integers(0, DNA, size=length).astype(np.uint8)
        qs.append(mutate(rng, r, div / 3, div / 3, div / 3, None))
        rs.append(r)
    unit = np.where(np.eye(DNA, dtype=bool), 0, -1).astype(np.int8)
    return pack(qs, rs, DNA, unit,
                dict(mode="global", affine=False, gap_open=0, gap_extend=1, traceback=False), seed)


def rna_structured(n: int, length: int, seed: int = 7, stems: int | None = None):
    """Synthetic RNAs for the folding transfer (Sec. 9.5's four RNA classes of
    76-500 bases stand-in): uniform ACGU (codes A=0 C=1 G=2 U=3), then
    `stems` hairpin stems planted -- a segment of 4-10 bases and, 4-40 bases
    further on, its reverse complement -- so the folds have nested helices.
    Returns (codes, offsets, lengths) of n sequences of `length` bases."""
    rng = np.random.default_rng(seed)
    comp = np.array([3, 2, 1, 0], np.uint8)  # A<->U, C<->G
    if stems is None:
        stems = max(1, length // 40)
    seqs = []
    for _ in range(n):
        x = rng.integers(0, 4, size=length).astype(np.uint8)
        for _s in range(stems):
            L = int(rng.integers(4, 11))
            loop = int(rng.integers(4, 41))
            if 2 * L + loop > length:
                continue
            a = int(rng.integers(0, length - 2 * L - loop + 1))
            b = a + L + loop
            x[b:b + L] = comp[x[a:a + L][::-1]]
        seqs.append(x)
    lens = np.full(n, length, dtype=np.uint32)
    off = np.zeros(n, dtype=np.uint64)
    if n:
        off[1:] = np.cumsum(lens[:-1].astype(np.uint64))
    return (np.concatenate(seqs) if n else np.zeros(0, np.uint8)), off, lens


def random_pairs(n: int, mmax: int, nmax: int, alphabet: int, seed: int, mmin: int = 0,
                 nmin: int = 0, related: float = 0.5) -> tuple[list, list]:
    """Small random pairs for parity tests: lengths uniform in [min, max]; with
    probability `related` the query is derived from the reference (so alignments
    have long matching runs), otherwise both are independent."""
    rng = np.random.default_rng(seed)
    qs, rs = [], []
    for _ in range(n):
        N = int(rng.integers(nmin, nmax + 1))
        r = rng.integers(0, alphabet, size=N).astype(np.uint8)
        if rng.random() < related and N > 0:
            q = mutate(rng, r, 0.1, 0.05, 0.05, 0.7, alphabet)
            M = int(rng.integers(mmin, mmax + 1))
            q = q[:M] if q.shape[0] >= M else np.concatenate(
                [q, rng.integers(0, alphabet, size=M - q.shape[0]).astype(np.uint8)])
        else:
            M = int(rng.integers(mmin, mmax + 1))
            q = rng.integers(0, alphabet, size=M).astype(np.uint8)
        qs.append(q.astype(np.uint8))
        rs.append(r)
    return qs, rs
