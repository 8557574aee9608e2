"""The host planner of filtr_align_batch, run on the CPU through
filtr_test_plan_host: every pair is planned exactly once, the waves cut the
cost-descending order where the traceback budget is used up, the traceback
areas inside a wave are contiguous and disjoint, every group runs one kernel
shape, and empty pairs are set aside (except under X-drop, whose row 0 and
column 0 cells are themselves pruned)."""
import ctypes as C

import numpy as np
import pytest

import synth

UMAX = 0xFFFFFFFF


@pytest.fixture(scope="module")
def L():
    from paper_2607_06225_gb300 import build

    build.build()
    import paper_2607_06225_gb300._lib as lib

    return lib


def plan(L, params, ql, rl, budget):
    n = len(ql)
    ql = np.ascontiguousarray(ql, np.uint32)
    rl = np.ascontiguousarray(rl, np.uint32)
    order = np.zeros(max(n, 1), np.uint32)
    wave = np.zeros(max(n, 1), np.uint32)
    off = np.zeros(max(n, 1), np.uint64)
    words = np.zeros(max(n, 1), np.uint64)
    kernel = np.zeros(max(n, 1), np.uint32)
    info = np.zeros(3 * max(n, 1), np.uint64)
    counts = np.zeros(3, np.uint32)
    ptr = lambda a: a.ctypes.data
    rc = L.lib().filtr_test_plan_host(C.byref(params), n, ptr(ql), ptr(rl), int(budget), ptr(order),
                                      ptr(wave), ptr(off), ptr(words), ptr(kernel), ptr(info),
                                      ptr(counts))
    return rc, dict(order=order[:n], wave=wave[:n], off=off[:n], words=words[:n],
                    kernel=kernel[:n], info=info.reshape(-1, 3)[:int(counts[1])],
                    planned=int(counts[0]), trivial=int(counts[2]))


def band_cells(M, N, B):
    """Cells (i, j), 1 <= i <= M, 1 <= j <= N, on the diagonals of the band
    widened to hold both corners, counted row by row."""
    lo, hi = min(0, N - M) - B, max(0, N - M) + B
    i = np.arange(1, M + 1)
    return int(np.clip(np.minimum(N, i + hi) - np.maximum(1, i + lo) + 1, 0, None).sum())


def check_plan(P, cells, budget, traceback):
    n = len(cells)
    order, wave = P["order"], P["wave"]
    # every pair once: the planned ones, then the ones with nothing to evaluate
    assert P["planned"] + P["trivial"] == n
    assert sorted(order.tolist()) == list(range(n))
    planned = order[:P["planned"]]
    assert (wave[order[P["planned"]:]] == UMAX).all()
    # the waves' slices of the order follow each other and hold their own pairs
    pos = 0
    for w, (tb, begin, end) in enumerate(P["info"].tolist()):
        assert begin == pos and end > begin
        ids = planned[begin:end]
        assert (wave[ids] == w).all()
        if traceback:
            assert tb <= budget
            assert tb == int(P["words"][ids].sum())
            # areas laid out back to back in launch order, from word 0
            assert P["off"][ids[0]] == 0
            assert (P["off"][ids[1:]] == P["off"][ids[:-1]] + P["words"][ids[:-1]]).all()
        else:
            assert tb == 0 and (P["words"][ids] == 0).all()
        # groups: each kernel shape is one contiguous run inside the wave,
        # cost-descending by bucket (a bucket spans less than a factor 1.5)
        k = P["kernel"][ids]
        runs = [k[0]] + [b for a, b in zip(k[:-1], k[1:]) if a != b]
        assert len(runs) == len(set(runs))
        for shape in set(runs):
            c = cells[ids[k == shape]].astype(np.float64)
            assert (c[1:] < 1.5 * np.minimum.accumulate(c)[:-1]).all()
        pos = end
    assert pos == P["planned"]
    # the waves cut one cost-descending order: no pair of a later wave costs
    # more than a bucket above any pair of an earlier one
    for w in range(len(P["info"]) - 1):
        a = cells[planned[int(P["info"][w][1]):int(P["info"][w][2])]]
        b = cells[planned[int(P["info"][w + 1][1]):int(P["info"][w + 1][2])]]
        assert b.max() < 1.5 * a.min()
    if traceback:  # a wave ends where the next pair in cost order would not fit
        for w in range(len(P["info"]) - 1):
            nxt = planned[int(P["info"][w + 1][1]):int(P["info"][w + 1][2])]
            assert int(P["info"][w][0]) + int(P["words"][nxt].max()) > budget


def test_tiled_waves(L):
    rng = np.random.default_rng(5)
    n = 400
    ql = rng.integers(100, 1001, n)
    rl = rng.integers(100, 1001, n)
    S = synth.protein_subst(np.random.default_rng(2))
    p = L.make_params(S, mode="local", gap_open=11, gap_extend=1, traceback=True)
    rc, P = plan(L, p, ql, rl, 1 << 40)
    assert rc == L.OK, L.last_error()
    assert len(P["info"]) == 1  # everything fits one wave
    total = int(P["words"].sum())
    budget = total // 5
    rc, P = plan(L, p, ql, rl, budget)
    assert rc == L.OK, L.last_error()
    assert len(P["info"]) >= 5
    check_plan(P, ql * rl, budget, True)
    fam = P["kernel"] >> 16
    R = (P["kernel"] >> 8) & 0xFF
    assert set(fam.tolist()) <= {0, 3}
    assert all(r in (8, 16, 24, 32) for r in R[fam == 0]) and all(
        8 <= r <= 32 and r % 2 == 0 for r in R[fam == 3])


def test_traceback_off_is_one_wave(L):
    rng = np.random.default_rng(6)
    ql = rng.integers(1, 3000, 200)
    rl = rng.integers(1, 3000, 200)
    p = L.make_params(synth.dna_subst(2, -4), gap_open=4, gap_extend=2, band=40)
    rc, P = plan(L, p, ql, rl, 1)  # no traceback: the budget does not apply
    assert rc == L.OK, L.last_error()
    assert len(P["info"]) == 1
    # banded pairs run the int32 tile; their cost is their band cells
    assert set((P["kernel"] >> 16).tolist()) == {0}
    cells = np.array([band_cells(int(m), int(n), 40) for m, n in zip(ql, rl)], np.int64)
    check_plan(P, cells, 1, False)


@pytest.mark.parametrize("xdrop", [None, 50])
def test_empty_pairs(L, xdrop):
    ql = np.array([0, 5, 0, 7, 300, 0], np.uint32)
    rl = np.array([5, 0, 0, 9, 200, 0], np.uint32)
    p = L.make_params(synth.dna_subst(2, -4), gap_open=4, gap_extend=2, xdrop=xdrop, traceback=True)
    rc, P = plan(L, p, ql, rl, 1 << 40)
    assert rc == L.OK, L.last_error()
    trivial = sorted(P["order"][P["planned"]:].tolist())
    if xdrop is None:
        assert trivial == [0, 1, 2, 5]
    else:  # row 0 / column 0 cells are pruned too: only 0 x 0 has nothing to do
        assert trivial == [2, 5]
        planned = P["order"][:P["planned"]]
        assert set((P["kernel"][planned] >> 16).tolist()) == {1}  # the antidiagonal sweep
        assert ((P["kernel"][planned] >> 8) & 0xFF == 8).all()  # 8 slots per lane


def test_xdrop_waves(L):
    b = synth.long_reads(n=120, lmin=1000, lmax=4000, seed=9)
    ql = np.asarray(b.q_len, np.uint32)
    rl = np.asarray(b.r_len, np.uint32)
    p = L.make_params(synth.dna_subst(2, -4), gap_open=4, gap_extend=2, band=256, xdrop=400,
                      traceback=True)
    rc, P = plan(L, p, ql, rl, 1 << 40)
    assert rc == L.OK, L.last_error()
    budget = int(P["words"].sum()) // 4
    rc, P = plan(L, p, ql, rl, budget)
    assert rc == L.OK, L.last_error()
    assert len(P["info"]) >= 4
    assert set((P["kernel"] >> 16).tolist()) == {1}
    # the sweep's cost is its band cells
    cells = np.array([band_cells(int(m), int(n), 256) for m, n in zip(ql, rl)], np.int64)
    check_plan(P, cells, budget, True)


def test_pair_over_budget_is_refused(L):
    p = L.make_params(synth.dna_subst(2, -4), gap_open=4, gap_extend=2, traceback=True)
    rc, _ = plan(L, p, [2000, 10], [2000, 10], 1000)
    assert rc == L.ERR_NOMEM
    assert "traceback" in L.last_error()


def test_bad_arguments(L):
    p = L.make_params(synth.dna_subst(2, -4), gap_open=4, gap_extend=2)
    lib = L.lib()
    assert lib.filtr_test_plan_host(C.byref(p), 1, None, None, 0, None, None, None, None, None,
                                    None, None) == L.ERR_INVALID
