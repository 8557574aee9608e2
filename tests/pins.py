"""Independent checkers used to pin the oracle (test code only).

Nothing here calls the oracle or the CUDA path: these are brute-force path
enumeration, a textbook two-row Levenshtein distance, and a CIGAR re-scorer.
"""
from __future__ import annotations

import functools

import numpy as np

OPS = {1: "I", 2: "D", 7: "=", 8: "X"}


@functools.lru_cache(maxsize=None)
def all_paths(M: int, N: int):
    """Every monotone path (0,0) -> (M,N) with steps 'M' (i+1, j+1), 'H' (j+1)
    and 'V' (i+1), as tuples.  Their number is the Delannoy number D(M, N)."""
    if M == 0 and N == 0:
        return ((),)
    out = []
    if M > 0 and N > 0:
        out += [p + ("M",) for p in all_paths(M - 1, N - 1)]
    if N > 0:
        out += [p + ("H",) for p in all_paths(M, N - 1)]
    if M > 0:
        out += [p + ("V",) for p in all_paths(M - 1, N)]
    return tuple(out)


def path_score(path, q, r, S, o, e):
    """Score one path: substitution scores on 'M' steps, and o + L*e for every
    maximal run of L equal gap steps ('H' runs and 'V' runs are separate gaps)."""
    i = j = 0
    sc = 0
    prev = None
    for mv in path:
        if mv == "M":
            sc += int(S[q[i]][r[j]])
            i += 1
            j += 1
        elif mv == "H":
            sc -= e + (o if prev != "H" else 0)
            j += 1
        else:
            sc -= e + (o if prev != "V" else 0)
            i += 1
        prev = mv
    return sc


def brute_global(q, r, S, o, e):
    return max(path_score(p, q, r, S, o, e) for p in all_paths(len(q), len(r)))


def mid_ok(path) -> bool:
    """Table 1's M/I/D grammar: I and D open from M only, so a horizontal gap
    step never directly follows or precedes a vertical one."""
    return all({a, b} != {"H", "V"} for a, b in zip(path, path[1:]))


def brute_global_mid(q, r, S, o, e):
    return max(path_score(p, q, r, S, o, e) for p in all_paths(len(q), len(r)) if mid_ok(p))


def brute_local_mid(q, r, S, o, e):
    best = 0
    M, N = len(q), len(r)
    for i0 in range(M + 1):
        for i1 in range(i0, M + 1):
            for j0 in range(N + 1):
                for j1 in range(j0, N + 1):
                    if i1 - i0 == 0 and j1 - j0 == 0:
                        continue
                    best = max(best, brute_global_mid(q[i0:i1], r[j0:j1], S, o, e))
    return best


def brute_local(q, r, S, o, e):
    best = 0  # the empty alignment
    M, N = len(q), len(r)
    for i0 in range(M + 1):
        for i1 in range(i0, M + 1):
            for j0 in range(N + 1):
                for j1 in range(j0, N + 1):
                    if i1 - i0 == 0 and j1 - j0 == 0:
                        continue
                    best = max(best, brute_global(q[i0:i1], r[j0:j1], S, o, e))
    return best


def path_in_band(path, i0, j0, lo, hi) -> bool:
    """Whether every cell a path visits from (i0, j0), its first cell included,
    lies on a diagonal d = j - i with lo <= d <= hi (Sec. 7.1's static band)."""
    i, j = i0, j0
    if not lo <= j - i <= hi:
        return False
    for mv in path:
        if mv != "V":
            j += 1
        if mv != "H":
            i += 1
        if not lo <= j - i <= hi:
            return False
    return True


def brute_global_band(q, r, S, o, e, lo, hi):
    """Best score over the paths (0,0) -> (M,N) that stay inside the band, or
    None when no path does."""
    scores = [path_score(p, q, r, S, o, e) for p in all_paths(len(q), len(r))
              if path_in_band(p, 0, 0, lo, hi)]
    return max(scores) if scores else None


def brute_local_band(q, r, S, o, e, lo, hi):
    """Best score over every path between two cells (i0, j0) <= (i1, j1) that
    stays inside the band, or 0 (the empty alignment)."""
    best = 0
    M, N = len(q), len(r)
    for i0 in range(M + 1):
        for i1 in range(i0, M + 1):
            for j0 in range(N + 1):
                for j1 in range(j0, N + 1):
                    if i1 - i0 == 0 and j1 - j0 == 0:
                        continue
                    for p in all_paths(i1 - i0, j1 - j0):
                        if path_in_band(p, i0, j0, lo, hi):
                            best = max(best, path_score(p, q[i0:i1], r[j0:j1], S, o, e))
    return best


def levenshtein(a, b) -> int:
    """Textbook two-row edit distance (unit substitution / insertion / deletion)."""
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


def rescore_cigar(ops, q, r, S, o, e, q_begin, r_begin):
    """Walk a BAM CIGAR over q[q_begin:], r[r_begin:]; return (score, query
    consumed, reference consumed).  Raises if '=' / 'X' disagree with the codes."""
    i, j, sc = q_begin, r_begin, 0
    for op in np.asarray(ops, dtype=np.uint32).tolist():
        n, c = op >> 4, OPS[op & 15]
        if n <= 0:
            raise AssertionError("empty CIGAR op")
        if c in "=X":
            for _ in range(n):
                if (q[i] == r[j]) != (c == "="):
                    raise AssertionError(f"op {c} at ({i},{j}) disagrees with residues")
                sc += int(S[q[i]][r[j]])
                i += 1
                j += 1
        elif c == "I":
            sc -= o + n * e
            i += n
        else:
            sc -= o + n * e
            j += n
    return sc, i - q_begin, j - r_begin


def cigar_from_str(s: str):
    code = {"I": 1, "D": 2, "=": 7, "X": 8}
    out, num = [], ""
    for ch in s:
        if ch.isdigit():
            num += ch
        else:
            out.append((int(num) << 4) | code[ch])
            num = ""
    return np.array(out, dtype=np.uint32)


# ---- RNA folding ------------------------------------------------------------
RNA_PAIRS = {(0, 3), (3, 0), (1, 2), (2, 1), (2, 3), (3, 2)}  # AU UA CG GC GU UG


def all_structures(n: int, can_pair):
    """Every secondary structure on positions 0..n-1 (sets of non-crossing pairs
    (i, j) with can_pair(i, j)), as tuples of pairs; exponential, for tiny n."""
    def rec(lo, hi):
        if lo >= hi:
            return [()]
        out = [s for s in rec(lo + 1, hi)]  # lo unpaired
        for j in range(lo + 1, hi + 1):
            if can_pair(lo, j):
                for inner in rec(lo + 1, j - 1):
                    for outer in rec(j + 1, hi):
                        out.append(((lo, j),) + inner + outer)
        return out
    return rec(0, n - 1)


def brute_fold(x, min_loop: int) -> int:
    """Largest number of base pairs over all secondary structures."""
    def can(i, j):
        return (int(x[i]), int(x[j])) in RNA_PAIRS and j - i - 1 >= min_loop
    return max(len(s) for s in all_structures(len(x), can))


def check_structure(x, partner, min_loop: int) -> int:
    """Validate a partner array (symmetric, allowed pairs, loops, non-crossing);
    returns its number of pairs."""
    n = len(x)
    pairs = []
    for i in range(n):
        j = int(partner[i])
        if j < 0:
            continue
        assert 0 <= j < n and int(partner[j]) == i, (i, j)
        if i < j:
            assert (int(x[i]), int(x[j])) in RNA_PAIRS, (i, j)
            assert j - i - 1 >= min_loop, (i, j)
            pairs.append((i, j))
    for a, b in pairs:
        for c, d in pairs:
            assert not (a < c < b < d), ((a, b), (c, d))
    return len(pairs)
