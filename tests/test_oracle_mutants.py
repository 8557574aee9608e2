"""Plants plausible mistakes in copies of the oracle (on the CPU) and checks that
the pin suite (test_oracle_pins.py) rejects every one of them: a transposed
operand, a dropped term, a wrong sign, each tie-break flipped, the X-drop rule
and domain altered, the Z-drop distance term dropped, signed or anchored, its
best-diagonal tie flipped, the band edge shifted, a neighbour outside the domain
read as zero, the CIGAR op table swapped and the cell counter widened."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "transposed_subst": ("c->p->subst[(int)c->q[i - 1] * a + (int)c->r[j - 1]]",
                         "c->p->subst[(int)c->r[j - 1] * a + (int)c->q[i - 1]]"),
    "E_open_drops_o": ("out->E = (mid ? l->M : l->H) - o - e;", "out->E = (mid ? l->M : l->H) - e;"),
    "F_ext_wrong_sign": ("int64_t ext = u->F - e;", "int64_t ext = u->F + e;"),
    "E_tie_prefers_ext": ("if (!out->vE || ext > out->E) {", "if (!out->vE || ext >= out->E) {"),
    "H_tie_E_over_diag": ("if (out->vE && (!out->vH || out->E > out->H))",
                          "if (out->vE && (!out->vH || out->E >= out->H))"),
    "H_tie_F_over_E": ("if (out->vF && (!out->vH || out->F > out->H))",
                       "if (out->vF && (!out->vH || out->F >= out->H))"),
    "xdrop_running_max": ("if (!c->p->running || nbest > best)", "if (nbest > best)"),
    "running_ties_move_reference": ("if (!c->p->running || nbest > best)",
                                    "if (!c->p->running || nbest >= best)"),
    "xdrop_non_strict": ("tmp.H >= best - X", "tmp.H > best - X"),
    "xdrop_domain_no_growth": ("if (lo - 1 > dl) dl = lo - 1;", "if (lo > dl) dl = lo;"),
    "band_edge_shift": ("c.hi = ((N - M) > 0 ? (N - M) : 0) + p->band;\n    }\n  }\n  memset(res",
                        "c.hi = ((N - M) > 0 ? (N - M) : 0) + p->band - 1;\n    }\n  }\n  memset(res"),
    "diag_op_swapped": ("(c->q[i - 1] == c->r[j - 1]) ? ORC_OP_EQ : ORC_OP_X",
                        "(c->q[i - 1] != c->r[j - 1]) ? ORC_OP_EQ : ORC_OP_X"),
    "E_emits_I": ("mv[n++] = ORC_OP_D;", "mv[n++] = ORC_OP_I;"),
    "zdrop_no_distance": ("const int64_t dist = zdrop ? (d > dbest ? d - dbest : dbest - d) : 0;",
                          "const int64_t dist = 0;"),
    "zdrop_signed_distance": ("(d > dbest ? d - dbest : dbest - d)", "(d - dbest)"),
    "zdrop_tie_smallest_i_flipped": ("(tmp.H == nbest && d > ndbest)", "(tmp.H == nbest && d < ndbest)"),
    "zdrop_best_diagonal_frozen": ("      dbest = ndbest;\n", "\n"),
    "mid_E_opens_from_H": ("out->E = (mid ? l->M : l->H) - o - e;", "out->E = l->H - o - e;"),
    "mid_F_opens_from_H": ("out->F = (mid ? u->M : u->H) - o - e;", "out->F = u->H - o - e;"),
    "mid_walk_skips_forced_diagonal": ("if (!ch.e_ext) state = after_open;",
                                       "if (!ch.e_ext) state = 0;"),
    "missing_left_neighbour_as_zero": ("if (l && (mid ? l->vM : l->vH)) {\n      out->E = (mid ? l->M : l->H) - o - e;",
                                       "if (!l || (mid ? l->vM : l->vH)) {\n      out->E = (l ? (mid ? l->M : l->H) : 0) - o - e;"),
    "cells_count_boundary": ("      if (i >= 1 && j >= 1) ++*cells;\n      if (alive)",
                             "      ++*cells;\n      if (alive)"),
}


SEARCH_MUTANTS = {
    "search_mismatch_no_step": ("v + 1 + d <= c->N) {\n    best = v + 1;",
                                "v + 1 + d <= c->N) {\n    best = v;"),
    "search_insertion_wrong_side": ("wave_get(prev, d + 1, &v)", "wave_get(prev, d - 1, &v)"),
    "search_deletion_steps_row": ("(which < 0 || v > best)) {\n    best = v;",
                                  "(which < 0 || v > best)) {\n    best = v + 1;"),
    "search_domain_frozen_low": ("(w->alo - 1 > dlo) ? w->alo - 1", "(w->alo > dlo) ? w->alo"),
    "search_target_mirrored": ("const int64_t target = N - M;", "const int64_t target = M - N;"),
    "search_extend_short": ("while (i < c->M && i + d < c->N", "while (i + 1 < c->M && i + d < c->N"),
    "search_cells_narrow": ("cells += hi - lo + 1;", "cells += hi - lo;"),
    "search_band_edge": ("- p->band;\n    const int64_t bhi", "- p->band + 1;\n    const int64_t bhi"),
    "adapt_non_strict": ("rmin > p->adapt_max_dist))\n        ++alo;",
                         "rmin >= p->adapt_max_dist))\n        ++alo;"),
    "adapt_min_remaining": ("return a > b ? a : b;", "return a < b ? a : b;"),
    "adapt_keeps_unreached": ("while (alo <= ahi && (!w->reached[alo - w->lo] ||",
                              "while (alo <= ahi && (0 ||"),
    "walk_insertion_moves_down": ("i = row - 1;\n        d = d + 1;", "i = row - 1;\n        d = d - 1;"),
}


FOLD_MUTANTS = {
    "fold_no_wobble": ("(a == 2 && b == 3) || (a == 3 && b == 2)", "0"),
    "fold_min_loop_off_by_one": ("j - i - 1 >= c->p->min_loop && val(c, i + 1, j - 1, &a) &&\n      (!have",
                                 "j - i >= c->p->min_loop && val(c, i + 1, j - 1, &a) &&\n      (!have"),
    "fold_split_skips_odd": ("for (int64_t m = i; m < j; ++m) /* two", "for (int64_t m = i; m < j; m += 2) /* two"),
    "fold_domain_no_growth": ("int64_t dl = lo - 1 > 0 ? lo - 1 : 0", "int64_t dl = lo"),
    "fold_prune_strict": ("f >= best - p->xdrop", "f > best - p->xdrop"),
    "fold_warmup_exclusive": ("k <= p->warmup", "k < p->warmup"),
    "fold_cells_skip_span0": ("int64_t cells = n, lo = 0", "int64_t cells = 0, lo = 0"),
}


def _run_mutant(src_name, pins, a, b, name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", src_name)).read()
    assert src.count(a) >= 1, "mutation site moved; update the mutant"
    ign = shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*")
    for d in ("oracle", "tests", "synth"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d, ignore=ign)
    (tmp_path / "oracle" / src_name).write_text(src.replace(a, b, 1))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        f"tests/{pins}"], capture_output=True, text=True, cwd=tmp_path,
                       timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    a, b = MUTANTS[name]
    _run_mutant("oracle.c", "test_oracle_pins.py", a, b, name, tmp_path)


@pytest.mark.parametrize("name", sorted(SEARCH_MUTANTS))
def test_search_pins_reject_mutant(name, tmp_path):
    a, b = SEARCH_MUTANTS[name]
    _run_mutant("search.c", "test_oracle_search_pins.py", a, b, name, tmp_path)



@pytest.mark.parametrize("name", sorted(FOLD_MUTANTS))
def test_fold_pins_reject_mutant(name, tmp_path):
    a, b = FOLD_MUTANTS[name]
    _run_mutant("fold.c", "test_oracle_fold_pins.py", a, b, name, tmp_path)
