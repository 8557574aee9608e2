/* oracle.h -- plain CPU oracle for pruned pairwise alignment.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this code.  It shares nothing with the CUDA path:
 * no header, no helper, no table.
 *
 * What it computes (integer scores, int64 arithmetic, explicit validity flags
 * in place of an infinity sentinel):
 *   - the alignment recurrence of the paper's edit-distance example (Sec. 2)
 *     generalised to substitution scores and gap costs, in two gap models:
 *       linear : H = max(H[i-1][j-1] + s, H[i][j-1] - e, H[i-1][j] - e)
 *       affine : Gotoh H/E/F  (Table 1 "Sequence Alignment", Sec. 3; the H/E/F
 *                form lets E and F open from H, so an insertion may touch a
 *                deletion -- see the reading list in the design notes), or
 *                Table 1's own M/I/D form: M = max(M, I, D)(i-1, j-1) + s,
 *                I and D open from M only (H = max(M, I, D) is the cell's score)
 *     global (Needleman-Wunsch) or local (Smith-Waterman, H floored at 0);
 *   - a static band as a prune axis  lo <= diag(i,j) <= hi  (Sec. 7.1);
 *   - X-drop as a dynamic prune (Sec. 5.2 conditional definition and the
 *     diag_lo / diag_hi domain recurrences; Sec. 7.2), read as: a cell on
 *     antidiagonal k is pruned when H < best(k-1) - X, best(k-1) being the
 *     largest unpruned H on antidiagonal k-1; the next antidiagonal covers the
 *     diagonals [lo_k - 1, hi_k + 1] of the unpruned cells of k;
 *   - Z-drop (Sec. 9.3's pruning condition): as X-drop, but a cell on antidiagonal
 *     k is pruned when best(k-1) - H > Z + |diag(i,j) - diag_best(k-1)|,
 *     diag_best(k-1) being the diagonal of antidiagonal k-1's best cell (the
 *     largest H; among equal H the smallest i, i.e. the largest diagonal);
 *   - the running variant of both (the BLAST-style reading of Sec. 9.3's "best
 *     score seen so far"): best is the largest best(t) over t <= k-1, and for
 *     Z-drop the reference diagonal is that of the antidiagonal that first
 *     reached it;
 *   - traceback with fixed tie-breaks, emitted as a SAM/BAM CIGAR.
 *   - edit distance by the search traversal (Sec. 6.3): the furthest row
 *     F[s][d] reached on diagonal d = j - i with s edits, from the three shifted
 *     terms of wavefront s-1 and a greedy run of matches; optionally inside a
 *     static band (Sec. 7.1 maps the band to d) and with WFA-Adapt trimming
 *     (Sec. 7.2, 9.3), read as: once a wavefront spans at least min_len
 *     diagonals, its domain bounds move inwards past every diagonal whose
 *     remaining distance max(M - i, N - j) exceeds the smallest one on the
 *     wavefront by more than max_dist.
 * Parity of the tie-break order and of the X-drop domain reading is pinned only
 * by hand-worked examples (the paper does not fix them); the search's distance is
 * pinned by the plain edit distance, its CIGAR choice and the WFA-Adapt reading
 * are not pinned beyond validity (parity unpinned).
 */
#ifndef FILTR_ORACLE_H
#define FILTR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t mode;        /* 0 global (NW), 1 local (SW) */
  int32_t affine;      /* 1 Gotoh H/E/F, 0 linear gap */
  int64_t gap_open;    /* o >= 0: a gap of length L costs o + L*e (affine), L*e (linear) */
  int64_t gap_extend;  /* e >= 0 */
  int32_t alphabet;    /* 4 or 20 (any 1..255 accepted) */
  const int8_t *subst; /* alphabet*alphabet, subst[q*alphabet + r] */
  int32_t use_band;    /* 1: band prune axis */
  int32_t band_literal;/* 1: lo = -B, hi = +B; 0: widened to hold both corners */
  int64_t band;        /* half-width B >= 0 */
  int32_t use_xdrop;   /* 1: X-drop */
  int64_t xdrop;       /* X >= 0; INT64_MAX means no threshold */
  int32_t traceback;   /* 1: emit CIGAR and begin coordinates */
  int32_t order;       /* evaluation order for unpruned / banded runs: 0 row-major, 1 antidiagonal */
  int32_t zdrop;       /* with use_xdrop: 1 = Z-drop with Z = xdrop (distance term added) */
  int32_t running;     /* with use_xdrop: 1 = the threshold follows the best score of every
                          antidiagonal so far (running maximum) instead of antidiagonal k-1's */
  int32_t mid;         /* with affine: 1 = Table 1's M/I/D form: gaps open from M (the
                          diagonal state) only, so a deletion never touches an insertion */
} orc_params;

typedef struct {
  int64_t score;
  int64_t q_begin, q_end, r_begin, r_end; /* residues [begin, end); end = last cell's i / j */
  int32_t status;   /* 0 OK, 1 DROPPED, 2 UNREACHABLE, 3 EMPTY */
  int64_t cells;    /* evaluated cells with i >= 1 and j >= 1 */
  int64_t n_ops;    /* CIGAR ops written (or needed, if cap was too small) */
  int64_t last_k;   /* last antidiagonal evaluated (X-drop), else M+N */
} orc_result;

enum { ORC_OK = 0, ORC_DROPPED = 1, ORC_UNREACHABLE = 2, ORC_EMPTY = 3 };
enum { ORC_OP_I = 1, ORC_OP_D = 2, ORC_OP_EQ = 7, ORC_OP_X = 8 };

/* Align one pair.  ops (may be NULL) receives up to cap uint32 BAM ops
 * (len << 4 | op).  Returns 0, or -1 on invalid arguments / out of memory. */
int orc_align(const orc_params *p, const uint8_t *q, int64_t M, const uint8_t *r,
              int64_t N, orc_result *res, uint32_t *ops, int64_t cap);

/* Align n pairs with nthreads worker threads (one pair per task).  Layout as the
 * batch C ABI: concatenated codes, offsets, lengths.  ops_off[p] is where pair p
 * writes its CIGAR inside ops; ops_cap[p] its capacity.  Returns 0 or -1. */
int orc_align_batch(const orc_params *p, int64_t n, const uint8_t *q_seq,
                    const uint64_t *q_off, const uint32_t *q_len, const uint8_t *r_seq,
                    const uint64_t *r_off, const uint32_t *r_len, orc_result *res,
                    uint32_t *ops, const uint64_t *ops_off, const uint64_t *ops_cap,
                    int nthreads);

/* Debug view: after an unpruned / banded / X-drop run on one pair, write the
 * evaluated cells (i, j) (i >= 1, j >= 1 excluded from nothing: every domain
 * cell, boundary included) into cells_ij (pairs of int64), at most cap cells;
 * also a flag per cell, 1 if it was left unpruned.  Returns the cell count. */
int64_t orc_domain(const orc_params *p, const uint8_t *q, int64_t M, const uint8_t *r,
                   int64_t N, int64_t *cells_ij, uint8_t *alive, int64_t cap);

typedef struct {
  int32_t traceback;   /* 1: emit the CIGAR */
  int32_t use_band;    /* 1: diagonals restricted to [min(0,N-M) - band, max(0,N-M) + band] */
  int64_t band;
  int64_t adapt_min_len;  /* 0: exact search; else WFA-Adapt from this wavefront width */
  int64_t adapt_max_dist;
} orc_search_params;

typedef struct {
  int64_t distance;   /* edits of the alignment found (the edit distance when exact) */
  int64_t cells;      /* wavefront entries evaluated: sum over s of the domain's width */
  int64_t n_ops;      /* CIGAR ops written (or needed, if cap was too small) */
} orc_search_result;

/* Edit distance of one pair by the search traversal.  ops as in orc_align.
 * Returns 0, or -1 on invalid arguments / out of memory. */
int orc_search(const orc_search_params *p, const uint8_t *q, int64_t M, const uint8_t *r,
               int64_t N, orc_search_result *res, uint32_t *ops, int64_t cap);

/* orc_search over n pairs on nthreads threads (layout as orc_align_batch). */
int orc_search_batch(const orc_search_params *p, int64_t n, const uint8_t *q_seq,
                     const uint64_t *q_off, const uint32_t *q_len, const uint8_t *r_seq,
                     const uint64_t *r_off, const uint32_t *r_len, orc_search_result *res,
                     uint32_t *ops, const uint64_t *ops_off, const uint64_t *ops_cap,
                     int nthreads);

/* Nussinov folding (Table 1, RNA folding) with X-drop transferred to it
 * (Sec. 9.5); fold.c states the readings. */
typedef struct {
  int64_t min_loop;   /* a pair (i, j) needs j - i - 1 >= min_loop */
  int32_t use_xdrop;  /* 1: X-drop on the span wavefronts */
  int64_t xdrop;      /* X >= 0 */
  int64_t warmup;     /* spans <= warmup are never pruned */
  int32_t traceback;  /* 1: fill partner[] */
} orc_fold_params;

typedef struct {
  int64_t score;       /* F of the end cell: base pairs of the fold */
  int64_t i_end, j_end;
  int32_t status;      /* ORC_OK, or ORC_DROPPED (the end cell is the best unpruned one) */
  int64_t cells;       /* cells evaluated, span 0 included */
  int64_t last_k;      /* last span evaluated */
} orc_fold_result;

/* Fold one RNA (codes A=0 C=1 G=2 U=3).  partner (n entries, may be NULL)
 * receives each base's partner or -1.  Returns 0 or -1 (bad arguments). */
int orc_fold(const orc_fold_params *p, const uint8_t *x, int64_t n, orc_fold_result *res,
             int32_t *partner);
int orc_fold_batch(const orc_fold_params *p, int64_t n, const uint8_t *seq, const uint64_t *off,
                   const uint32_t *len, orc_fold_result *res, int32_t *partner, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
