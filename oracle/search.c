/* search.c -- edit distance by the search traversal (Sec. 6.3), plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
 * benchmark).  Nothing here is shared with the CUDA path.
 *
 * The edit-distance recurrence F(i,j) = min(F(i-1,j-1) + [q_i != r_j],
 * F(i-1,j) + 1, F(i,j-1) + 1) turned score-major: F[s][d] is the furthest row i
 * on diagonal d = j - i that s edits reach,
 *
 *   F[s][d] = extend(max(F[s-1][d] + 1, F[s-1][d+1] + 1, F[s-1][d-1]))
 *
 * (mismatch, insertion = a step down from diagonal d+1, deletion = a step right
 * from diagonal d-1), extend() following matches for free; the domain of s is
 * one diagonal wider on each side than that of s-1, and the search stops at the
 * first s with F[s][N-M] >= M.  Readings where the paper is silent (each one is
 * listed in the design notes):
 *   - a term exists only when its predecessor was reached and the move stays
 *     inside the matrix (row <= M, column <= N); a diagonal with no term is
 *     unreached;
 *   - the domain never leaves the matrix (-M <= d <= N) nor, when a band is
 *     asked for, the widened band of the alignment kernels (Sec. 7.1 maps the
 *     band to d);
 *   - WFA-Adapt (Sec. 7.2, 9.3): once wavefront s spans at least min_len
 *     diagonals, its domain bounds move inwards past every reached diagonal
 *     whose remaining distance max(M - i, N - j) exceeds the wavefront's
 *     smallest by more than max_dist (and past unreached ones); diagonals outside
 *     the moved bounds feed nothing, and the domain of s+1 grows from them;
 *   - the CIGAR: walking back from (M, N), each level takes the first of
 *     mismatch, insertion, deletion that gives the level's value.
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  int64_t lo, hi;    /* diagonals evaluated at this score */
  int64_t alo, ahi;  /* diagonals that may feed the next score (WFA-Adapt moves these) */
  int64_t *F;        /* furthest row, F[d - lo] */
  uint8_t *reached;  /* 0 where no term reached a cell */
} wave_t;

typedef struct {
  const uint8_t *q, *r;
  int64_t M, N;
  wave_t *w;
  int64_t nw, capw;
} sctx_t;

static int wave_get(const wave_t *w, int64_t d, int64_t *out) {
  if (d < w->alo || d > w->ahi) return 0;
  if (!w->reached[d - w->lo]) return 0;
  *out = w->F[d - w->lo];
  return 1;
}

/* free transitions: matches along diagonal d from row i */
static int64_t extend(const sctx_t *c, int64_t i, int64_t d) {
  while (i < c->M && i + d < c->N && c->q[i] == c->r[i + d]) ++i;
  return i;
}

/* Largest term of F[s][d] from wavefront prev; *row receives it.  Returns 0
 * (mismatch), 1 (insertion) or 2 (deletion), the first in that order on ties,
 * or -1 when no term exists. */
static int terms(const sctx_t *c, const wave_t *prev, int64_t d, int64_t *row) {
  int which = -1;
  int64_t best = 0, v;
  if (wave_get(prev, d, &v) && v + 1 <= c->M && v + 1 + d <= c->N) {
    best = v + 1;
    which = 0;
  }
  if (wave_get(prev, d + 1, &v) && v + 1 <= c->M && (which < 0 || v + 1 > best)) {
    best = v + 1;
    which = 1;
  }
  if (wave_get(prev, d - 1, &v) && v + d <= c->N && (which < 0 || v > best)) {
    best = v;
    which = 2;
  }
  *row = best;
  return which;
}

static wave_t *new_wave(sctx_t *c, int64_t lo, int64_t hi) {
  if (c->nw == c->capw) {
    int64_t nc = c->capw ? 2 * c->capw : 64;
    wave_t *w = (wave_t *)realloc(c->w, (size_t)nc * sizeof(wave_t));
    if (!w) return NULL;
    c->w = w;
    c->capw = nc;
  }
  wave_t *w = &c->w[c->nw];
  w->lo = w->alo = lo;
  w->hi = w->ahi = hi;
  w->F = (int64_t *)calloc((size_t)(hi - lo + 1), sizeof(int64_t));
  w->reached = (uint8_t *)calloc((size_t)(hi - lo + 1), 1);
  if (!w->F || !w->reached) {
    free(w->F);
    free(w->reached);
    return NULL;
  }
  ++c->nw;
  return w;
}

static void free_waves(sctx_t *c) {
  for (int64_t s = 0; s < c->nw; ++s) {
    free(c->w[s].F);
    free(c->w[s].reached);
  }
  free(c->w);
}

static int64_t remaining(const sctx_t *c, int64_t i, int64_t d) {
  const int64_t a = c->M - i, b = c->N - (i + d);
  return a > b ? a : b;
}

int orc_search(const orc_search_params *p, const uint8_t *q, int64_t M, const uint8_t *r,
               int64_t N, orc_search_result *res, uint32_t *ops, int64_t cap) {
  if (!p || !res || M < 0 || N < 0 || (p->use_band && p->band < 0) || p->adapt_min_len < 0 ||
      p->adapt_max_dist < 0 || (M > 0 && !q) || (N > 0 && !r))
    return -1;
  memset(res, 0, sizeof *res);
  sctx_t c;
  memset(&c, 0, sizeof c);
  c.q = q;
  c.r = r;
  c.M = M;
  c.N = N;
  int64_t dlo = -M, dhi = N;
  if (p->use_band) {
    const int64_t blo = ((N - M) < 0 ? (N - M) : 0) - p->band;
    const int64_t bhi = ((N - M) > 0 ? (N - M) : 0) + p->band;
    if (blo > dlo) dlo = blo;
    if (bhi < dhi) dhi = bhi;
  }
  const int64_t target = N - M;

  /* score 0: the origin, then its run of matches */
  wave_t *w = new_wave(&c, 0, 0);
  if (!w) return -1;
  w->F[0] = extend(&c, 0, 0);
  w->reached[0] = 1;
  int64_t cells = 1, s = 0;
  for (;;) {
    w = &c.w[s];
    if (target >= w->lo && target <= w->hi && w->reached[target - w->lo] &&
        w->F[target - w->lo] >= M)
      break;
    if (p->adapt_min_len > 0 && w->hi - w->lo + 1 >= p->adapt_min_len) {
      int64_t rmin = -1;
      for (int64_t d = w->lo; d <= w->hi; ++d)
        if (w->reached[d - w->lo]) {
          const int64_t rd = remaining(&c, w->F[d - w->lo], d);
          if (rmin < 0 || rd < rmin) rmin = rd;
        }
      int64_t alo = w->lo, ahi = w->hi;
      while (alo <= ahi && (!w->reached[alo - w->lo] ||
                            remaining(&c, w->F[alo - w->lo], alo) - rmin > p->adapt_max_dist))
        ++alo;
      while (ahi >= alo && (!w->reached[ahi - w->lo] ||
                            remaining(&c, w->F[ahi - w->lo], ahi) - rmin > p->adapt_max_dist))
        --ahi;
      w->alo = alo;
      w->ahi = ahi;
    }
    const int64_t lo = (w->alo - 1 > dlo) ? w->alo - 1 : dlo;
    const int64_t hi = (w->ahi + 1 < dhi) ? w->ahi + 1 : dhi;
    if (s >= M + N + 1 || lo > hi) { /* cannot happen: the leading diagonal always advances */
      free_waves(&c);
      return -1;
    }
    wave_t *nw = new_wave(&c, lo, hi);
    if (!nw) {
      free_waves(&c);
      return -1;
    }
    const wave_t *prev = &c.w[s];
    for (int64_t d = lo; d <= hi; ++d) {
      int64_t row;
      if (terms(&c, prev, d, &row) >= 0) {
        nw->F[d - lo] = extend(&c, row, d);
        nw->reached[d - lo] = 1;
      }
    }
    cells += hi - lo + 1;
    ++s;
  }
  res->distance = s;
  res->cells = cells;

  if (p->traceback) {
    uint8_t *mv = (uint8_t *)malloc((size_t)(M + N + 1));
    if (!mv) {
      free_waves(&c);
      return -1;
    }
    int64_t n = 0, d = target, i = M;
    for (int64_t t = s; t > 0; --t) {
      int64_t row;
      const int which = terms(&c, &c.w[t - 1], d, &row);
      for (int64_t k = row; k < i; ++k) mv[n++] = ORC_OP_EQ;
      if (which == 0) {
        mv[n++] = ORC_OP_X;
        i = row - 1;
      } else if (which == 1) {
        mv[n++] = ORC_OP_I;
        i = row - 1;
        d = d + 1;
      } else {
        mv[n++] = ORC_OP_D;
        i = row;
        d = d - 1;
      }
    }
    for (int64_t k = 0; k < i; ++k) mv[n++] = ORC_OP_EQ; /* score 0: d == 0 */
    int64_t nops = 0, t = n - 1;
    while (t >= 0) {
      const uint8_t op = mv[t];
      int64_t len = 0;
      while (t >= 0 && mv[t] == op) {
        ++len;
        --t;
      }
      if (ops && nops < cap) ops[nops] = (uint32_t)((len << 4) | op);
      ++nops;
    }
    res->n_ops = nops;
    free(mv);
  }
  free_waves(&c);
  return 0;
}

typedef struct {
  const orc_search_params *p;
  int64_t n;
  const uint8_t *q_seq, *r_seq;
  const uint64_t *q_off, *r_off, *ops_off, *ops_cap;
  const uint32_t *q_len, *r_len;
  orc_search_result *res;
  uint32_t *ops;
  int64_t next;
  int err;
  pthread_mutex_t mu;
} spool_t;

static void *sworker(void *arg) {
  spool_t *w = (spool_t *)arg;
  for (;;) {
    pthread_mutex_lock(&w->mu);
    const int64_t t = w->next++;
    pthread_mutex_unlock(&w->mu);
    if (t >= w->n) break;
    uint32_t *o = w->ops ? w->ops + w->ops_off[t] : NULL;
    const int64_t cap = w->ops ? (int64_t)w->ops_cap[t] : 0;
    if (orc_search(w->p, w->q_seq + w->q_off[t], w->q_len[t], w->r_seq + w->r_off[t],
                   w->r_len[t], &w->res[t], o, cap)) {
      pthread_mutex_lock(&w->mu);
      w->err = 1;
      pthread_mutex_unlock(&w->mu);
    }
  }
  return NULL;
}

int orc_search_batch(const orc_search_params *p, int64_t n, const uint8_t *q_seq,
                     const uint64_t *q_off, const uint32_t *q_len, const uint8_t *r_seq,
                     const uint64_t *r_off, const uint32_t *r_len, orc_search_result *res,
                     uint32_t *ops, const uint64_t *ops_off, const uint64_t *ops_cap,
                     int nthreads) {
  spool_t w;
  memset(&w, 0, sizeof w);
  w.p = p;
  w.n = n;
  w.q_seq = q_seq;
  w.q_off = q_off;
  w.q_len = q_len;
  w.r_seq = r_seq;
  w.r_off = r_off;
  w.r_len = r_len;
  w.res = res;
  w.ops = ops;
  w.ops_off = ops_off;
  w.ops_cap = ops_cap;
  pthread_mutex_init(&w.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  pthread_t *th = (pthread_t *)malloc((size_t)nthreads * sizeof(pthread_t));
  if (!th) return -1;
  int started = 0;
  for (int t = 0; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, sworker, &w) == 0) ++started;
  if (started == 0) sworker(&w);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&w.mu);
  return w.err ? -1 : 0;
}
