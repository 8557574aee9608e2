/* oracle.c -- plain, slow CPU oracle for pruned pairwise alignment.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
 * benchmark).  Nothing here is shared with the CUDA path.
 *
 * Every evaluated cell is kept (int64 H, E, F plus a validity flag each), so the
 * traceback re-derives each choice from the stored neighbours with the same
 * function that produced the cell.  Cells are stored per antidiagonal k = i + j
 * at diagonal d = j - i (the sheared layout of Sec. 6.2: i = k - m, j = m with
 * m = j); row-major evaluation writes into the same store.
 *
 * Conventions (the paper leaves them open; each is one reading, listed in the
 * design notes):
 *   - a gap of length L costs o + L*e (affine) or L*e (linear);
 *   - E is the horizontal gap state (consumes the reference, CIGAR 'D'),
 *     F the vertical one (consumes the query, CIGAR 'I');
 *   - boundary cells (row 0 / column 0) follow the same recurrence with the
 *     missing neighbours invalid; (0,0) holds H = 0;
 *   - H's source on ties: diagonal, then E, then F; local H == 0 is a stop;
 *     E / F prefer opening over extending on ties;
 *   - best cell: largest H, then smallest i, then smallest j.
 */
#include "oracle.h"

#include <limits.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int64_t H, E, F, M; /* M: the diagonal candidate H(i-1,j-1) + s (Table 1's M state) */
  uint8_t vH, vE, vF, alive, vM;
  uint8_t pad[3];
} cell_t;

typedef struct {
  int64_t M, N;
  int64_t nk;       /* antidiagonals with a stored range: 0 .. nk-1 */
  int64_t *dlo, *dhi;
  int64_t *base;
  cell_t *cells;
  int64_t ncells, cap;
} store_t;

typedef struct {
  const orc_params *p;
  const uint8_t *q, *r;
  int64_t M, N;
  int64_t lo, hi; /* band on d = j - i */
  store_t st;
} ctx_t;

/* choice made at one cell */
typedef struct {
  int src;   /* 0 diagonal, 1 E, 2 F, 3 zero (local stop), -1 none */
  int e_ext; /* E took the extension */
  int f_ext; /* F took the extension */
} choice_t;

/* smallest value >= a with the parity of k */
static int64_t up_to_parity(int64_t a, int64_t k) { return (((a - k) % 2) == 0) ? a : a + 1; }
/* largest value <= a with the parity of k */
static int64_t down_to_parity(int64_t a, int64_t k) { return (((a - k) % 2) == 0) ? a : a - 1; }

static cell_t *get(ctx_t *c, int64_t i, int64_t j) {
  if (i < 0 || j < 0 || i > c->M || j > c->N) return NULL;
  int64_t k = i + j, d = j - i;
  if (k >= c->st.nk) return NULL;
  if (d < c->st.dlo[k] || d > c->st.dhi[k]) return NULL;
  return &c->st.cells[c->st.base[k] + (d - c->st.dlo[k]) / 2];
}

static int64_t subst(ctx_t *c, int64_t i, int64_t j) {
  int a = c->p->alphabet;
  return (int64_t)c->p->subst[(int)c->q[i - 1] * a + (int)c->r[j - 1]];
}

/* Evaluate the recurrence at (i, j) from the stored neighbours; write H/E/F and
 * validity into *out and the tie-broken choices into *ch. */
static void eval_cell(ctx_t *c, int64_t i, int64_t j, cell_t *out, choice_t *ch) {
  const orc_params *p = c->p;
  const int64_t o = p->affine ? p->gap_open : 0, e = p->gap_extend;
  memset(out, 0, sizeof *out);
  ch->src = -1;
  ch->e_ext = 0;
  ch->f_ext = 0;
  if (i == 0 && j == 0) {
    out->H = 0;
    out->vH = 1;
    out->M = 0; /* the origin is where every path starts in the M state */
    out->vM = 1;
    ch->src = 3;
    return;
  }
  const int mid = p->affine && p->mid; /* gaps open from M instead of H */
  /* E: horizontal gap ending at (i, j), from (i, j-1) */
  if (j >= 1) {
    cell_t *l = get(c, i, j - 1);
    if (l && (mid ? l->vM : l->vH)) {
      out->E = (mid ? l->M : l->H) - o - e;
      out->vE = 1;
    }
    if (p->affine && l && l->vE) {
      int64_t ext = l->E - e;
      if (!out->vE || ext > out->E) { /* strict: ties keep the opening */
        out->E = ext;
        out->vE = 1;
        ch->e_ext = 1;
      }
    }
  }
  /* F: vertical gap ending at (i, j), from (i-1, j) */
  if (i >= 1) {
    cell_t *u = get(c, i - 1, j);
    if (u && (mid ? u->vM : u->vH)) {
      out->F = (mid ? u->M : u->H) - o - e;
      out->vF = 1;
    }
    if (p->affine && u && u->vF) {
      int64_t ext = u->F - e;
      if (!out->vF || ext > out->F) {
        out->F = ext;
        out->vF = 1;
        ch->f_ext = 1;
      }
    }
  }
  /* H: diagonal, then E, then F (first maximum wins) */
  if (i >= 1 && j >= 1) {
    cell_t *g = get(c, i - 1, j - 1);
    if (g && g->vH) {
      out->H = g->H + subst(c, i, j);
      out->vH = 1;
      out->M = out->H;
      out->vM = 1;
      ch->src = 0;
    }
  }
  if (out->vE && (!out->vH || out->E > out->H)) {
    out->H = out->E;
    out->vH = 1;
    ch->src = 1;
  }
  if (out->vF && (!out->vH || out->F > out->H)) {
    out->H = out->F;
    out->vH = 1;
    ch->src = 2;
  }
  if (p->mode == 1 && (!out->vH || out->H <= 0)) {
    out->H = 0; /* local: floor at zero; a zero is a stop */
    out->vH = 1;
    ch->src = 3;
  }
}

static int store_reserve(store_t *st, int64_t more) {
  if (st->ncells + more <= st->cap) return 0;
  int64_t nc = st->cap ? st->cap : 1024;
  while (nc < st->ncells + more) nc *= 2;
  cell_t *n = (cell_t *)realloc(st->cells, (size_t)nc * sizeof(cell_t));
  if (!n) return -1;
  st->cells = n;
  st->cap = nc;
  return 0;
}

static void store_free(store_t *st) {
  free(st->dlo);
  free(st->dhi);
  free(st->base);
  free(st->cells);
  memset(st, 0, sizeof *st);
}

static int store_init(store_t *st, int64_t M, int64_t N) {
  memset(st, 0, sizeof *st);
  st->M = M;
  st->N = N;
  int64_t K = M + N + 1;
  st->dlo = (int64_t *)malloc((size_t)K * sizeof(int64_t));
  st->dhi = (int64_t *)malloc((size_t)K * sizeof(int64_t));
  st->base = (int64_t *)malloc((size_t)K * sizeof(int64_t));
  if (!st->dlo || !st->dhi || !st->base) return -1;
  return 0;
}

/* Open antidiagonal k with diagonals [dl, dh] (parity of k; empty if dl > dh). */
static int store_push(store_t *st, int64_t k, int64_t dl, int64_t dh) {
  int64_t cnt = (dl <= dh) ? (dh - dl) / 2 + 1 : 0;
  if (store_reserve(st, cnt)) return -1;
  st->dlo[k] = dl;
  st->dhi[k] = dh;
  st->base[k] = st->ncells;
  memset(st->cells + st->ncells, 0, (size_t)cnt * sizeof(cell_t));
  st->ncells += cnt;
  st->nk = k + 1;
  return 0;
}

/* Diagonal range of antidiagonal k inside the matrix (and the band). */
static void static_range(ctx_t *c, int64_t k, int64_t *dl, int64_t *dh) {
  int64_t a = -k, b = k;
  if (k - 2 * c->M > a) a = k - 2 * c->M;
  if (2 * c->N - k < b) b = 2 * c->N - k;
  if (c->p->use_band) {
    int64_t bl = up_to_parity(c->lo, k), bh = down_to_parity(c->hi, k);
    if (bl > a) a = bl;
    if (bh < b) b = bh;
  }
  *dl = a;
  *dh = b;
}

/* Unpruned or banded: every cell of the static domain, in row-major (order 0)
 * or antidiagonal (order 1) order.  Reordering leaves every value unchanged
 * (Sec. 6: ordering rewrites preserve values and traceback). */
static int run_static(ctx_t *c, int64_t *cells) {
  int64_t K = c->M + c->N;
  for (int64_t k = 0; k <= K; ++k) {
    int64_t dl, dh;
    static_range(c, k, &dl, &dh);
    if (store_push(&c->st, k, dl, dh)) return -1;
  }
  choice_t ch;
  cell_t tmp;
  *cells = 0;
  if (c->p->order == 0) {
    for (int64_t i = 0; i <= c->M; ++i) {
      int64_t j0 = 0, j1 = c->N;
      if (c->p->use_band) { /* lo <= j - i <= hi */
        if (i + c->lo > j0) j0 = i + c->lo;
        if (i + c->hi < j1) j1 = i + c->hi;
      }
      for (int64_t j = j0; j <= j1; ++j) {
        cell_t *x = get(c, i, j);
        if (!x) continue;
        eval_cell(c, i, j, &tmp, &ch);
        *x = tmp;
        x->alive = tmp.vH;
        if (i >= 1 && j >= 1) ++*cells;
      }
    }
  } else {
    for (int64_t k = 0; k <= K; ++k) {
      for (int64_t d = c->st.dlo[k]; d <= c->st.dhi[k]; d += 2) {
        int64_t i = (k - d) / 2, j = (k + d) / 2;
        cell_t *x = get(c, i, j);
        eval_cell(c, i, j, &tmp, &ch);
        *x = tmp;
        x->alive = tmp.vH;
        if (i >= 1 && j >= 1) ++*cells;
      }
    }
  }
  return 0;
}

/* X-drop, antidiagonal by antidiagonal.  Antidiagonal 0 is the single cell
 * (0,0), never pruned.  For k >= 1 the candidate diagonals are
 * [lo_{k-1} - 1, hi_{k-1} + 1] (same parity as k) inside the matrix and the
 * band; a cell is pruned (H = E = F = invalid) when its H is invalid or
 * H < best_{k-1} - X.  Z-drop (zdrop = 1, Z = xdrop) prunes when
 * best_{k-1} - H > Z + |d - dbest_{k-1}|, dbest_{k-1} the diagonal of
 * antidiagonal k-1's best cell (ties: smallest i, i.e. largest d).  The sweep
 * stops after the first antidiagonal without an unpruned cell. */
static int run_xdrop(ctx_t *c, int64_t *cells, int64_t *last_k) {
  const int64_t X = c->p->xdrop;
  const int no_thresh = (X == INT64_MAX);
  int64_t K = c->M + c->N;
  cell_t tmp;
  choice_t ch;
  if (store_push(&c->st, 0, 0, 0)) return -1;
  cell_t *o = get(c, 0, 0);
  eval_cell(c, 0, 0, &tmp, &ch);
  *o = tmp;
  o->alive = 1;
  int64_t best = 0, lo = 0, hi = 0, dbest = 0;
  const int zdrop = c->p->zdrop != 0;
  *cells = 0;
  *last_k = 0;
  for (int64_t k = 1; k <= K; ++k) {
    int64_t dl, dh;
    static_range(c, k, &dl, &dh);
    if (lo - 1 > dl) dl = lo - 1;
    if (hi + 1 < dh) dh = hi + 1;
    if (store_push(&c->st, k, dl, dh)) return -1;
    *last_k = k;
    int any = 0;
    int64_t nbest = 0, nlo = 0, nhi = 0, ndbest = 0;
    for (int64_t d = dl; d <= dh; d += 2) {
      int64_t i = (k - d) / 2, j = (k + d) / 2;
      cell_t *x = get(c, i, j);
      eval_cell(c, i, j, &tmp, &ch);
      const int64_t dist = zdrop ? (d > dbest ? d - dbest : dbest - d) : 0;
      int alive = tmp.vH && (no_thresh || tmp.H >= best - X - dist);
      if (!alive) memset(&tmp, 0, sizeof tmp);
      *x = tmp;
      x->alive = (uint8_t)alive;
      if (i >= 1 && j >= 1) ++*cells;
      if (alive) {
        if (!any || tmp.H > nbest || (tmp.H == nbest && d > ndbest)) {
          nbest = tmp.H;
          ndbest = d;
        }
        if (!any || d < nlo) nlo = d;
        if (!any || d > nhi) nhi = d;
        any = 1;
      }
    }
    if (!any) break;
    if (!c->p->running || nbest > best) { /* running: keep the first maximum */
      best = nbest;
      dbest = ndbest;
    }
    lo = nlo;
    hi = nhi;
  }
  return 0;
}

/* Walk back from (i, j) in state H; write single-move ops (reversed) into mv.
 * Returns the number of moves; *bi, *bj receive the start cell. */
static int64_t walk(ctx_t *c, int64_t i, int64_t j, uint8_t *mv, int64_t *bi, int64_t *bj) {
  int state = 0; /* 0 H, 1 E, 2 F, 3 M (M/I/D: a gap opened here, so this cell is a diagonal step) */
  const int after_open = (c->p->affine && c->p->mid) ? 3 : 0;
  int64_t n = 0;
  cell_t tmp;
  choice_t ch;
  for (;;) {
    if (state == 0) {
      if (i == 0 && j == 0) break;
      cell_t *x = get(c, i, j);
      if (c->p->mode == 1 && x->H == 0) break; /* local: zero is a stop */
      eval_cell(c, i, j, &tmp, &ch);
      if (ch.src == 0) {
        mv[n++] = (c->q[i - 1] == c->r[j - 1]) ? ORC_OP_EQ : ORC_OP_X;
        --i;
        --j;
      } else if (ch.src == 1) {
        state = 1;
      } else if (ch.src == 2) {
        state = 2;
      } else {
        break;
      }
    } else if (state == 1) {
      eval_cell(c, i, j, &tmp, &ch);
      mv[n++] = ORC_OP_D;
      --j;
      if (!ch.e_ext) state = after_open;
    } else if (state == 2) {
      eval_cell(c, i, j, &tmp, &ch);
      mv[n++] = ORC_OP_I;
      --i;
      if (!ch.f_ext) state = after_open;
    } else {
      if (i == 0 && j == 0) break; /* the origin */
      mv[n++] = (c->q[i - 1] == c->r[j - 1]) ? ORC_OP_EQ : ORC_OP_X;
      --i;
      --j;
      state = 0;
    }
  }
  *bi = i;
  *bj = j;
  return n;
}

int orc_align(const orc_params *p, const uint8_t *q, int64_t M, const uint8_t *r, int64_t N,
              orc_result *res, uint32_t *ops, int64_t cap) {
  if (!p || !res || M < 0 || N < 0 || p->gap_open < 0 || p->gap_extend < 0 || p->alphabet <= 0 ||
      !p->subst || (p->use_xdrop && p->xdrop < 0) || (p->use_band && p->band < 0))
    return -1;
  for (int64_t i = 0; i < M; ++i)
    if (q[i] >= p->alphabet) return -1;
  for (int64_t j = 0; j < N; ++j)
    if (r[j] >= p->alphabet) return -1;
  ctx_t c;
  memset(&c, 0, sizeof c);
  c.p = p;
  c.q = q;
  c.r = r;
  c.M = M;
  c.N = N;
  if (p->use_band) {
    if (p->band_literal) {
      c.lo = -p->band;
      c.hi = p->band;
    } else { /* widened so the band holds both (0,0) and (M,N) */
      c.lo = ((N - M) < 0 ? (N - M) : 0) - p->band;
      c.hi = ((N - M) > 0 ? (N - M) : 0) + p->band;
    }
  }
  memset(res, 0, sizeof *res);
  if (store_init(&c.st, M, N)) {
    store_free(&c.st);
    return -1;
  }
  int64_t cells = 0, last_k = M + N;
  int rc = p->use_xdrop ? run_xdrop(&c, &cells, &last_k) : run_static(&c, &cells);
  if (rc) {
    store_free(&c.st);
    return -1;
  }
  res->cells = cells;
  res->last_k = last_k;

  /* pick the end cell */
  int64_t ei = -1, ej = -1, score = 0;
  int status = ORC_OK;
  if (p->mode == 0) {
    cell_t *x = get(&c, M, N);
    if (x && x->alive) {
      ei = M;
      ej = N;
      score = x->H;
    } else if (p->use_xdrop) {
      status = ORC_DROPPED; /* best unpruned cell anywhere, then smallest i, j */
      int found = 0;
      for (int64_t k = 0; k < c.st.nk; ++k)
        for (int64_t d = c.st.dlo[k]; d <= c.st.dhi[k]; d += 2) {
          int64_t i = (k - d) / 2, j = (k + d) / 2;
          cell_t *y = get(&c, i, j);
          if (!y->alive) continue;
          if (!found || y->H > score || (y->H == score && (i < ei || (i == ei && j < ej)))) {
            score = y->H;
            ei = i;
            ej = j;
            found = 1;
          }
        }
    } else {
      status = ORC_UNREACHABLE;
    }
  } else {
    int found = 0;
    for (int64_t k = 0; k < c.st.nk; ++k)
      for (int64_t d = c.st.dlo[k]; d <= c.st.dhi[k]; d += 2) {
        int64_t i = (k - d) / 2, j = (k + d) / 2;
        cell_t *y = get(&c, i, j);
        if (!y->alive || y->H <= 0) continue;
        if (!found || y->H > score || (y->H == score && (i < ei || (i == ei && j < ej)))) {
          score = y->H;
          ei = i;
          ej = j;
          found = 1;
        }
      }
    if (!found) status = ORC_EMPTY;
  }
  res->status = status;
  if (status == ORC_EMPTY || status == ORC_UNREACHABLE) {
    res->score = 0;
    res->q_begin = res->q_end = res->r_begin = res->r_end = 0;
    if (status == ORC_UNREACHABLE) {
      res->q_end = M;
      res->r_end = N;
    }
    res->n_ops = 0;
    store_free(&c.st);
    return 0;
  }
  res->score = score;
  res->q_end = ei;
  res->r_end = ej;
  res->q_begin = (p->mode == 0) ? 0 : -1;
  res->r_begin = (p->mode == 0) ? 0 : -1;
  res->n_ops = 0;
  if (p->traceback) {
    uint8_t *mv = (uint8_t *)malloc((size_t)(M + N + 1));
    if (!mv) {
      store_free(&c.st);
      return -1;
    }
    int64_t bi, bj;
    int64_t nm = walk(&c, ei, ej, mv, &bi, &bj);
    res->q_begin = bi;
    res->r_begin = bj;
    /* reverse into forward order, run-length encode */
    int64_t nops = 0;
    int64_t t = nm - 1;
    while (t >= 0) {
      uint8_t op = mv[t];
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
  store_free(&c.st);
  return 0;
}

typedef struct {
  const orc_params *p;
  int64_t n;
  const uint8_t *q_seq, *r_seq;
  const uint64_t *q_off, *r_off, *ops_off, *ops_cap;
  const uint32_t *q_len, *r_len;
  orc_result *res;
  uint32_t *ops;
  int64_t next;
  int err;
  pthread_mutex_t mu;
} pool_t;

static void *worker(void *arg) {
  pool_t *w = (pool_t *)arg;
  for (;;) {
    pthread_mutex_lock(&w->mu);
    int64_t t = w->next++;
    pthread_mutex_unlock(&w->mu);
    if (t >= w->n) break;
    uint32_t *o = w->ops ? w->ops + w->ops_off[t] : NULL;
    int64_t cap = w->ops ? (int64_t)w->ops_cap[t] : 0;
    if (orc_align(w->p, w->q_seq + w->q_off[t], w->q_len[t], w->r_seq + w->r_off[t], w->r_len[t],
                  &w->res[t], o, cap)) {
      pthread_mutex_lock(&w->mu);
      w->err = 1;
      pthread_mutex_unlock(&w->mu);
    }
  }
  return NULL;
}

int orc_align_batch(const orc_params *p, int64_t n, const uint8_t *q_seq, const uint64_t *q_off,
                    const uint32_t *q_len, const uint8_t *r_seq, const uint64_t *r_off,
                    const uint32_t *r_len, orc_result *res, uint32_t *ops, const uint64_t *ops_off,
                    const uint64_t *ops_cap, int nthreads) {
  pool_t w;
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
    if (pthread_create(&th[t], NULL, worker, &w) == 0) ++started;
  if (started == 0) worker(&w);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&w.mu);
  return w.err ? -1 : 0;
}

int64_t orc_domain(const orc_params *p, const uint8_t *q, int64_t M, const uint8_t *r, int64_t N,
                   int64_t *cells_ij, uint8_t *alive, int64_t cap) {
  ctx_t c;
  memset(&c, 0, sizeof c);
  c.p = p;
  c.q = q;
  c.r = r;
  c.M = M;
  c.N = N;
  if (p->use_band) {
    if (p->band_literal) {
      c.lo = -p->band;
      c.hi = p->band;
    } else {
      c.lo = ((N - M) < 0 ? (N - M) : 0) - p->band;
      c.hi = ((N - M) > 0 ? (N - M) : 0) + p->band;
    }
  }
  if (store_init(&c.st, M, N)) {
    store_free(&c.st);
    return -1;
  }
  int64_t cells = 0, last_k = 0;
  int rc = p->use_xdrop ? run_xdrop(&c, &cells, &last_k) : run_static(&c, &cells);
  if (rc) {
    store_free(&c.st);
    return -1;
  }
  int64_t n = 0;
  for (int64_t k = 0; k < c.st.nk; ++k)
    for (int64_t d = c.st.dlo[k]; d <= c.st.dhi[k]; d += 2) {
      if (n < cap) {
        cells_ij[2 * n] = (k - d) / 2;
        cells_ij[2 * n + 1] = (k + d) / 2;
        alive[n] = get(&c, (k - d) / 2, (k + d) / 2)->alive;
      }
      ++n;
    }
  store_free(&c.st);
  return n;
}
