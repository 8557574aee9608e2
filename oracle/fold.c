/* fold.c -- Nussinov RNA folding with X-drop transferred to it (Sec. 9.5),
 * plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
 * benchmark).  Nothing here is shared with the CUDA path.
 *
 * Table 1's RNA folding recurrence over the triangle 0 <= i <= j < n:
 *
 *   F(i,j) = max(F(i+1,j), F(i,j-1), F(i+1,j-1) + in1(i,j),
 *                max over i <= m < j of F(i,m) + F(m+1,j)),   F(i,i) = 0,
 *
 * evaluated wavefront by wavefront along the span k = j - i (the cells of one
 * span depend only on shorter spans).  Readings where the paper is silent (each
 * listed in the design notes):
 *   - in1(i,j) = 1 when the bases pair (Watson-Crick A-U, C-G, or the G-U
 *     wobble; codes A=0 C=1 G=2 U=3) and at least min_loop bases lie between
 *     them (j - i - 1 >= min_loop); otherwise the pair term does not exist.
 *     F of an empty interval (i+1 > j-1) is 0;
 *   - X-drop as in alignment (Sec. 5.2): once the span exceeds the warm-up
 *     (spans <= warmup are never pruned), a cell is pruned when
 *     F < best(k-1) - X, best(k-1) being the largest unpruned F of span k-1;
 *     pruned cells are minus infinity for every later term.  The domain of span
 *     k is the positions i in [lo(k-1) - 1, hi(k-1)] (cell (i, i+k) reads
 *     positions i and i+1 of span k-1), lo / hi the first and last unpruned
 *     positions of span k-1, inside the triangle; the sweep stops at the first
 *     span with no unpruned cell, or at span n-1;
 *   - the result is F(0, n-1) when it was evaluated and left unpruned (OK);
 *     otherwise DROPPED with the best unpruned cell: largest F, then longest
 *     span, then smallest i;
 *   - the fold: walking from the end cell, the first of (i unpaired),
 *     (j unpaired), (i pairs j), (split at the smallest m) that gives F(i,j).
 */
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  const uint8_t *x;
  int64_t n;
  const orc_fold_params *p;
  int64_t *F;      /* F(i, j) at i * n + j */
  uint8_t *alive;  /* evaluated and left unpruned */
} fctx_t;

static int pairs_with(int a, int b) {
  return (a == 0 && b == 3) || (a == 3 && b == 0) || (a == 1 && b == 2) || (a == 2 && b == 1) ||
         (a == 2 && b == 3) || (a == 3 && b == 2);
}

/* F(i, j) if it exists (an empty interval is 0), via *v; returns 0 when it is
 * minus infinity (outside the triangle's evaluated part, or pruned). */
static int val(const fctx_t *c, int64_t i, int64_t j, int64_t *v) {
  if (i > j) {
    *v = 0;
    return 1;
  }
  if (!c->alive[i * c->n + j]) return 0;
  *v = c->F[i * c->n + j];
  return 1;
}

/* The recurrence at (i, j); *ok = 0 when no term exists. */
static int64_t eval(const fctx_t *c, int64_t i, int64_t j, int *ok) {
  int64_t best = 0, a, b;
  int have = 0;
  if (val(c, i + 1, j, &a)) { /* i unpaired */
    best = a;
    have = 1;
  }
  if (val(c, i, j - 1, &a) && (!have || a > best)) { /* j unpaired */
    best = a;
    have = 1;
  }
  if (pairs_with(c->x[i], c->x[j]) && j - i - 1 >= c->p->min_loop && val(c, i + 1, j - 1, &a) &&
      (!have || a + 1 > best)) { /* i pairs j */
    best = a + 1;
    have = 1;
  }
  for (int64_t m = i; m < j; ++m) /* two independent parts */
    if (val(c, i, m, &a) && val(c, m + 1, j, &b) && (!have || a + b > best)) {
      best = a + b;
      have = 1;
    }
  *ok = have;
  return best;
}

/* The fold below (i, j): partner[] gets both ends of every pair. */
static int walk(const fctx_t *c, int64_t i, int64_t j, int32_t *partner) {
  int64_t *stack = (int64_t *)malloc((size_t)(2 * c->n + 2) * sizeof(int64_t));
  if (!stack) return -1;
  int64_t top = 0;
  stack[top++] = i;
  stack[top++] = j;
  while (top) {
    j = stack[--top];
    i = stack[--top];
    if (i >= j) continue;
    int64_t f = c->F[i * c->n + j], a, b;
    if (val(c, i + 1, j, &a) && a == f) {
      stack[top++] = i + 1;
      stack[top++] = j;
    } else if (val(c, i, j - 1, &a) && a == f) {
      stack[top++] = i;
      stack[top++] = j - 1;
    } else if (pairs_with(c->x[i], c->x[j]) && j - i - 1 >= c->p->min_loop &&
               val(c, i + 1, j - 1, &a) && a + 1 == f) {
      partner[i] = (int32_t)j;
      partner[j] = (int32_t)i;
      stack[top++] = i + 1;
      stack[top++] = j - 1;
    } else {
      int64_t m = i;
      for (; m < j; ++m)
        if (val(c, i, m, &a) && val(c, m + 1, j, &b) && a + b == f) break;
      if (m == j) { /* no term gives F(i, j): cannot happen */
        free(stack);
        return -1;
      }
      stack[top++] = i;
      stack[top++] = m;
      stack[top++] = m + 1;
      stack[top++] = j;
    }
  }
  free(stack);
  return 0;
}

int orc_fold(const orc_fold_params *p, const uint8_t *x, int64_t n, orc_fold_result *res,
             int32_t *partner) {
  if (!p || !res || n < 0 || (n > 0 && !x) || p->min_loop < 0 || (p->use_xdrop && p->xdrop < 0))
    return -1;
  for (int64_t t = 0; t < n; ++t)
    if (x[t] > 3) return -1;
  memset(res, 0, sizeof *res);
  if (partner)
    for (int64_t t = 0; t < n; ++t) partner[t] = -1;
  if (n == 0) return 0;
  fctx_t c;
  c.x = x;
  c.n = n;
  c.p = p;
  c.F = (int64_t *)calloc((size_t)(n * n), sizeof(int64_t));
  c.alive = (uint8_t *)calloc((size_t)(n * n), 1);
  if (!c.F || !c.alive) {
    free(c.F);
    free(c.alive);
    return -1;
  }
  /* span 0 */
  for (int64_t i = 0; i < n; ++i) {
    c.F[i * n + i] = 0;
    c.alive[i * n + i] = 1;
  }
  int64_t cells = n, lo = 0, hi = n - 1, best = 0, last_k = 0;
  for (int64_t k = 1; k < n; ++k) {
    int64_t dl = lo - 1 > 0 ? lo - 1 : 0, dh = hi < n - 1 - k ? hi : n - 1 - k;
    if (dl > dh) break;
    int64_t nbest = 0, nlo = -1, nhi = -1;
    for (int64_t i = dl; i <= dh; ++i) {
      const int64_t j = i + k;
      int ok;
      const int64_t f = eval(&c, i, j, &ok);
      ++cells;
      const int alive = ok && (!p->use_xdrop || k <= p->warmup || f >= best - p->xdrop);
      if (!alive) continue;
      c.F[i * n + j] = f;
      c.alive[i * n + j] = 1;
      if (nlo < 0 || f > nbest) nbest = f;
      if (nlo < 0) nlo = i;
      nhi = i;
    }
    last_k = k;
    if (nlo < 0) break;
    best = nbest;
    lo = nlo;
    hi = nhi;
  }
  res->cells = cells;
  res->last_k = last_k;
  int64_t ei = 0, ej = n - 1;
  if (c.alive[ej]) {
    res->status = ORC_OK;
  } else { /* the best unpruned cell: largest F, then longest span, then smallest i */
    res->status = ORC_DROPPED;
    int64_t bf = -1;
    for (int64_t k = n - 1; k >= 0; --k)
      for (int64_t i = 0; i + k < n; ++i)
        if (c.alive[i * n + i + k] && c.F[i * n + i + k] > bf) {
          bf = c.F[i * n + i + k];
          ei = i;
          ej = i + k;
        }
  }
  res->score = c.F[ei * n + ej];
  res->i_end = ei;
  res->j_end = ej;
  int rc = 0;
  if (partner && p->traceback) rc = walk(&c, ei, ej, partner);
  free(c.F);
  free(c.alive);
  return rc;
}

typedef struct {
  const orc_fold_params *p;
  int64_t n;
  const uint8_t *seq;
  const uint64_t *off;
  const uint32_t *len;
  orc_fold_result *res;
  int32_t *partner;
  int64_t next;
  int err;
  pthread_mutex_t mu;
} fpool_t;

static void *fworker(void *arg) {
  fpool_t *w = (fpool_t *)arg;
  for (;;) {
    pthread_mutex_lock(&w->mu);
    const int64_t t = w->next++;
    pthread_mutex_unlock(&w->mu);
    if (t >= w->n) break;
    if (orc_fold(w->p, w->seq + w->off[t], w->len[t], &w->res[t],
                 w->partner ? w->partner + w->off[t] : NULL)) {
      pthread_mutex_lock(&w->mu);
      w->err = 1;
      pthread_mutex_unlock(&w->mu);
    }
  }
  return NULL;
}

int orc_fold_batch(const orc_fold_params *p, int64_t n, const uint8_t *seq, const uint64_t *off,
                   const uint32_t *len, orc_fold_result *res, int32_t *partner, int nthreads) {
  fpool_t w;
  memset(&w, 0, sizeof w);
  w.p = p;
  w.n = n;
  w.seq = seq;
  w.off = off;
  w.len = len;
  w.res = res;
  w.partner = partner;
  pthread_mutex_init(&w.mu, NULL);
  if (nthreads < 1) nthreads = 1;
  pthread_t *th = (pthread_t *)malloc((size_t)nthreads * sizeof(pthread_t));
  if (!th) return -1;
  int started = 0;
  for (int t = 0; t < nthreads; ++t)
    if (pthread_create(&th[t], NULL, fworker, &w) == 0) ++started;
  if (started == 0) fworker(&w);
  for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
  free(th);
  pthread_mutex_destroy(&w.mu);
  return w.err ? -1 : 0;
}
