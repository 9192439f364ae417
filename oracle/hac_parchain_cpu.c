/*
 * hac_parchain_cpu.c -- TEST INFRASTRUCTURE AND TIMED CPU BASELINE ONLY.
 *
 * A plain multithreaded CPU implementation of the parallel nearest-neighbour
 * chain (ParChain, Algorithm 1) in FP64 with linear memory, for inputs too
 * large for the O(n^2)-memory oracle (hac_oracle.c).  Only tests/ and
 * bench.py's CPU-baseline / reference legs use it; the GPU library never
 * loads it and the two share no code.
 *
 * Rounds are those of Algorithm 1, exactly as oracle_rounds runs them:
 *   - terminals = active clusters with no successor;
 *   - every terminal finds its nearest active cluster, the least (D, cid)
 *     (Section 1: ties broken lexicographically), in parallel over the host
 *     threads;
 *   - succ is set and pred takes the least (D, terminal cid) (WriteMin);
 *   - each reciprocal pair among the terminals' edges merges once; the merged
 *     cluster keeps the smaller cid (Section 1 footnote);
 *   - merged clusters start fresh chains, successors that merged are dropped.
 * The nearest neighbour of a terminal comes from a branch-and-bound range
 * query over a kd-tree of the active clusters' centroids, rebuilt every
 * round (Section 4: "Algorithms 2-3"), starting from beta = the distance to
 * its predecessor (Algorithm 2).  A subtree is skipped only when a lower
 * bound on the linkage distance of every cluster under it exceeds the best
 * candidate found so far:
 *   Ward (Section 4.1)    D^2 = 2|A||B|/(|A|+|B|) ||c_A - c_B||^2 is increasing
 *                         in |B|: bound with the subtree's smallest size;
 *   average (Sec. 4.2)    ||c_A - c_B|| <= D_avg (Jensen);
 *   complete (Sec. 4.3)   ||c_A - c_B|| <= D_comp, and per axis
 *                         max(hi_B - lo_A, hi_A - lo_B) <= D_comp (the points
 *                         on those box faces are a pair of A x B);
 *   avg-2 (Table 1)       ||c_A - c_B||^2 + SSE_A/|A| <= D_avg2.
 * Cluster distances are the Table 1 definitions: Ward and avg-2 in O(d) from
 * FP64 centroids and sums of squared deviations (merged as in Section 2),
 * complete and average from the point pairs (point lists, linked in merge
 * order).  Ward's key is D^2 and its height D, as in the oracle.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

enum { LK_COMPLETE = 0, LK_AVERAGE = 1, LK_WARD = 2, LK_AVG2 = 3 };
enum { LEAF = 8, MAXSTK = 256 };

typedef struct {
  int64_t lo, hi;   /* range in the tree's index array */
  int64_t left, right;
  int64_t nmin;     /* smallest cluster size under the node */
} node_t;

typedef struct {
  const double *X;
  int64_t n;
  int d, linkage;
  /* clusters, indexed by cid */
  int64_t *size, *head, *tail, *nxt;
  double *sum, *cent, *lo, *hi, *sse;
  char *active;
  /* chains */
  int64_t *succ, *pred, *E;
  double *predd, *Ed;
  char *isterm, *merged;
  /* the round's kd-tree over active clusters' centroids */
  int64_t *idx, nnodes, *work;
  node_t *nodes;
  double *nlo, *nhi;        /* centroid box per node */
  double *nhmin, *nlmax;    /* complete: min of box hi / max of box lo per node */
  /* the round's terminals (work list for the threads) */
  int64_t *terms, nterms;
  int64_t next_term;        /* shared counter */
  pthread_mutex_t mu;
  uint64_t pair_evals;      /* point pairs evaluated (statistics) */
} cstate;

/* ------------------------------------------------------------------------ */
/* cluster distances (Table 1)                                              */
/* ------------------------------------------------------------------------ */

static double pdist2(const double *x, const double *y, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = x[k] - y[k];
    s += t * t;
  }
  return s;
}

/* The key of the pair (D for complete / average, D^2 for Ward, D for avg-2);
 * +inf once the pair provably loses to `bound` (complete / average: the
 * partial max / partial mean already exceeds it). */
static double pair_key(cstate *s, int64_t a, int64_t b, double bound, uint64_t *pp) {
  const int d = s->d;
  if (a > b) {  /* one order of summation for both directions: symmetric keys */
    const int64_t t = a;
    a = b;
    b = t;
  }
  const double na = (double)s->size[a], nb = (double)s->size[b];
  if (s->linkage == LK_WARD)
    return 2.0 * na * nb / (na + nb) * pdist2(s->cent + a * d, s->cent + b * d, d);
  if (s->linkage == LK_AVG2)
    return pdist2(s->cent + a * d, s->cent + b * d, d) + s->sse[a] / na + s->sse[b] / nb;
  const double nn = na * nb;
  double acc = 0.0;
  uint64_t cnt = 0;
  for (int64_t i = s->head[a]; i >= 0; i = s->nxt[i]) {
    for (int64_t j = s->head[b]; j >= 0; j = s->nxt[j]) {
      const double t = sqrt(pdist2(s->X + i * d, s->X + j * d, d));
      if (s->linkage == LK_COMPLETE) {
        if (t > acc) acc = t;
      } else {
        acc += t;
      }
    }
    cnt += (uint64_t)nb;
    if (s->linkage == LK_COMPLETE ? acc > bound : acc / nn > bound) {
      *pp += cnt;
      return INFINITY;
    }
  }
  *pp += cnt;
  return s->linkage == LK_COMPLETE ? acc : acc / nn;
}

/* squared distance from point c to box [lo, hi] */
static double box_d2(const double *c, const double *lo, const double *hi, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    double t = 0.0;
    if (c[k] < lo[k]) t = lo[k] - c[k];
    else if (c[k] > hi[k]) t = c[k] - hi[k];
    s += t * t;
  }
  return s;
}

/* lower bounds are shrunk by 1e-12 relative: computed in FP64 they could
 * otherwise exceed an equal key by a rounding */
#define LB_SHRINK (1.0 - 1e-12)

/* Lower bound on the key from terminal a to every cluster under node v. */
static double node_lb(const cstate *s, int64_t a, int64_t v) {
  const int d = s->d;
  const double *ca = s->cent + a * d;
  const double g2 = box_d2(ca, s->nlo + v * d, s->nhi + v * d, d);
  const double na = (double)s->size[a];
  switch (s->linkage) {
    case LK_WARD: {
      const double m = (double)s->nodes[v].nmin;
      return 2.0 * na * m / (na + m) * g2 * LB_SHRINK;
    }
    case LK_AVG2:
      return (g2 + s->sse[a] / na) * LB_SHRINK;
    case LK_AVERAGE:
      return sqrt(g2) * LB_SHRINK;
    default: {
      double lb = sqrt(g2);
      for (int k = 0; k < d; ++k) {
        const double t1 = s->nhmin[v * d + k] - s->lo[a * d + k];
        const double t2 = s->hi[a * d + k] - s->nlmax[v * d + k];
        if (t1 > lb) lb = t1;
        if (t2 > lb) lb = t2;
      }
      return lb * LB_SHRINK;
    }
  }
}

/* the same bound for one cluster b */
static double cluster_lb(const cstate *s, int64_t a, int64_t b) {
  const int d = s->d;
  const double g2 = pdist2(s->cent + a * d, s->cent + b * d, d);
  const double na = (double)s->size[a], nb = (double)s->size[b];
  switch (s->linkage) {
    case LK_WARD:
      return 2.0 * na * nb / (na + nb) * g2 * LB_SHRINK;
    case LK_AVG2:
      return (g2 + s->sse[a] / na + s->sse[b] / nb) * LB_SHRINK;
    case LK_AVERAGE:
      return sqrt(g2) * LB_SHRINK;
    default: {
      double lb = sqrt(g2);
      for (int k = 0; k < d; ++k) {
        const double t1 = s->hi[b * d + k] - s->lo[a * d + k];
        const double t2 = s->hi[a * d + k] - s->lo[b * d + k];
        if (t1 > lb) lb = t1;
        if (t2 > lb) lb = t2;
      }
      return lb * LB_SHRINK;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* the round's kd-tree                                                      */
/* ------------------------------------------------------------------------ */

static void nth_by_axis(cstate *s, int64_t *a, int64_t lo, int64_t hi, int64_t nth, int axis) {
  /* quickselect on centroid coordinate `axis` (ties by cid, for determinism) */
  const int d = s->d;
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    const int64_t pv = a[mid];
    const double pvv = s->cent[pv * d + axis];
    /* three-way partition around the key (pvv, pv) */
    int64_t lt = lo, gt = hi - 1, k = lo;
    while (k <= gt) {
      const double v = s->cent[a[k] * d + axis];
      const int less = v < pvv || (v == pvv && a[k] < pv);
      const int more = v > pvv || (v == pvv && a[k] > pv);
      if (less) {
        const int64_t t = a[lt]; a[lt] = a[k]; a[k] = t;
        ++lt; ++k;
      } else if (more) {
        const int64_t t = a[gt]; a[gt] = a[k]; a[k] = t;
        --gt;
      } else {
        ++k;
      }
    }
    if (nth < lt) hi = lt;
    else if (nth > gt) lo = gt + 1;
    else return;
  }
}

static int64_t build_node(cstate *s, int64_t lo, int64_t hi) {
  const int d = s->d;
  const int64_t v = s->nnodes++;
  node_t *nd = &s->nodes[v];
  nd->lo = lo;
  nd->hi = hi;
  nd->left = nd->right = -1;
  double *blo = s->nlo + v * d, *bhi = s->nhi + v * d;
  double *hm = s->nhmin + v * d, *lm = s->nlmax + v * d;
  int64_t nmin = INT64_MAX;
  for (int k = 0; k < d; ++k) {
    blo[k] = INFINITY;
    bhi[k] = -INFINITY;
    hm[k] = INFINITY;
    lm[k] = -INFINITY;
  }
  for (int64_t i = lo; i < hi; ++i) {
    const int64_t c = s->idx[i];
    for (int k = 0; k < d; ++k) {
      const double x = s->cent[c * d + k];
      if (x < blo[k]) blo[k] = x;
      if (x > bhi[k]) bhi[k] = x;
      if (s->linkage == LK_COMPLETE) {
        if (s->hi[c * d + k] < hm[k]) hm[k] = s->hi[c * d + k];
        if (s->lo[c * d + k] > lm[k]) lm[k] = s->lo[c * d + k];
      }
    }
    if (s->size[c] < nmin) nmin = s->size[c];
  }
  nd->nmin = nmin;
  if (hi - lo <= LEAF) return v;
  int axis = 0;
  double w = -1.0;
  for (int k = 0; k < d; ++k)
    if (bhi[k] - blo[k] > w) {
      w = bhi[k] - blo[k];
      axis = k;
    }
  const int64_t mid = lo + (hi - lo) / 2;
  nth_by_axis(s, s->idx, lo, hi, mid, axis);
  const int64_t l = build_node(s, lo, mid);
  const int64_t r = build_node(s, mid, hi);
  s->nodes[v].left = l;
  s->nodes[v].right = r;
  return v;
}

/* ------------------------------------------------------------------------ */
/* nearest neighbour of one terminal                                        */
/* ------------------------------------------------------------------------ */

/* depth-first, nearer child first; the stack holds at most two entries per
 * tree level (depth ~ log2(n / LEAF) < 64) */
static void nn_search(cstate *s, int64_t a, int64_t *stk, uint64_t *pp) {
  double best = INFINITY;
  int64_t bc = INT64_MAX;
  if (s->pred[a] >= 0) {  /* beta: the predecessor is an active candidate */
    best = s->predd[a];
    bc = s->pred[a];
  }
  int64_t top = 0;
  stk[top++] = 0;
  while (top > 0) {
    const int64_t v = stk[--top];
    const node_t *nd = &s->nodes[v];
    if (node_lb(s, a, v) > best) continue;
    if (nd->left < 0) {
      for (int64_t i = nd->lo; i < nd->hi; ++i) {
        const int64_t b = s->idx[i];
        if (b == a) continue;
        if (cluster_lb(s, a, b) > best) continue;
        const double k = pair_key(s, a, b, best, pp);
        if (k < best || (k == best && b < bc)) {
          best = k;
          bc = b;
        }
      }
      continue;
    }
    /* nearer child on top of the stack */
    const double l1 = node_lb(s, a, nd->left), l2 = node_lb(s, a, nd->right);
    if (l1 <= l2) {
      stk[top++] = nd->right;
      stk[top++] = nd->left;
    } else {
      stk[top++] = nd->left;
      stk[top++] = nd->right;
    }
  }
  s->E[a] = bc;
  s->Ed[a] = best;
}

static void *worker(void *arg) {
  cstate *s = (cstate *)arg;
  int64_t stk[MAXSTK];
  uint64_t pp = 0;
  for (;;) {
    pthread_mutex_lock(&s->mu);
    const int64_t t0 = s->next_term;
    s->next_term += 64;
    pthread_mutex_unlock(&s->mu);
    if (t0 >= s->nterms) break;
    const int64_t t1 = t0 + 64 < s->nterms ? t0 + 64 : s->nterms;
    for (int64_t t = t0; t < t1; ++t) nn_search(s, s->terms[t], stk, &pp);
  }
  pthread_mutex_lock(&s->mu);
  s->pair_evals += pp;
  pthread_mutex_unlock(&s->mu);
  return NULL;
}

/* ------------------------------------------------------------------------ */
/* merges                                                                   */
/* ------------------------------------------------------------------------ */

static void merge(cstate *s, int64_t a, int64_t b) {
  const int d = s->d;
  const double na = (double)s->size[a], nb = (double)s->size[b];
  double g2 = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = s->cent[a * d + k] - s->cent[b * d + k];
    g2 += t * t;
  }
  /* Section 2: SSE(A u B) = SSE(A) + SSE(B) + |A||B|/(|A|+|B|) ||c_A - c_B||^2 */
  s->sse[a] = s->sse[a] + s->sse[b] + na * nb / (na + nb) * g2;
  for (int k = 0; k < d; ++k) {
    s->sum[a * d + k] += s->sum[b * d + k];
    s->cent[a * d + k] = s->sum[a * d + k] / (na + nb);
    if (s->lo[b * d + k] < s->lo[a * d + k]) s->lo[a * d + k] = s->lo[b * d + k];
    if (s->hi[b * d + k] > s->hi[a * d + k]) s->hi[a * d + k] = s->hi[b * d + k];
  }
  s->nxt[s->tail[a]] = s->head[b];
  s->tail[a] = s->tail[b];
  s->size[a] += s->size[b];
  s->active[b] = 0;
}

static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* Runs the rounds; out_* receive the merges in the order made (heights in
 * distance units: D for Ward, the linkage value otherwise) and the round of
 * each.  threads <= 0: one.  timeout_s > 0 stops between rounds once
 * exceeded.  stats[0] = rounds, [1] = point pairs evaluated, [2] = seconds.
 * Returns the number of merges made (n - 1 when complete), or negative on
 * bad arguments (-1) or allocation failure (-2). */
int64_t parchain_cpu(const double *X, int64_t n, int d, int linkage, int threads,
                     double timeout_s, int64_t *out_a, int64_t *out_b, double *out_h,
                     int64_t *out_size, int64_t *out_round, double *stats) {
  if (!X || n < 1 || d < 1 || linkage < 0 || linkage > 3) return -1;
  if (threads < 1) threads = 1;
  const double t_start = now_s();
  stats[0] = stats[1] = stats[2] = 0.0;
  if (n == 1) return 0;
  cstate s;
  memset(&s, 0, sizeof(s));
  s.X = X;
  s.n = n;
  s.d = d;
  s.linkage = linkage;
  const size_t nd = (size_t)n * d;
  s.size = malloc(n * sizeof(int64_t));
  s.head = malloc(n * sizeof(int64_t));
  s.tail = malloc(n * sizeof(int64_t));
  s.nxt = malloc(n * sizeof(int64_t));
  s.sum = malloc(nd * sizeof(double));
  s.cent = malloc(nd * sizeof(double));
  s.lo = malloc(nd * sizeof(double));
  s.hi = malloc(nd * sizeof(double));
  s.sse = malloc(n * sizeof(double));
  s.active = malloc(n);
  s.succ = malloc(n * sizeof(int64_t));
  s.pred = malloc(n * sizeof(int64_t));
  s.E = malloc(n * sizeof(int64_t));
  s.predd = malloc(n * sizeof(double));
  s.Ed = malloc(n * sizeof(double));
  s.isterm = malloc(n);
  s.merged = malloc(n);
  s.idx = malloc(n * sizeof(int64_t));
  s.terms = malloc(n * sizeof(int64_t));
  s.nodes = malloc(2 * (size_t)n * sizeof(node_t));
  s.nlo = malloc(2 * nd * sizeof(double));
  s.nhi = malloc(2 * nd * sizeof(double));
  s.nhmin = malloc(2 * nd * sizeof(double));
  s.nlmax = malloc(2 * nd * sizeof(double));
  int64_t *pa = malloc(n * sizeof(int64_t)), *pb = malloc(n * sizeof(int64_t));
  pthread_t *th = malloc((size_t)threads * sizeof(pthread_t));
  int64_t ret = -2;
  if (!s.size || !s.head || !s.tail || !s.nxt || !s.sum || !s.cent || !s.lo || !s.hi ||
      !s.sse || !s.active || !s.succ || !s.pred || !s.E || !s.predd || !s.Ed || !s.isterm ||
      !s.merged || !s.idx || !s.terms || !s.nodes || !s.nlo || !s.nhi || !s.nhmin ||
      !s.nlmax || !pa || !pb || !th)
    goto done;
  pthread_mutex_init(&s.mu, NULL);
  for (int64_t i = 0; i < n; ++i) {
    s.size[i] = 1;
    s.head[i] = s.tail[i] = i;
    s.nxt[i] = -1;
    s.sse[i] = 0.0;
    s.active[i] = 1;
    s.succ[i] = s.pred[i] = -1;
    s.predd[i] = INFINITY;
    for (int k = 0; k < d; ++k) {
      const double x = X[i * d + k];
      s.sum[i * d + k] = s.cent[i * d + k] = s.lo[i * d + k] = s.hi[i * d + k] = x;
    }
  }
  int64_t nm = 0, round = 0, nactive = n;
  while (nactive > 1) {
    if (timeout_s > 0 && now_s() - t_start > timeout_s) break;
    /* terminals and the tree over the active clusters */
    int64_t K = 0;
    s.nterms = 0;
    for (int64_t i = 0; i < n; ++i) {
      s.isterm[i] = s.active[i] && s.succ[i] < 0;
      if (s.active[i]) s.idx[K++] = i;
      if (s.isterm[i]) s.terms[s.nterms++] = i;
    }
    s.nnodes = 0;
    build_node(&s, 0, K);
    /* find_nearest_neighbors, in parallel */
    s.next_term = 0;
    int started = 0;
    for (int t = 0; t < threads; ++t)
      if (pthread_create(&th[t], NULL, worker, &s) == 0) ++started;
    if (started == 0) worker(&s);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    /* succ / WriteMin(pred) with key (d, cid), in cid order */
    for (int64_t t = 0; t < s.nterms; ++t) {
      const int64_t i = s.terms[t], j = s.E[i];
      s.succ[i] = j;
      if (s.Ed[i] < s.predd[j] || (s.Ed[i] == s.predd[j] && i < s.pred[j])) {
        s.predd[j] = s.Ed[i];
        s.pred[j] = i;
      }
    }
    /* reciprocal pairs among the terminals' edges, each once */
    int64_t np = 0;
    for (int64_t t = 0; t < s.nterms; ++t) {
      const int64_t i = s.terms[t], j = s.succ[i];
      if (s.succ[j] == i && (i < j || !s.isterm[j])) {
        pa[np] = i < j ? i : j;
        pb[np] = i < j ? j : i;
        ++np;
      }
    }
    if (np == 0) break; /* cannot happen for a reducible linkage */
    memset(s.merged, 0, (size_t)n);
    for (int64_t p = 0; p < np; ++p) {
      const int64_t a = pa[p], b = pb[p];
      const double key = s.Ed[s.isterm[a] && s.succ[a] == b ? a : b];
      out_a[nm] = a;
      out_b[nm] = b;
      out_h[nm] = linkage == LK_WARD ? sqrt(key) : key;
      out_size[nm] = s.size[a] + s.size[b];
      if (out_round) out_round[nm] = round;
      ++nm;
      s.merged[a] = s.merged[b] = 1;
    }
    for (int64_t p = 0; p < np; ++p) merge(&s, pa[p], pb[p]);
    /* new clusters start fresh chains; successors that merged are dropped */
    for (int64_t p = 0; p < np; ++p) {
      s.succ[pa[p]] = -1;
      s.pred[pa[p]] = -1;
      s.predd[pa[p]] = INFINITY;
    }
    for (int64_t i = 0; i < n; ++i) {
      if (!s.active[i] || s.merged[i]) continue;
      if (s.succ[i] >= 0 && s.merged[s.succ[i]]) s.succ[i] = -1;
      if (s.pred[i] >= 0 && s.merged[s.pred[i]]) {  /* beta must name an active cluster */
        s.pred[i] = -1;
        s.predd[i] = INFINITY;
      }
    }
    nactive -= np;
    ++round;
  }
  stats[0] = (double)round;
  stats[1] = (double)s.pair_evals;
  ret = nm;
  pthread_mutex_destroy(&s.mu);
done:
  stats[2] = now_s() - t_start;
  free(s.size); free(s.head); free(s.tail); free(s.nxt); free(s.sum); free(s.cent);
  free(s.lo); free(s.hi); free(s.sse); free(s.active); free(s.succ); free(s.pred);
  free(s.E); free(s.predd); free(s.Ed); free(s.isterm); free(s.merged); free(s.idx);
  free(s.terms); free(s.nodes); free(s.nlo); free(s.nhi); free(s.nhmin); free(s.nlmax);
  free(pa); free(pb); free(th);
  return ret;
}
