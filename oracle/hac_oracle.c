/*
 * CPU oracle for nearest-neighbor-chain HAC (ParChain, arXiv 2106.04727).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is plain, slow, FP64 C written to be
 * checked against the paper by eye.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the GPU library never does, and
 * the two share no code, headers or tables.
 *
 * What it computes (the plain definition of HAC, Section 2):
 *   start from n singleton clusters; repeatedly merge the pair of active
 *   clusters with the smallest linkage distance; record (cid_a, cid_b,
 *   height, size) for each of the n-1 merges.
 *
 * Conventions taken from the paper, with the reading where it is silent:
 *   - cluster id (cid) = smallest input index of a point in the cluster
 *     (footnote to the Section 1 example: "ID of the lexicographically first
 *     point");  a merged cluster keeps min(cid_a, cid_b).
 *   - ties are broken lexicographically (Section 1 example, Fig. 1 caption):
 *     for a fixed cluster X the candidates Y are ordered by the key
 *     (D(X,Y), cid_Y); on unordered pairs this is the order
 *     (D, min cid, max cid).
 *   - linkages (Table 1): complete = max point distance, average (avg-1) =
 *     mean Euclidean point distance, Ward = sqrt(2|A||B|/(|A|+|B|)) *
 *     ||mean_A - mean_B||, avg-2 = mean SQUARED Euclidean point distance
 *     (reported as is: its height is in squared units).
 *   - Lance-Williams update (Section 2, "Lance-Williams Formula", Table 2).
 *     The Ward coefficients are applied to SQUARED Ward distances: with D
 *     defined by the square-root form of Table 1, the update is exact only on
 *     D^2.  The matrix therefore stores D^2 for Ward and D for the others.
 *   - complete linkage: with a1 = a2 = c = 1/2 and b = 0 the Lance-Williams
 *     value is exactly max(D(A,C), D(B,C)); the oracle stores that exact value
 *     (fmax) so that equal point distances stay bit-equal after merges.
 *
 * Entry points (all return 0 on success, negative on bad arguments / OOM):
 *   oracle_nnchain   sequential NN-chain over an FP64 condensed matrix
 *                    (Section 1 description of the sequential algorithm).
 *   oracle_rounds    Algorithm 1 run literally, round by round: all
 *                    terminals find their nearest neighbour, succ/pred are
 *                    set (pred by WriteMin), every reciprocal pair merges,
 *                    chains are repaired; nearest neighbours come from a full
 *                    row scan (the range query of Algorithms 2-3 only prunes
 *                    and cannot change the result).
 *   oracle_greedy    the generic O(n^3) algorithm, recomputing every cluster
 *                    distance from the points each step (no Lance-Williams):
 *                    an independent pin for the matrix updates.
 *   oracle_validate  replays a given dendrogram and checks, step by step in
 *                    height order, that each merged pair is a globally
 *                    minimal pair within a relative tolerance.
 *   oracle_lw        one Lance-Williams update, exposed for unit tests.
 *   oracle_cluster_dist  a linkage distance between two explicit point sets.
 *   oracle_dist_to_all   the linkage distance from one cluster of a labelling
 *                    to every other cluster, from the points (linear memory,
 *                    for checks at sizes the matrix cannot hold).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { LK_COMPLETE = 0, LK_AVERAGE = 1, LK_WARD = 2, LK_AVG2 = 3 };

/* ------------------------------------------------------------------------ */
/* helpers                                                                   */
/* ------------------------------------------------------------------------ */

static double point_dist(const double *x, const double *y, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    double t = x[k] - y[k];
    s += t * t;
  }
  return sqrt(s);
}

static double point_dist2(const double *x, const double *y, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    double t = x[k] - y[k];
    s += t * t;
  }
  return s;
}

/* condensed upper-triangular index, i != j */
static inline size_t cidx(int64_t n, int64_t i, int64_t j) {
  if (i > j) { int64_t t = i; i = j; j = t; }
  return (size_t)i * (size_t)n - (size_t)i * (size_t)(i + 1) / 2 + (size_t)(j - i - 1);
}

/* Lance-Williams update (Table 2).  dac = D(A,C), dbc = D(B,C), dab = D(A,B);
 * for Ward all three are squared distances and so is the result. */
double oracle_lw(int linkage, double dac, double dbc, double dab,
                 double na, double nb, double nc) {
  switch (linkage) {
    case LK_COMPLETE:
      /* a1 = a2 = c = 1/2, b = 0:  (dac + dbc + |dac - dbc|) / 2 = max */
      return fmax(dac, dbc);
    case LK_AVERAGE:
    case LK_AVG2:
      /* a1 = |A|/(|A|+|B|), a2 = |B|/(|A|+|B|), b = c = 0 (avg-2: on squared
       * point distances, which is exactly its own distance) */
      return (na * dac + nb * dbc) / (na + nb);
    case LK_WARD:
      /* a1 = (|A|+|C|)/T, a2 = (|B|+|C|)/T, b = -|C|/T, c = 0, T = |A|+|B|+|C| */
      return ((na + nc) * dac + (nb + nc) * dbc - nc * dab) / (na + nb + nc);
    default:
      return NAN;
  }
}

/* Initial matrix entry between singletons i and j. */
static double singleton_entry(int linkage, const double *X, int d, int64_t i, int64_t j) {
  if (linkage == LK_WARD || linkage == LK_AVG2)
    return point_dist2(X + i * d, X + j * d, d); /* Ward: D^2; avg-2: D */
  return point_dist(X + i * d, X + j * d, d);
}

static double entry_to_height(int linkage, double v) {
  return linkage == LK_WARD ? sqrt(v) : v;
}

/* Linkage distance between two explicit point sets (Table 1), from the
 * points alone.  Used by the brute-force algorithm and by unit tests. */
double oracle_cluster_dist(int linkage, const double *A, int64_t na,
                           const double *B, int64_t nb, int d) {
  if (na <= 0 || nb <= 0) return NAN;
  if (linkage == LK_COMPLETE) {
    double m = 0.0;
    for (int64_t i = 0; i < na; ++i)
      for (int64_t j = 0; j < nb; ++j) {
        double t = point_dist(A + i * d, B + j * d, d);
        if (t > m) m = t;
      }
    return m;
  }
  if (linkage == LK_AVERAGE) {
    double s = 0.0;
    for (int64_t i = 0; i < na; ++i)
      for (int64_t j = 0; j < nb; ++j) s += point_dist(A + i * d, B + j * d, d);
    return s / ((double)na * (double)nb);
  }
  if (linkage == LK_AVG2) {
    double s = 0.0;
    for (int64_t i = 0; i < na; ++i)
      for (int64_t j = 0; j < nb; ++j) s += point_dist2(A + i * d, B + j * d, d);
    return s / ((double)na * (double)nb);
  }
  if (linkage == LK_WARD) {
    double dd = 0.0;
    for (int k = 0; k < d; ++k) {
      double ma = 0.0, mb = 0.0;
      for (int64_t i = 0; i < na; ++i) ma += A[i * d + k];
      for (int64_t j = 0; j < nb; ++j) mb += B[j * d + k];
      ma /= (double)na;
      mb /= (double)nb;
      dd += (ma - mb) * (ma - mb);
    }
    return sqrt(2.0 * (double)na * (double)nb / (double)(na + nb) * dd);
  }
  return NAN;
}

/* Linkage distance (Table 1) from the cluster labelled q to every cluster of
 * a labelling, from the points alone: label[i] in [0, ncl) names the cluster
 * of point i.  out[c] = D(Q, C_c) for every label c != q that has points, NAN
 * for c == q and for labels without points.  Time O(|Q| n d) (Ward and
 * avg-2 as for the others: no centroid shortcut), memory O(ncl d). */
int oracle_dist_to_all(int linkage, const double *X, int64_t n, int d, const int64_t *label,
                       int64_t ncl, int64_t q, double *out) {
  if (!X || !label || !out || n < 1 || d < 1 || ncl < 1 || q < 0 || q >= ncl) return -1;
  if (linkage < LK_COMPLETE || linkage > LK_AVG2) return -1;
  int64_t *cnt = (int64_t *)calloc((size_t)ncl, sizeof(int64_t));
  double *acc = (double *)calloc((size_t)ncl * (linkage == LK_WARD ? (size_t)d : 1), sizeof(double));
  int64_t *qi = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!cnt || !acc || !qi) {
    free(cnt);
    free(acc);
    free(qi);
    return -2;
  }
  int64_t nq = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (label[i] < 0 || label[i] >= ncl) {
      free(cnt);
      free(acc);
      free(qi);
      return -1;
    }
    cnt[label[i]] += 1;
    if (label[i] == q) qi[nq++] = i;
  }
  if (nq == 0) {
    free(cnt);
    free(acc);
    free(qi);
    return -1;
  }
  if (linkage == LK_WARD) {
    /* means of Q and of every cluster, then the Table 1 formula */
    double *mq = (double *)calloc((size_t)d, sizeof(double));
    if (!mq) {
      free(cnt);
      free(acc);
      free(qi);
      return -2;
    }
    for (int64_t i = 0; i < n; ++i)
      for (int k = 0; k < d; ++k) acc[label[i] * d + k] += X[i * d + k];
    for (int64_t t = 0; t < nq; ++t)
      for (int k = 0; k < d; ++k) mq[k] += X[qi[t] * d + k];
    for (int k = 0; k < d; ++k) mq[k] /= (double)nq;
    for (int64_t c = 0; c < ncl; ++c) {
      if (c == q || cnt[c] == 0) {
        out[c] = NAN;
        continue;
      }
      double dd = 0.0;
      for (int k = 0; k < d; ++k) {
        double t = mq[k] - acc[c * d + k] / (double)cnt[c];
        dd += t * t;
      }
      out[c] = sqrt(2.0 * (double)nq * (double)cnt[c] / (double)(nq + cnt[c]) * dd);
    }
    free(mq);
  } else {
    /* every point pair (x in Q, y anywhere), folded into y's cluster */
    for (int64_t i = 0; i < n; ++i) {
      const int64_t c = label[i];
      if (c == q) continue;
      for (int64_t t = 0; t < nq; ++t) {
        const double *x = X + qi[t] * d, *y = X + i * d;
        if (linkage == LK_COMPLETE) {
          double v = point_dist(x, y, d);
          if (v > acc[c]) acc[c] = v;
        } else if (linkage == LK_AVERAGE) {
          acc[c] += point_dist(x, y, d);
        } else {
          acc[c] += point_dist2(x, y, d);
        }
      }
    }
    for (int64_t c = 0; c < ncl; ++c) {
      if (c == q || cnt[c] == 0) out[c] = NAN;
      else if (linkage == LK_COMPLETE) out[c] = acc[c];
      else out[c] = acc[c] / ((double)nq * (double)cnt[c]);
    }
  }
  free(cnt);
  free(acc);
  free(qi);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* shared matrix state                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n;
  int linkage;
  double *M;       /* condensed matrix, n(n-1)/2 entries */
  int64_t *size;   /* cluster size by slot (slot == cid)  */
  char *active;
} mstate;

static void ms_free(mstate *s) {
  free(s->M);
  free(s->size);
  free(s->active);
}

static int ms_init(mstate *s, const double *X, int64_t n, int d, int linkage) {
  s->n = n;
  s->linkage = linkage;
  size_t m = (size_t)n * (size_t)(n - 1) / 2;
  s->M = (double *)malloc((m ? m : 1) * sizeof(double));
  s->size = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  s->active = (char *)malloc((size_t)n);
  if (!s->M || !s->size || !s->active) { ms_free(s); return -2; }
  for (int64_t i = 0; i < n; ++i) {
    s->size[i] = 1;
    s->active[i] = 1;
    for (int64_t j = i + 1; j < n; ++j) s->M[cidx(n, i, j)] = singleton_entry(linkage, X, d, i, j);
  }
  return 0;
}

/* Nearest active neighbour of slot x under the key (D, cid). */
static int64_t ms_nn(const mstate *s, int64_t x, double *dout) {
  int64_t best = -1;
  double bd = INFINITY;
  for (int64_t y = 0; y < s->n; ++y) {
    if (y == x || !s->active[y]) continue;
    double v = s->M[cidx(s->n, x, y)];
    if (best < 0 || v < bd) { /* y increases, so equal v keeps the smaller cid */
      bd = v;
      best = y;
    }
  }
  *dout = bd;
  return best;
}

/* Merge slots a and b (a < b); the new cluster lives in slot a. */
static void ms_merge(mstate *s, int64_t a, int64_t b) {
  double dab = s->M[cidx(s->n, a, b)];
  double na = (double)s->size[a], nb = (double)s->size[b];
  for (int64_t k = 0; k < s->n; ++k) {
    if (k == a || k == b || !s->active[k]) continue;
    double dak = s->M[cidx(s->n, a, k)];
    double dbk = s->M[cidx(s->n, b, k)];
    s->M[cidx(s->n, a, k)] = oracle_lw(s->linkage, dak, dbk, dab, na, nb, (double)s->size[k]);
  }
  s->size[a] += s->size[b];
  s->active[b] = 0;
}

static int check_args(const double *X, int64_t n, int d, int linkage) {
  if (!X || n < 1 || d < 1 || linkage < 0 || linkage > 3) return -1;
  for (int64_t i = 0; i < n * d; ++i)
    if (!isfinite(X[i])) return -1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* sequential NN-chain                                                       */
/* ------------------------------------------------------------------------ */

/* Outputs n-1 merges in the order they were made.  `start` picks the first
 * cluster a chain is grown from; after each merge that empties the chain the
 * next start is the first active slot at or after the previous start. */
int oracle_nnchain(const double *X, int64_t n, int d, int linkage, int64_t start,
                   int64_t *out_a, int64_t *out_b, double *out_h, int64_t *out_size) {
  if (check_args(X, n, d, linkage)) return -1;
  if (n == 1) return 0;
  mstate s;
  if (ms_init(&s, X, n, d, linkage)) return -2;
  int64_t *chain = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!chain) { ms_free(&s); return -2; }
  int64_t len = 0, nm = 0;
  int64_t cursor = ((start % n) + n) % n;
  while (nm < n - 1) {
    if (len == 0) {
      while (!s.active[cursor]) cursor = (cursor + 1) % n;
      chain[len++] = cursor;
    }
    int64_t top = chain[len - 1];
    double dnn;
    int64_t nn = ms_nn(&s, top, &dnn);
    if (len >= 2 && nn == chain[len - 2]) {
      /* reciprocal nearest neighbours: merge them */
      int64_t a = top < nn ? top : nn, b = top < nn ? nn : top;
      out_a[nm] = a;
      out_b[nm] = b;
      out_h[nm] = entry_to_height(linkage, s.M[cidx(n, a, b)]);
      out_size[nm] = s.size[a] + s.size[b];
      ++nm;
      ms_merge(&s, a, b);
      len -= 2;
    } else {
      chain[len++] = nn;
    }
  }
  free(chain);
  ms_free(&s);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1, round by round                                               */
/* ------------------------------------------------------------------------ */

/* Merges are reported with the round (0-based) they happened in.  If
 * term_round/term_cid are non-null, every (round, cid) of a terminal whose
 * nearest neighbour was searched is logged, up to term_cap entries;
 * *n_term receives the number logged.  *n_rounds receives the round count. */
int oracle_rounds(const double *X, int64_t n, int d, int linkage,
                  int64_t *out_a, int64_t *out_b, double *out_h, int64_t *out_size,
                  int64_t *out_round, int64_t *n_rounds,
                  int64_t *term_round, int64_t *term_cid, int64_t term_cap, int64_t *n_term) {
  if (check_args(X, n, d, linkage)) return -1;
  if (n_rounds) *n_rounds = 0;
  if (n_term) *n_term = 0;
  if (n == 1) return 0;
  mstate s;
  if (ms_init(&s, X, n, d, linkage)) return -2;
  int64_t *succ = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *pred = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  double *predd = (double *)malloc((size_t)n * sizeof(double));
  int64_t *E = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  double *Ed = (double *)malloc((size_t)n * sizeof(double));
  char *isterm = (char *)malloc((size_t)n);
  char *merged = (char *)malloc((size_t)n);
  int64_t *pa = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *pb = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!succ || !pred || !predd || !E || !Ed || !isterm || !merged || !pa || !pb) {
    free(succ); free(pred); free(predd); free(E); free(Ed); free(isterm); free(merged);
    free(pa); free(pb); ms_free(&s);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i) {
    succ[i] = -1;
    pred[i] = -1;
    predd[i] = INFINITY;
  }
  int64_t nm = 0, round = 0, nlog = 0, nactive = n;
  while (nactive > 1) {
    /* terminals: active clusters with no successor */
    for (int64_t i = 0; i < n; ++i) isterm[i] = s.active[i] && succ[i] < 0;
    /* find_nearest_neighbors for every terminal (Algorithm 2, full scan) */
    for (int64_t i = 0; i < n; ++i) {
      if (!isterm[i]) continue;
      E[i] = ms_nn(&s, i, &Ed[i]);
      if (term_round && nlog < term_cap) {
        term_round[nlog] = round;
        term_cid[nlog] = i;
      }
      ++nlog;
    }
    /* succ / WriteMin(pred) with key (d, cid) */
    for (int64_t i = 0; i < n; ++i) {
      if (!isterm[i]) continue;
      int64_t j = E[i];
      succ[i] = j;
      if (Ed[i] < predd[j] || (Ed[i] == predd[j] && i < pred[j])) {
        predd[j] = Ed[i];
        pred[j] = i;
      }
    }
    /* reciprocal pairs among terminals' edges (each pair once) */
    int64_t np = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (!isterm[i]) continue;
      int64_t j = succ[i];
      if (succ[j] == i && (i < j || !isterm[j])) {
        pa[np] = i < j ? i : j;
        pb[np] = i < j ? j : i;
        ++np;
      }
    }
    memset(merged, 0, (size_t)n);
    for (int64_t p = 0; p < np; ++p) {
      int64_t a = pa[p], b = pb[p];
      out_a[nm] = a;
      out_b[nm] = b;
      out_h[nm] = entry_to_height(linkage, s.M[cidx(n, a, b)]);
      out_size[nm] = s.size[a] + s.size[b];
      if (out_round) out_round[nm] = round;
      ++nm;
      merged[a] = merged[b] = 1;
    }
    for (int64_t p = 0; p < np; ++p) ms_merge(&s, pa[p], pb[p]);
    /* new clusters start fresh chains; successors that merged are dropped */
    for (int64_t p = 0; p < np; ++p) {
      succ[pa[p]] = -1;
      pred[pa[p]] = -1;
      predd[pa[p]] = INFINITY;
    }
    for (int64_t i = 0; i < n; ++i)
      if (s.active[i] && !merged[i] && succ[i] >= 0 && merged[succ[i]]) succ[i] = -1;
    nactive -= np;
    ++round;
    if (np == 0) break; /* cannot happen for a reducible linkage */
  }
  if (n_rounds) *n_rounds = round;
  if (n_term) *n_term = nlog;
  free(succ); free(pred); free(predd); free(E); free(Ed); free(isterm); free(merged);
  free(pa); free(pb);
  ms_free(&s);
  return nactive == 1 ? 0 : -3;
}

/* ------------------------------------------------------------------------ */
/* generic brute-force algorithm (no Lance-Williams)                          */
/* ------------------------------------------------------------------------ */

int oracle_greedy(const double *X, int64_t n, int d, int linkage,
                  int64_t *out_a, int64_t *out_b, double *out_h, int64_t *out_size) {
  if (check_args(X, n, d, linkage)) return -1;
  if (n == 1) return 0;
  int64_t *label = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *size = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *start = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
  int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  double *G = (double *)malloc((size_t)n * d * sizeof(double));
  if (!label || !size || !start || !fill || !G) {
    free(label); free(size); free(start); free(fill); free(G);
    return -2;
  }
  for (int64_t i = 0; i < n; ++i) { label[i] = i; size[i] = 1; }
  for (int64_t m = 0; m < n - 1; ++m) {
    /* gather every cluster's points contiguously, clusters in cid order */
    start[0] = 0;
    for (int64_t c = 0; c < n; ++c) start[c + 1] = start[c] + (label[c] == c ? size[c] : 0);
    for (int64_t c = 0; c < n; ++c) fill[c] = start[c];
    for (int64_t p = 0; p < n; ++p)
      memcpy(G + (fill[label[p]]++) * d, X + p * d, (size_t)d * sizeof(double));
    double bd = INFINITY;
    int64_t ba = -1, bb = -1;
    for (int64_t a = 0; a < n; ++a) {
      if (label[a] != a) continue; /* a is a cid iff its own point is labelled a */
      for (int64_t b = a + 1; b < n; ++b) {
        if (label[b] != b) continue;
        double v = oracle_cluster_dist(linkage, G + start[a] * d, size[a],
                                       G + start[b] * d, size[b], d);
        /* pairs are visited in increasing (a, b), so strict < keeps the
         * lexicographically smallest (D, a, b) */
        if (v < bd) { bd = v; ba = a; bb = b; }
      }
    }
    out_a[m] = ba;
    out_b[m] = bb;
    out_h[m] = bd;
    out_size[m] = size[ba] + size[bb];
    for (int64_t p = 0; p < n; ++p)
      if (label[p] == bb) label[p] = ba;
    size[ba] += size[bb];
  }
  free(label); free(size); free(start); free(fill); free(G);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* greedy-validity replay                                                    */
/* ------------------------------------------------------------------------ */

/* Replays `m` merges (any order; they are scheduled here).  A merge
 * (a, b, h, size) is ready when slots a and b are active and their sizes add
 * up to `size`; among ready merges the one of least h goes next.  At each
 * step the merged pair's distance D (from the FP64 Lance-Williams matrix) must
 * satisfy |D - h| <= htol * max(D, atol_scale) (the reported height) and
 * D <= (1 + rtol) * Dmin + rtol * atol_scale (the merge itself: how far above
 * the global minimum a tie-zone choice may sit), where Dmin is the smallest
 * distance over all active pairs.  stats[0] = merges whose D exceeded Dmin (tie-zone choices),
 * stats[1] = largest relative excess of D over Dmin, stats[2] = largest
 * relative height error.  Returns 0 if valid, a positive 1-based merge
 * position of the first violation, or negative on bad input. */
int64_t oracle_validate(const double *X, int64_t n, int d, int linkage,
                        const int64_t *ma, const int64_t *mb, const double *mh,
                        const int64_t *msize, int64_t m, double rtol, double htol,
                        double atol_scale, double *stats) {
  if (check_args(X, n, d, linkage)) return -1;
  if (m != n - 1) return -4;
  stats[0] = stats[1] = stats[2] = 0.0;
  if (n == 1) return 0;
  mstate s;
  if (ms_init(&s, X, n, d, linkage)) return -2;
  char *done = (char *)calloc((size_t)m, 1);
  if (!done) { ms_free(&s); return -2; }
  int64_t ret = 0;
  for (int64_t step = 0; step < m; ++step) {
    int64_t pick = -1;
    for (int64_t t = 0; t < m; ++t) {
      if (done[t]) continue;
      int64_t a = ma[t], b = mb[t];
      if (a < 0 || b >= n || a >= b || !s.active[a] || !s.active[b]) continue;
      if (s.size[a] + s.size[b] != msize[t]) continue;
      if (pick < 0 || mh[t] < mh[pick]) pick = t;
    }
    if (pick < 0) { ret = step + 1; break; }
    done[pick] = 1;
    int64_t a = ma[pick], b = mb[pick];
    double D = entry_to_height(linkage, s.M[cidx(n, a, b)]);
    double Dmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
      if (!s.active[i]) continue;
      for (int64_t j = i + 1; j < n; ++j) {
        if (!s.active[j]) continue;
        double v = s.M[cidx(n, i, j)];
        if (v < Dmin) Dmin = v;
      }
    }
    Dmin = entry_to_height(linkage, Dmin);
    double herr = fabs(D - mh[pick]) / fmax(D, atol_scale);
    if (herr > stats[2]) stats[2] = herr;
    if (D > Dmin) {
      stats[0] += 1.0;
      double ex = (D - Dmin) / fmax(Dmin, atol_scale);
      if (ex > stats[1]) stats[1] = ex;
    }
    /* two separate tolerances: rtol on how far the merged pair may sit above
     * the global minimum (the tree), htol on the reported height */
    if (herr > htol || D > (1.0 + rtol) * Dmin + rtol * atol_scale) {
      ret = step + 1;
      break;
    }
    ms_merge(&s, a, b);
  }
  free(done);
  ms_free(&s);
  return ret;
}
