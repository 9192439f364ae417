// Nearest-neighbour search of every terminal cluster (ParChain Algorithms 2-4).
//
// One warp per terminal C_i.  The active clusters sit in spatial order in
// `order`; a 32-ary implicit tree over that order stores, per node, the box of
// its clusters' centroids, the smallest cluster size under it, and (for
// complete linkage) the per-axis min of box-hi / max of box-lo.  The search is
// the paper's range query with the ball radius of Section 4 for each linkage,
// run as branch-and-bound: the radius starts from beta = pred.d (Algorithm 2)
// and shrinks to the best distance found so far, so every cluster that could
// still beat the current best is evaluated and nothing else is.  The first
// candidate is the nearest-looking cluster of C_i's own leaf (a spatially
// adjacent cluster: the "distance to a nearby cluster" of Algorithm 2).
//
//   Ward    (Sec. 4.1): ||c_i - c_B|| <= beta * sqrt((|C_i| + m) / (2 m |C_i|)),
//                        m = smallest cluster size under the node (the paper
//                        uses the global n_min; a per-node minimum is tighter)
//   average (Sec. 4.2): ||c_i - c_B|| <= beta  (centroid distance <= D_avg)
//   complete(Sec. 4.3): ||c_i - c_B|| <= beta, and per axis
//                        max(hi_B - lo_A, hi_A - lo_B) <= beta (the points
//                        attaining those box faces are a pair of A x B)
//
// Every lower bound is tested in FP32 with a relative slack EPS and an
// absolute slack (coordinate scale * 2^-18), so a bound can only admit extra
// candidates, never drop the true nearest neighbour.
//
// Precision modes (the nearest neighbour is always the candidate of least
// (FP64 key, cid): ties broken lexicographically, Section 1):
//   F64     every candidate that survives the bound tests is evaluated in FP64
//           (Table 1 definitions).
//   F32     pass 1 evaluates candidates in FP32 with the error model
//           |D32 - D| <= delta + rho * D  (D in distance units;
//           delta = 2.01 u M sqrt(d) [* sqrt(2|A||B|/(|A|+|B|)) for Ward],
//           u = 2^-24, M = largest |coordinate| after recentring,
//           rho = (d + 16) u [+ 32 u for average: FP32 partial sums of at most
//           32 terms]).  lo = (D32 - delta)(1 - rho) and
//           up = (D32 + delta)(1 + rho) bracket the true D.  With U = min up,
//           the FP64 winner is among the candidates with lo <= U.  If only one
//           candidate has lo <= U it is the winner; otherwise a second
//           traversal re-scores every candidate with lo <= U in FP64.
//
// Keys: Ward compares D^2 = 2|A||B|/(|A|+|B|) ||c_A - c_B||^2, complete
// sqrt(max ||x - y||^2), average the mean of ||x - y||.  Exact keys are
// compared as the bit patterns of non-negative doubles (integer compares), so
// the bookkeeping issues no FP64 instructions.
#pragma once

#include "hac_dev.cuh"

#include <cfloat>
#include <climits>

namespace hacg {

namespace {

// block shape of the search (the tuner's compiled variants override these)
#ifndef HAC_QWARPS
#define HAC_QWARPS 4
#endif
#ifndef HAC_QMINB
#define HAC_QMINB 8
#endif
#ifndef HAC_QMINB_COMPLETE
#define HAC_QMINB_COMPLETE 6
#endif
constexpr int QWARPS = HAC_QWARPS;  // warps per block
// resident blocks per SM the register budget must allow.  The searches are
// latency-bound, and more resident warps beat the register spills they cost:
// the shape tuner's whole-run times at 10^6 points (5-D mixture), at
// 4 / 5 / 6 / 8 blocks (128 / 96 / 80 / 64 registers): average 431 / 431 /
// 423 / 415 ms, Ward 68 / - / 61 / 59 ms; complete 365 / 374 / 366 / - ms
// (its box bounds hold more registers), so complete keeps 6.
constexpr int qminb(int lk) { return lk == LK_COMPLETE ? HAC_QMINB_COMPLETE : HAC_QMINB; }
constexpr int STK = 288;           // per-warp stack: >= 32 + 31 * (levels - 1), 9 levels for n < 2^31
constexpr float EPS = 1e-5f;       // relative slack of the FP32 bound tests
constexpr long long SMALLP = 32;   // pairs of at most this many point pairs run per lane
constexpr float U32 = 5.9604645e-8f;  // 2^-24
constexpr unsigned long long KINF = 0x7ff0000000000000ull;  // bits of +inf

enum { M_F64 = 0, M_F32 = 1, M_RECHECK = 2 };
// per-warp search counters (shared memory), added to the instance's at the end
enum { C_CPAIRS, C_PPAIRS, C_NODES, C_LTESTS, C_PROWS, C_RECHECKS, C_HITS, C_N };

// The warp-wide pair evaluations, which a search takes for its larger
// candidates only, are kept out of line (HAC_Q_OUTLINE=1), so that their
// registers do not count against the scan of tree nodes and leaves.
#ifndef HAC_Q_OUTLINE
#define HAC_Q_OUTLINE 0
#endif
#if HAC_Q_OUTLINE
#define HAC_Q_COLD __noinline__
#else
#define HAC_Q_COLD
#endif

__device__ __forceinline__ unsigned long long kbits(double k) {
  return (unsigned long long)__double_as_longlong(k);
}

__device__ __forceinline__ bool kless(unsigned long long k1, int c1, unsigned long long k2,
                                      int c2) {
  return k1 < k2 || (k1 == k2 && c1 < c2);
}

__device__ __forceinline__ void warp_argmin_u(unsigned long long &k, int &c) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
    int c2 = __shfl_xor_sync(0xffffffffu, c, o);
    if (kless(k2, c2, k, c)) {
      k = k2;
      c = c2;
    }
  }
}

// (value, lane) argmin; ties go to the lower lane
__device__ __forceinline__ void warp_argmin_f(float &v, int &l) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    float v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int l2 = __shfl_xor_sync(0xffffffffu, l, o);
    if (v2 < v || (v2 == v && l2 < l)) {
      v = v2;
      l = l2;
    }
  }
}

__device__ __forceinline__ float warp_minf(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// exact key -> distance (FP32, rounded up)
template <int LK>
__device__ __forceinline__ float key_dist_ru(unsigned long long kb) {
  if (kb >= KINF) return INFINITY;
  const float f = __double2float_ru(__longlong_as_double((long long)kb));
  return LK == LK_WARD || LK == LK_AVG2 ? __fsqrt_ru(f) : f;  // squared-unit keys
}

// Squared distance from point c to box [lo, hi] (0 inside).
template <int DP>
__device__ __forceinline__ float box_d2(const float *c, const float *lo, const float *hi) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    float t = fmaxf(fmaxf(lo[k] - c[k], c[k] - hi[k]), 0.f);
    s = fmaf(t, t, s);
  }
  return s;
}

// 2|A||B|/(|A|+|B|) in FP32 (relative error <= 3u)
__device__ __forceinline__ float ward_w(float na, float nb) {
  return 2.f * na * nb * __frcp_rn(na + nb);
}

// Lower bound on D(C_i, B) for every cluster B under a node, in D units.
template <int LK, int DP>
__device__ __forceinline__ float node_lb(const QueryArgs &a, int node, const float *ci32,
                                         const float *alo, const float *ahi, float na,
                                         float va) {
  float lo[DP], hi[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    lo[k] = a.nclo[(size_t)node * DP + k];
    hi[k] = a.nchi[(size_t)node * DP + k];
  }
  const float dc2 = box_d2<DP>(ci32, lo, hi);
  if (LK == LK_WARD) return sqrtf(ward_w(na, (float)a.nnmin[node]) * dc2);
  // avg-2: D = ||c_A - c_B||^2 + var A + var B >= dc2 + var A
  if (LK == LK_AVG2) return sqrtf(dc2 + va);
  float lb = sqrtf(dc2);
  if (LK == LK_COMPLETE) {
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      lb = fmaxf(lb, a.nhmin[(size_t)node * DP + k] - alo[k]);
      lb = fmaxf(lb, ahi[k] - a.nlmax[(size_t)node * DP + k]);
    }
  }
  return lb;
}

// Ward key 2|A||B|/(|A|+|B|) ||c_A - c_B||^2 in FP64 (Table 1).
template <int DP>
__device__ __forceinline__ double ward_key(const double *cA, const double *cB, int na, int nb,
                                           int d) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    if (k < d) {  // the padding coordinates add +0
      double t = cA[k] - cB[k];
      s += t * t;
    }
  }
  return (2.0 * (double)na * (double)nb) / (double)(na + nb) * s;
}

template <int DP, typename T>
__device__ __forceinline__ T pt_d2(const T *x, const T *y) {
  T s = 0;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    T t = x[k] - y[k];
    s = s + t * t;
  }
  return s;
}

// ---- FP64 pair evaluation (average / complete) -----------------------------

// One lane evaluates a whole small pair in FP64.
template <int LK, int DP>
__device__ double eval64_lane(const double *P, int sa, int na, int sb, int nb) {
  double acc = 0.0;
  for (int i = 0; i < na; ++i) {
    double x[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) x[k] = P[(size_t)(sa + i) * DP + k];
    for (int j = 0; j < nb; ++j) {
      double d2 = pt_d2<DP>(x, P + (size_t)(sb + j) * DP);
      if (LK == LK_COMPLETE)
        acc = fmax(acc, d2);
      else
        acc += sqrt(d2);
    }
  }
  if (LK == LK_COMPLETE) return sqrt(acc);
  return acc / ((double)na * (double)nb);
}

// The whole warp evaluates one pair in FP64: lanes stride over the larger
// cluster's points, each lane loops over the smaller one (broadcast loads).
// Returns +inf once a partial result proves D > bound (D units).
template <int LK, int DP>
HAC_Q_COLD __device__ double eval64_warp(const double *P, int sa, int na, int sb, int nb, double bound,
                              int lane, unsigned long long &pp) {
  int sL = sa, nL = na, sS = sb, nS = nb;
  if (nb > na) {
    sL = sb;
    nL = nb;
    sS = sa;
    nS = na;
  }
  const double nn = (double)na * (double)nb;
  double thr = INFINITY;
  if (bound < INFINITY)
    thr = LK == LK_COMPLETE ? bound * bound * (1.0 + 1e-9) : bound * nn * (1.0 + 1e-9);
  double acc = 0.0;
  for (int base = 0; base < nL; base += 32) {
    const int l = base + lane;
    if (l < nL) {
      double x[DP];
#pragma unroll
      for (int k = 0; k < DP; ++k) x[k] = P[(size_t)(sL + l) * DP + k];
      for (int j = 0; j < nS; ++j) {
        double d2 = pt_d2<DP>(x, P + (size_t)(sS + j) * DP);
        if (LK == LK_COMPLETE)
          acc = fmax(acc, d2);
        else
          acc += sqrt(d2);
      }
    }
    if (thr < INFINITY) {
      const double tot = LK == LK_COMPLETE ? warp_max(acc) : warp_sum(acc);
      if (tot > thr) {
        pp += (unsigned long long)min(nL, base + 32) * nS;
        return INFINITY;
      }
    }
  }
  pp += (unsigned long long)nL * nS;
  const double tot = LK == LK_COMPLETE ? warp_max(acc) : warp_sum(acc);
  if (LK == LK_COMPLETE) return sqrt(tot);
  return tot / nn;
}

// ---- FP32 pair evaluation (average / complete) -----------------------------

// One lane, FP32, at most SMALLP point pairs (one FP32 partial sum).
template <int LK, int DP>
__device__ float eval32_lane(const float *P, int sa, int na, int sb, int nb) {
  float acc = 0.f;
  for (int i = 0; i < na; ++i) {
    float x[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) x[k] = P[(size_t)(sa + i) * DP + k];
    for (int j = 0; j < nb; ++j) {
      const float d2 = pt_d2<DP>(x, P + (size_t)(sb + j) * DP);
      if (LK == LK_COMPLETE)
        acc = fmaxf(acc, d2);
      else
        acc += sqrtf(d2);
    }
  }
  if (LK == LK_COMPLETE) return sqrtf(acc);
  return acc / ((float)na * (float)nb);
}

// Warp-cooperative FP32 evaluation: lanes stride over the larger cluster's
// points, each lane loops over the smaller one (broadcast loads).  A squared
// distance takes H = ceil(d/2) coordinate pairs as f32x2 words (even and odd
// coordinates summed apart, then added; padding coordinates are 0 on both
// sides).  Average flushes FP32 partial sums of at most 16 terms into an FP64
// accumulator.  Returns +inf once the partial result's lower bound exceeds
// `bound` (D units).
template <int LK, int H, int DP>
__device__ float eval32_warp_h(const float *P, int sa, int na, int sb, int nb, float bound,
                               float delta, float rho, int lane, unsigned long long &pp) {
  int sL = sa, nL = na, sS = sb, nS = nb;
  if (nb > na) {
    sL = sb;
    nL = nb;
    sS = sa;
    nS = na;
  }
  const double nn = (double)na * (double)nb;
  float macc = 0.f;
  double sacc = 0.0;
  for (int base = 0; base < nL; base += 32) {
    const int l = base + lane;
    if (l < nL) {
      const unsigned long long *xr = (const unsigned long long *)(P + (size_t)(sL + l) * DP);
      unsigned long long x[H];
#pragma unroll
      for (int h = 0; h < H; ++h) x[h] = xr[h];
      float part = 0.f;
      int cnt = 0;
      for (int j = 0; j < nS; ++j) {
        const unsigned long long *yr = (const unsigned long long *)(P + (size_t)(sS + j) * DP);
        unsigned long long t = f2_sub(x[0], yr[0]);
        unsigned long long d2 = f2_mul(t, t);
#pragma unroll
        for (int h = 1; h < H; ++h) {
          t = f2_sub(x[h], yr[h]);
          d2 = f2_fma(t, t, d2);
        }
        const float s2 = f2_hsum(d2);
        if (LK == LK_COMPLETE) {
          macc = fmaxf(macc, s2);
        } else {
          part += sqrt_approx(s2);
          if (++cnt == 16) {
            sacc += (double)part;
            part = 0.f;
            cnt = 0;
          }
        }
      }
      if (LK != LK_COMPLETE) sacc += (double)part;
    }
    if (bound < INFINITY) {
      float est;
      if (LK == LK_COMPLETE)
        est = sqrtf(warp_maxf(macc));
      else
        est = (float)(warp_sum(sacc) / nn);
      if ((est - delta) * (1.f - rho) > bound) {
        pp += (unsigned long long)min(nL, base + 32) * nS;
        return INFINITY;
      }
    }
  }
  pp += (unsigned long long)nL * nS;
  if (LK == LK_COMPLETE) return sqrtf(warp_maxf(macc));
  return (float)(warp_sum(sacc) / nn);
}

// eval32_warp_h for the instance's true dimension d (rows have stride DP)
template <int LK, int DP>
HAC_Q_COLD __device__ float eval32_warp(const float *P, int d, int sa, int na, int sb, int nb, float bound,
                             float delta, float rho, int lane, unsigned long long &pp) {
  const int H = (d + 1) >> 1;
  if (DP == 2) return eval32_warp_h<LK, 1, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
  if (DP == 4) return eval32_warp_h<LK, 2, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
  if (DP == 8) {
    if (H <= 3) return eval32_warp_h<LK, 3, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
    return eval32_warp_h<LK, 4, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
  }
  if (H <= 5) return eval32_warp_h<LK, 5, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
  if (H == 6) return eval32_warp_h<LK, 6, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
  if (H == 7) return eval32_warp_h<LK, 7, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
  return eval32_warp_h<LK, 8, DP>(P, sa, na, sb, nb, bound, delta, rho, lane, pp);
}

// ---------------------------------------------------------------------------

template <int LK, int DP, int MODE>
struct Searcher {
  const QueryArgs &a;
  int lane, ci, na, sa;
  int myinst;     // instance slot of C_i (its parameters)
  int myseq;      // its admission number: candidates come from the same instance only
  float fna;
  float dpts;     // error term of FP32 point distances for this instance
  float ci32[DP], alo[DP], ahi[DP];
  float slack;
  float beta_d;   // pred bound, D units
  float Uv;       // least upper bound on D(C_i, candidate) from cluster summaries
  float vA;       // variance of C_i, rounded up (average linkage)
  float bd;       // current upper bound on the NN distance, D units
  float T;        // pruning threshold: bd * (1 + EPS) + slack
  // exact (FP64) best, as key bits and cid
  unsigned long long bk;
  int bc;
  // FP32 pass-1 state
  float U;        // min over candidates of the FP32 upper bound
  float L1, L2;   // two smallest FP32 lower bounds
  int c1;         // cid holding L1
  float d1, e1;   // FP32 value and error term of that candidate
  double pv;      // partial entry found by the last cache_get: value,
  float pe;       //   error term,
  int ppart;      //   covered points of its owner (> 0 prefix, < 0 suffix),
  bool pown_ci;   //   and whether C_i owns it
  bool deferred;  // a big pair was handed to the GPU-wide evaluation
  float delta0, rho;
  unsigned long long ppairs;  // point pairs this search evaluated (its budget)
  unsigned long long *sc;     // this warp's counters in shared memory (C_*)

  __device__ Searcher(const QueryArgs &args, int lane_, int ci_, float Ufix,
                       unsigned long long *sc_)
      : a(args), lane(lane_), ci(ci_), sc(sc_) {
    na = a.csize[ci];
    fna = (float)na;
    myinst = a.inst[ci];
    myseq = a.qinst[a.pos[ci]];
    dpts = a.idpts[myinst];
    sa = a.seg[ci];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      ci32[k] = a.cent32[(size_t)ci * DP + k];
      alo[k] = a.blo[(size_t)ci * DP + k];
      ahi[k] = a.bhi[(size_t)ci * DP + k];
    }
    const unsigned long long pv = a.pred[ci];
    if (pv == PRED_EMPTY) {
      beta_d = INFINITY;
    } else {
      const float bkey = __uint_as_float((unsigned)(pv >> 32));
      beta_d = LK == LK_WARD || LK == LK_AVG2 ? __fsqrt_ru(bkey) : bkey;
    }
    slack = a.islack[myinst] * (LK == LK_WARD ? sqrtf(2.f * fna) : 2.f);
    delta0 = 2.01f * U32 * a.iscale[myinst] * sqrtf((float)a.d);
    rho = ((float)a.d + 16.f) * U32 + (LK == LK_AVERAGE ? 32.f * U32 : 0.f);
    bk = KINF;
    bc = INT_MAX;
    U = Ufix;
    Uv = INFINITY;
    vA = LK == LK_AVERAGE || LK == LK_AVG2 ? a.qvar[a.pos[ci]] : 0.f;
    L1 = L2 = INFINITY;
    c1 = INT_MAX;
    d1 = e1 = INFINITY;
    deferred = false;
    ppairs = 0;
    refresh();
  }

  // add a warp-uniform amount to counter k (lane 0 keeps the warp's counts)
  __device__ void count(int k, unsigned long long v) const {
    if (lane == 0) sc[k] += v;
  }

  // Section 5 cache: look for the entry of `nbr` in the table of `owner`
  // (warp-cooperative; valid only while the neighbour's generation matches)
  // (`part` receives the entry's partial tag, 0 for a full value)
  __device__ bool cache_find(int owner, int nbr, double &v, float &e, int &part) const {
    const int S = a.cache_slots;
    const unsigned long long want = ckey_of(nbr, a.gen[nbr]);
    for (int base = 0; base < S; base += 32) {
      const int t = base + lane;
      const bool m = t < S && a.ckey[(size_t)owner * S + t] == want;
      const unsigned b = __ballot_sync(0xffffffffu, m);
      if (b) {
        const size_t slot = (size_t)owner * S + base + __ffs(b) - 1;
        v = a.cval[slot];
        e = a.cerr[slot];
        part = a.cpart[slot];
        return true;
      }
    }
    return false;
  }

  // this round's big-pair results (lane 0 probes, the warp shares the answer)
  __device__ bool side_find(int cw, double &v, float &e) const {
    if (!a.defer || a.side_cap <= 0) return false;
    int at = -1;
    if (lane == 0) {
      const int lo = min(ci, cw), hi = max(ci, cw);
      const unsigned long long want = ((unsigned long long)(unsigned)lo << 32) | (unsigned)hi;
      unsigned h = side_hash(lo, hi, a.side_cap);
      for (int q = 0; q < SIDE_PROBES; ++q, h = (h + 1) & (unsigned)(a.side_cap - 1)) {
        const unsigned long long cur = a.side_key[h];
        if (cur == want) {
          at = (int)h;
          break;
        }
        if (cur == CKEY_EMPTY) break;
      }
    }
    at = __shfl_sync(0xffffffffu, at, 0);
    if (at < 0) return false;
    v = a.side_val[at];
    e = a.side_err[at];
    return true;
  }

  // 0: nothing known; 1: D(C_i, C_w) in v, e; 2: only a partial entry
  // (kept in pv, pe, ppart, pown_ci for try_defer_part)
  __device__ int cache_get(int cw, int nw, double &v, float &e) {
    if (a.cache_slots <= 0 || (long long)na * nw < CACHE_MIN_PAIRS) return 0;
    double v1, v2;
    float f1, f2;
    int p1 = 0, p2 = 0;
    const bool h1 = cache_find(ci, cw, v1, f1, p1);
    if (h1 && p1 == 0) {
      v = v1;
      e = f1;
      count(C_HITS, 1);
      return 1;
    }
    const bool h2 = cache_find(cw, ci, v2, f2, p2);
    if (h2 && p2 == 0) {
      v = v2;
      e = f2;
      count(C_HITS, 1);
      return 1;
    }
    if ((long long)na * nw >= BIG_MIN_PAIRS && side_find(cw, v, e)) {
      count(C_HITS, 1);
      return 1;
    }
    if (h1 || h2) {
      pv = h1 ? v1 : v2;
      pe = h1 ? f1 : f2;
      ppart = h1 ? p1 : p2;
      pown_ci = h1;
      return 2;
    }
    return 0;
  }

  // queue a computed distance for insertion into both tables (after the search)
  __device__ void cache_put(int cw, int nw, double v, float e) const {
    if (a.cache_slots <= 0 || (long long)na * nw < CACHE_MIN_PAIRS || lane != 0) return;
    const int q = atomicAdd(&a.ctr->nins, 1);
    if (q < a.ins_cap) {
      a.ins_i[q] = ci;
      a.ins_j[q] = cw;
      a.ins_v[q] = v;
      a.ins_e[q] = e;
    }
  }

  __device__ void refresh() {
    if (MODE == M_F32)
      bd = fminf(beta_d, U);
    else if (MODE == M_RECHECK)
      bd = fminf(U, key_dist_ru<LK>(bk));
    else
      bd = fminf(fminf(beta_d, key_dist_ru<LK>(bk)), Uv);
    T = bd * (1.f + EPS) + slack;
  }

  // Upper bounds on D(C_i, B) that need no point pairs (one per lane, INF if
  // none): the nearest neighbour is no farther than the least of them, so
  // candidates whose lower bound exceeds it are pruned before any evaluation.
  // In the FP32 passes the bound also joins U (it bounds the true distance).
  __device__ void offer_ub(float ub) {
    const float m = warp_minf(ub);
    if (m < Uv) {
      Uv = m;
      if (MODE != M_F64) U = fminf(U, m);
      refresh();
    }
  }

  __device__ bool pass(float lb) const { return lb <= T || a.noprune; }

  __device__ float lower(float d32, float dlt) const { return fmaxf(d32 - dlt, 0.f) * (1.f - rho); }

  // exact candidates: every lane offers its own (k, c) (c = INT_MAX if none)
  __device__ void offer_exact(unsigned long long k, int c) {
    warp_argmin_u(k, c);
    if (kless(k, c, bk, bc)) {
      bk = k;
      bc = c;
      refresh();
    }
  }

  // FP32 candidates: every lane offers its own estimate (has = false if none).
  // U (which sets the pruning threshold) is reduced over the warp at once; the
  // two least lower bounds and the candidate of the least are kept per lane
  // and combined once, by finish_f32, after the traversal.
  __device__ void offer_f32(bool has, float d32, float dlt, int c) {
    const float lo = has ? lower(d32, dlt) : INFINITY;
    const float up = has ? (d32 + dlt) * (1.f + rho) : INFINITY;
    if (has) {
      if (lo < L1 || (lo == L1 && c < c1)) {
        L2 = L1;
        L1 = lo;
        c1 = c;
        d1 = d32;
        e1 = dlt;
      } else {
        L2 = fminf(L2, lo);
      }
    }
    const float umin = warp_minf(up);
    if (umin < U) {
      U = umin;
      refresh();
    }
  }

  // The warp's two least FP32 lower bounds (L1, L2) over every candidate
  // offered, with the candidate, value and error term of the least (ties on
  // L1 to the smaller cid); warp-uniform afterwards.
  __device__ void finish_f32() {
    // lower bounds are >= +0, so their bits order like their values
    unsigned long long k = ((unsigned long long)__float_as_uint(L1) << 32) | (unsigned)c1;
    int who = lane;
    int cw = c1;
    warp_argmin_u(k, cw);
    const unsigned m = __ballot_sync(0xffffffffu, L1 == __uint_as_float((unsigned)(k >> 32)) &&
                                                      c1 == cw);
    who = __ffs(m) - 1;
    const float l2 = warp_minf(fminf(L2, lane == who ? INFINITY : L1));
    L1 = __uint_as_float((unsigned)(k >> 32));
    L2 = l2;
    c1 = cw;
    d1 = __shfl_sync(0xffffffffu, d1, who);
    e1 = __shfl_sync(0xffffffffu, e1, who);
  }

  // exact (FP64) key of a closed-form linkage: Ward from the centroids and
  // sizes; avg-2 = ||c_A - c_B||^2 + SSE_A/|A| + SSE_B/|B| (Table 1)
  // (coordinates from d up to the row stride DP are zero on both sides: they
  // are skipped, which leaves every sum bit for bit unchanged and spares the
  // small FP64 pipe)
  __device__ unsigned long long ward64(int q, int nb, int cb) const {
    double cA[DP], cB[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      cA[k] = k < a.d ? a.cent[(size_t)ci * DP + k] : 0.0;
      cB[k] = k < a.d ? a.q64[(size_t)q * DP + k] : 0.0;
    }
    if (LK == LK_AVG2) {
      double g2 = 0.0;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        if (k < a.d) {
          const double t = cA[k] - cB[k];
          g2 += t * t;
        }
      }
      return kbits(g2 + a.sse[ci] / (double)na + a.sse[cb] / (double)nb);
    }
    return kbits(ward_key<DP>(cA, cB, na, nb, a.d));
  }

  // the records of bucket j, one per lane
  __device__ void leaf(int j, bool seed) {
    const int b = a.nch[a.chb[0] + j];
    leaf_at(b + lane, lane < a.nch[a.chb[0] + j + 1] - b && b + lane < a.K, seed);
  }

  // the candidate at position idx of this lane (in: the lane has one); the
  // 32 lanes' candidates are tested, scored and offered together
  __device__ void leaf_at(int idx, bool in, bool seed) {
    // every load of the candidate's record is issued before any test on it,
    // so a leaf step waits for memory once, not once per dependent test
    int cb = -1, qi = -1, nbq = 1, sbq = 0;
    float qc[DP], qv = 0.f;
    if (in) {
      cb = a.order[idx];
      qi = a.qinst[idx];
      nbq = a.qsz[idx];
#pragma unroll
      for (int k = 0; k < DP; ++k) qc[k] = a.q32[(size_t)idx * DP + k];
      if (LK == LK_AVERAGE || LK == LK_AVG2) qv = a.qvar[idx];
      if (LK == LK_COMPLETE || LK == LK_AVERAGE) sbq = a.qseg[idx];
    }
    const bool valid = in && cb != ci && qi == myseq;
    const int nb = valid ? nbq : 1;
    float dc2 = INFINITY, bx = 0.f;
    if (valid) {
      dc2 = 0.f;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        const float t = ci32[k] - qc[k];
        dc2 = fmaf(t, t, dc2);
        if (LK == LK_COMPLETE) {
          bx = fmaxf(bx, a.qbhi[(size_t)idx * DP + k] - alo[k]);
          bx = fmaxf(bx, ahi[k] - a.qblo[(size_t)idx * DP + k]);
        }
      }
    }
    count(C_LTESTS, __popc(__ballot_sync(0xffffffffu, valid)));
    if (LK == LK_WARD || LK == LK_AVG2) {
      float d32, dlt;  // FP32 distance (D units) and its absolute error term
      if (LK == LK_WARD) {
        const float w = valid ? ward_w(fna, (float)nb) : 0.f;
        d32 = valid ? sqrtf(w * dc2) : INFINITY;
        dlt = delta0 * sqrtf(w);
      } else {
        d32 = valid ? sqrtf(dc2 + vA + qv) : INFINITY;
        dlt = delta0;
      }
      if (MODE == M_F32) {
        const bool has = valid && (lower(d32, dlt) <= T || a.noprune);
        if (__any_sync(0xffffffffu, has)) {
          count(C_CPAIRS, __popc(__ballot_sync(0xffffffffu, has)));
          offer_f32(has, d32, dlt, cb);
        }
        return;
      }
      bool ok = valid && pass(d32);
      if (MODE == M_RECHECK) ok = ok && lower(d32, dlt) <= U;
      unsigned m = __ballot_sync(0xffffffffu, ok);
      if (!m) return;
      if (seed && __popc(m) > 1) {
        // nearest-looking candidate first: it usually settles the bound
        float v = ok ? d32 : INFINITY;
        int who = lane;
        warp_argmin_f(v, who);
        unsigned long long k = KINF;
        int c = INT_MAX;
        if (lane == who) {
          k = ward64(idx, nb, cb);
          c = cb;
        }
        count(C_CPAIRS, 1);
        if (MODE == M_RECHECK) count(C_RECHECKS, 1);
        offer_exact(k, c);
        ok = ok && lane != who && pass(d32);
        m = __ballot_sync(0xffffffffu, ok);
        if (!m) return;
      }
      unsigned long long k = KINF;
      int c = INT_MAX;
      if (ok) {
        k = ward64(idx, nb, cb);
        c = cb;
      }
      count(C_CPAIRS, __popc(m));
      if (MODE == M_RECHECK) count(C_RECHECKS, __popc(m));
      offer_exact(k, c);
      return;
    }
    // ---- complete / average ----
    if (__any_sync(0xffffffffu, valid)) {
      float ub = INFINITY;
      if (valid) {
        if (LK == LK_AVERAGE) {
          // mean ||x - y|| <= sqrt(mean ||x - y||^2) = sqrt(||c_A - c_B||^2 + var A + var B)
          // (Jensen); the FP32 centroid distance is widened by its error bound
          const float r = __fadd_ru(__fmul_ru(__fsqrt_ru(dc2), 1.f + rho), delta0);
          ub = __fsqrt_ru(__fadd_ru(__fadd_ru(__fmul_ru(r, r), vA), qv));
        } else {
          // max ||x - y|| <= distance between the farthest corners of the boxes
          float s2 = 0.f;
#pragma unroll
          for (int k = 0; k < DP; ++k) {
            const float m = fmaxf(fmaxf(__fsub_ru(a.qbhi[(size_t)idx * DP + k], alo[k]),
                                        __fsub_ru(ahi[k], a.qblo[(size_t)idx * DP + k])), 0.f);
            s2 = __fadd_ru(s2, __fmul_ru(m, m));
          }
          ub = __fsqrt_ru(s2);
        }
      }
      offer_ub(ub);
    }
    const float lb = valid ? fmaxf(sqrtf(dc2), bx) : INFINITY;
    const bool ok = valid && pass(lb);
    const int sb = valid ? sbq : 0;
    const float dlt = dpts;
    const bool small = ok && (long long)na * nb <= SMALLP;
    const unsigned sm = __ballot_sync(0xffffffffu, small);
    if (sm) {
      unsigned long long k = KINF;
      int c = INT_MAX;
      float d32 = INFINITY;
      bool rec = false;
      if (small) {
        if (MODE == M_F64) {
          k = kbits(eval64_lane<LK, DP>(a.p64, sa, na, sb, nb));
        } else {
          d32 = eval32_lane<LK, DP>(a.p32, sa, na, sb, nb);
          if (MODE == M_RECHECK && lower(d32, dlt) <= fminf(U, bd)) {
            k = kbits(eval64_lane<LK, DP>(a.p64, sa, na, sb, nb));
            rec = true;
          }
        }
        c = cb;
      }
      ppairs += __reduce_add_sync(0xffffffffu, small ? (unsigned)(na * nb) : 0u);
      count(C_PROWS, __reduce_add_sync(0xffffffffu, small ? (unsigned)(na + nb) : 0u));
      count(C_CPAIRS, __popc(sm));
      if (MODE == M_F32) {
        offer_f32(small, d32, dlt, cb);
      } else {
        if (MODE == M_RECHECK) count(C_RECHECKS, __popc(__ballot_sync(0xffffffffu, rec)));
        offer_exact(k, c);
      }
    }
    unsigned big = __ballot_sync(0xffffffffu, ok && !small);
    while (big) {
      float v = (big >> lane) & 1u ? lb : INFINITY;
      int who = lane;
      warp_argmin_f(v, who);
      big &= ~(1u << who);
      if (!pass(v)) break;  // remaining candidates have lb >= v
      const int cw = __shfl_sync(0xffffffffu, cb, who);
      const int nw = __shfl_sync(0xffffffffu, nb, who);
      const int sw = __shfl_sync(0xffffffffu, sb, who);
      unsigned long long pp = 0;
      count(C_CPAIRS, 1);
      count(C_PROWS, (unsigned long long)(na + nw));
      double cv = 0.0;
      float ce = 0.f;
      const int hit = cache_get(cw, nw, cv, ce);
      const bool cached = hit == 1;
      // values that will be cached are computed in full (no early exit)
      const bool cacheable = a.cache_slots > 0 && (long long)na * nw >= CACHE_MIN_PAIRS;
      const long long np = (long long)na * nw;
      // big pairs go to the GPU-wide kernels, and so does every pair of at
      // least BIG_MIN_PAIRS once this search has spent its own budget
      const bool over = ppairs >= (unsigned long long)a.warp_budget && np >= BIG_MIN_PAIRS;
      const bool huge = np >= a.big_pairs || over;
      const bool huge64 = np >= a.big_pairs64 || over;  // for FP64 evaluations
      // a partial entry is completed by evaluating its missing points only:
      // by the GPU-wide kernels if they are many, else in this warp
      const bool partial = hit == 2;
      const long long npm = partial ? part_pairs(nw) : 0;
      const bool hugep = npm >= a.big_pairs || (over && npm >= BIG_MIN_PAIRS);
      const bool hugep64 = npm >= a.big_pairs64 || (over && npm >= BIG_MIN_PAIRS);
      if (MODE == M_F64) {
        double key = cv;
        if (!cached) {
          if (partial && hugep64 && try_defer_part(cw, sw, nw, 1)) continue;
          if (!partial && huge64 && try_defer(cw, sw, nw, 1)) continue;
          if (partial && pe == 0.f)
            key = part64(cw, sw, nw, pp);
          else
            key = eval64_warp<LK, DP>(a.p64, sa, na, sw, nw, cacheable ? INFINITY : (double)bd,
                                      lane, pp);
          ppairs += pp;
          if (key < INFINITY) cache_put(cw, nw, key, 0.f);
        }
        const unsigned long long kb = kbits(key);
        if (key < INFINITY && kless(kb, cw, bk, bc)) {
          bk = kb;
          bc = cw;
          refresh();
        }
      } else if (MODE == M_F32) {
        float d32 = (float)cv, e32 = ce;
        if (!cached) {
          if (partial && hugep && try_defer_part(cw, sw, nw, 0)) continue;
          if (!partial && huge && try_defer(cw, sw, nw, 0)) continue;
          if (partial) {
            d32 = part32(cw, sw, nw, dlt, pp, e32);
          } else {
            d32 = eval32_warp<LK, DP>(a.p32, a.d, sa, na, sw, nw, cacheable ? INFINITY : bd, dlt,
                                      rho, lane, pp);
            e32 = dlt;
          }
          ppairs += pp;
          // an estimate's error term is never 0 in the cache (0 marks FP64)
          if (d32 < INFINITY) cache_put(cw, nw, (double)d32, fmaxf(e32, EST_MARK));
        }
        offer_f32(lane == 0 && d32 < INFINITY, d32, e32, cw);
      } else {  // M_RECHECK
        double key = INFINITY;
        if (cached && ce == 0.f) {
          key = cv;
        } else {
          float d32 = (float)cv, e32 = ce;
          if (!cached) {
            if (partial && hugep && try_defer_part(cw, sw, nw, 0)) continue;
            if (!partial && huge && try_defer(cw, sw, nw, 1)) continue;
            if (partial) {
              d32 = part32(cw, sw, nw, dlt, pp, e32);
            } else {
              d32 = eval32_warp<LK, DP>(a.p32, a.d, sa, na, sw, nw,
                                        cacheable ? INFINITY : fminf(U, bd), dlt, rho, lane, pp);
              e32 = dlt;
            }
            ppairs += pp;
          }
          if (d32 < INFINITY && lower(d32, e32) <= fminf(U, bd)) {
            if (huge64 && try_defer(cw, sw, nw, 1)) continue;
            unsigned long long pp2 = 0;
            key = eval64_warp<LK, DP>(a.p64, sa, na, sw, nw, INFINITY, lane, pp2);
            ppairs += pp2;
            count(C_RECHECKS, 1);
            cache_put(cw, nw, key, 0.f);
          }
        }
        const unsigned long long kb = kbits(key);
        if (key < INFINITY && kless(kb, cw, bk, bc)) {
          bk = kb;
          bc = cw;
          refresh();
        }
      }
    }
  }

  // Hand a big pair to the GPU-wide evaluation; the search is then re-run
  // once the value is in the cache.  Returns false if deferral is off or the
  // request queue is full (the warp evaluates the pair itself).
  __device__ bool try_defer(int cw, int sw, int nw, int exact) {
    if (!a.defer || a.cache_slots <= 0) return false;
    int r = 0;
    if (lane == 0) r = atomicAdd(&a.ctr->nbreq, 1);
    r = __shfl_sync(0xffffffffu, r, 0);
    if (r >= a.breq_cap) return false;
    if (lane == 0) {
      a.breq_i[r] = ci;
      a.breq_j[r] = cw;
      a.breq_sa[r] = sa;
      a.breq_na[r] = na;
      a.breq_sb[r] = sw;
      a.breq_nb[r] = nw;
      a.breq_exact[r] = (uint8_t)exact;
      a.breq_cov[r] = 0;
      a.breq_base[r] = 0.0;
      a.breq_berr[r] = 0.f;
    }
    deferred = true;
    return true;
  }

  // point pairs left to evaluate for the partial entry found by cache_get
  __device__ long long part_pairs(int nw) const {
    const int cov = ppart > 0 ? ppart : -ppart;
    const int on = pown_ci ? na : nw, xn = pown_ci ? nw : na;
    return (long long)(on - cov) * xn;
  }

  // the partial entry found by cache_get completed in this warp: FP32
  // estimate of the missing points, combined with the covered part (the
  // error terms combine the same way: weighted mean, or max)
  __device__ float part32(int cw, int sw, int nw, float dlt, unsigned long long &pp, float &err) {
    const int cov = ppart > 0 ? ppart : -ppart;
    const int os = pown_ci ? sa : sw, on = pown_ci ? na : nw;
    const int xs = pown_ci ? sw : sa, xn = pown_ci ? nw : na;
    const int mn = on - cov;
    const float dm = eval32_warp<LK, DP>(a.p32, a.d, ppart > 0 ? os + cov : os, mn, xs, xn,
                                         INFINITY, dlt, rho, lane, pp);
    if (LK == LK_COMPLETE) {
      err = fmaxf(pe, dlt);
      return fmaxf((float)pv, dm);
    }
    err = (float)(((double)cov * pe + (double)mn * dlt) / on);
    return (float)(((double)cov * pv + (double)mn * dm) / on);
  }

  // the same in FP64 (an FP64 partial entry)
  __device__ double part64(int cw, int sw, int nw, unsigned long long &pp) {
    const int cov = ppart > 0 ? ppart : -ppart;
    const int os = pown_ci ? sa : sw, on = pown_ci ? na : nw;
    const int xs = pown_ci ? sw : sa, xn = pown_ci ? nw : na;
    const int mn = on - cov;
    const double dm =
        eval64_warp<LK, DP>(a.p64, ppart > 0 ? os + cov : os, mn, xs, xn, INFINITY, lane, pp);
    if (LK == LK_COMPLETE) return fmax(pv, dm);
    return ((double)cov * pv + (double)mn * dm) / on;
  }

  // Complete the partial entry found by cache_get: only the points of its
  // owner that it does not cover are evaluated against the other cluster;
  // the covered part's distance (sum of distances for average) rides along.
  // An FP64 value needs an FP64 partial (pe == 0).
  __device__ bool try_defer_part(int cw, int sw, int nw, int exact) {
    if (!a.defer || a.cache_slots <= 0 || (exact && pe != 0.f)) return false;
    const int cov = ppart > 0 ? ppart : -ppart;
    const int os = pown_ci ? sa : sw, on = pown_ci ? na : nw;  // owner's points
    const int xs = pown_ci ? sw : sa, xn = pown_ci ? nw : na;  // the other cluster's
    if (cov <= 0 || cov >= on) return false;
    int r = 0;
    if (lane == 0) r = atomicAdd(&a.ctr->nbreq, 1);
    r = __shfl_sync(0xffffffffu, r, 0);
    if (r >= a.breq_cap) return false;
    if (lane == 0) {
      a.breq_i[r] = pown_ci ? ci : cw;
      a.breq_j[r] = pown_ci ? cw : ci;
      a.breq_sa[r] = ppart > 0 ? os + cov : os;  // a prefix is covered: the rest follows it
      a.breq_na[r] = on - cov;
      a.breq_sb[r] = xs;
      a.breq_nb[r] = xn;
      a.breq_exact[r] = (uint8_t)exact;
      a.breq_cov[r] = cov;
      a.breq_base[r] = LK == LK_COMPLETE ? pv : pv * (double)cov * (double)xn;
      a.breq_berr[r] = pe;
    }
    deferred = true;
    return true;
  }

  // FP64 key of (ci, the cluster at position q): the winner of an FP32 search
  // whose window held a single candidate
  __device__ unsigned long long exact_of(int q, int c) {
    const int nb = a.qsz[q];
    if (LK == LK_WARD || LK == LK_AVG2) return ward64(q, nb, c);
    double cv;
    float ce;
    const int hit = cache_get(c, nb, cv, ce);
    if (hit == 1 && ce == 0.f) return kbits(cv);
    // an FP32 value whose stated bound is within 4e-6 stands in for FP64:
    // its upper bound is returned (a valid beta; height error <= 8e-6)
    if (d1 < INFINITY && e1 + rho * d1 <= 4e-6f * d1)
      return kbits((double)((d1 + e1) * (1.f + rho)));
    if (hit == 2 && (long long)na * nb >= BIG_MIN_PAIRS && try_defer_part(c, a.qseg[q], nb, 1))
      return KINF;
    if ((long long)na * nb >= a.big_pairs64 && try_defer(c, a.qseg[q], nb, 1)) return KINF;
    unsigned long long pp = 0;
    const double key = eval64_warp<LK, DP>(a.p64, sa, na, a.qseg[q], nb, INFINITY, lane, pp);
    ppairs += pp;
    cache_put(c, nb, key, 0.f);
    return kbits(key);
  }
};

// Branch-and-bound traversal of the tree for one Searcher: the terminal's
// own bucket first (it usually settles a tight bound), then depth first from
// the nodes of the top level, nearest child first, pruning every node whose
// lower bound exceeds the threshold.
template <int LK, int DP, int MODE>
__device__ int push_children(const QueryArgs &a, const int *ti, Searcher<LK, DP, MODE> &S,
                             uint32_t *sn, float *sl, int top, int Lc, int c0, int cnt,
                             int lane) {
  const int child = c0 + lane;
  float lbc = INFINITY;
  bool ok = false;
  // (the bound on the level's node count only guards a malformed tree,
  // which the build flags as ERR_TREE)
  const bool in = lane < cnt && child < ti[Lc];
  if (in) {
    // the node's bound is computed while its instance range is still in
    // flight (both loads issued together)
    const int node = a.lvl_base[Lc] + child;
    const int ilo = a.ninlo[node], ihi = a.ninhi[node];
    const float lb = node_lb<LK, DP>(a, node, S.ci32, S.alo, S.ahi, S.fna, S.vA);
    if (ilo <= S.myseq && S.myseq <= ihi) {
      lbc = lb;
      ok = S.pass(lbc);
    }
  }
  S.count(C_NODES, __popc(__ballot_sync(0xffffffffu, in)));
  unsigned m = __ballot_sync(0xffffffffu, ok);
  if (top + __popc(m) > STK) {  // cannot happen for the level counts of tree_caps
    if (lane == 0) atomicOr(&a.ctr->err, ERR_STACK);
    m = 0;
  }
  if (m) {
    const int rank = __popc(m & ((1u << lane) - 1u));
    if (ok) {
      sn[top + rank] = ((uint32_t)Lc << 28) | (uint32_t)child;
      sl[top + rank] = lbc;
    }
    float mv = ok ? lbc : INFINITY;
    int ml = lane;
    warp_argmin_f(mv, ml);
    __syncwarp();
    if (lane == 0) {  // nearest child popped first
      const int mp = top + __popc(m & ((1u << ml) - 1u));
      const int last = top + __popc(m) - 1;
      const uint32_t tn = sn[mp];
      const float tl = sl[mp];
      sn[mp] = sn[last];
      sl[mp] = sl[last];
      sn[last] = tn;
      sl[last] = tl;
    }
    top += __popc(m);
    __syncwarp();
  }
  return top;
}

template <int LK, int DP, int MODE>
__device__ void traverse(const QueryArgs &a, const int *ti, Searcher<LK, DP, MODE> &S,
                         uint32_t *sn, float *sl, int own, int lane) {
  S.leaf(own, true);
  const int tl = ti[TI_TOP] - 1;  // top level: at most 32 nodes
  if (tl < 0 || tl > MAXLEV) {    // never for a finished build
    if (lane == 0) atomicOr(&a.ctr->err, ERR_TREE);
    return;
  }
  int top = push_children(a, ti, S, sn, sl, 0, tl, 0, min(ti[tl], FAN), lane);
  while (top > 0) {
    --top;
    const uint32_t e = sn[top];
    const float lb = sl[top];
    __syncwarp();
    if (!S.pass(lb)) continue;
    const int L = (int)(e >> 28), j = (int)(e & ((1u << 28) - 1));
    if (L == 0) {
      if (j != own) S.leaf(j, false);
      continue;
    }
    const int c0 = a.nch[a.chb[L] + j];
    top = push_children(a, ti, S, sn, sl, top, L - 1, c0, a.nch[a.chb[L] + j + 1] - c0, lane);
  }
}

// The same search over an explicit candidate list (positions, by increasing
// lower bound) written by the exhaustive candidate scan of hac_brute.cu: every
// cluster whose centroid lower bound is within the least summary upper bound
// of the terminal (that bound is offered first).
template <int LK, int DP, int MODE>
__device__ void traverse_list(const QueryArgs &a, Searcher<LK, DP, MODE> &S, int p, int cnt,
                              int lane) {
  S.offer_ub(lane == 0 ? a.lub[p] : INFINITY);
  const int32_t *L = a.lpos + (size_t)p * a.lcap;
  for (int b = 0; b < cnt; b += 32) {
    const int i = b + lane;
    S.leaf_at(i < cnt ? L[i] : 0, i < cnt, false);
  }
}


template <int LK, int DP, int PREC>
__global__ void __launch_bounds__(QWARPS * 32, qminb(LK)) k_query(QueryArgs a) {
  __shared__ uint32_t s_node[QWARPS][STK];
  __shared__ float s_lb[QWARPS][STK];
  __shared__ unsigned long long s_cnt[QWARPS][C_N];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  uint32_t *sn = s_node[wib];
  float *sl = s_lb[wib];
  unsigned long long *sc = s_cnt[wib];
  if (lane < C_N) sc[lane] = 0;
  // the tree's level counts and top level, read once per block
  __shared__ int s_ti[TI_SIZE];
  for (int i = threadIdx.x; i < TI_SIZE; i += blockDim.x) s_ti[i] = a.tinfo[i];
  __syncthreads();
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < a.nterm; t += nw) {
    const int ci = a.term[t];
    const int own = a.pbkt[a.pos[ci]];
    // a candidate list from the exhaustive scan replaces the tree traversal
    const int lc = a.lcnt ? a.lcnt[a.pos[ci]] : -1;
    unsigned long long bk;
    int bc;
    bool deferred = false;
    if (PREC == 0) {
      Searcher<LK, DP, M_F64> S(a, lane, ci, INFINITY, sc);
      if (lc >= 0)
        traverse_list(a, S, a.pos[ci], lc, lane);
      else
        traverse(a, s_ti, S, sn, sl, own, lane);
      bk = S.bk;
      bc = S.bc;
      deferred = S.deferred;
      S.count(C_PPAIRS, S.ppairs);
    } else {
      Searcher<LK, DP, M_F32> S(a, lane, ci, INFINITY, sc);
      if (lc >= 0)
        traverse_list(a, S, a.pos[ci], lc, lane);
      else
        traverse(a, s_ti, S, sn, sl, own, lane);
      S.finish_f32();
      if (S.deferred) {
        // incomplete: some candidates still wait for their values
        deferred = true;
        bk = KINF;
        bc = INT_MAX;
        S.count(C_PPAIRS, S.ppairs);
      } else if (S.L2 > S.U && S.c1 != INT_MAX) {
        // exactly one candidate can be the FP64 winner
        bc = S.c1;
        bk = S.exact_of(a.pos[bc], bc);
        S.count(C_RECHECKS, 1);
        deferred = S.deferred;
        S.count(C_PPAIRS, S.ppairs);
      } else {
        S.count(C_PPAIRS, S.ppairs);
        Searcher<LK, DP, M_RECHECK> R(a, lane, ci, S.U, sc);
        if (lc >= 0)
          traverse_list(a, R, a.pos[ci], lc, lane);
        else
          traverse(a, s_ti, R, sn, sl, own, lane);
        bk = R.bk;
        bc = R.bc;
        deferred = R.deferred;
        R.count(C_PPAIRS, R.ppairs);
      }
    }
    if (deferred) {
      // re-searched once its big pairs are in the cache
      if (lane == 0) a.pend_out[atomicAdd(&a.ctr->npend, 1)] = ci;
      continue;
    }
    if (lane == 0) {
      a.Ekey[ci] = __longlong_as_double((long long)bk);
      a.Ecid[ci] = bc == INT_MAX ? -1 : bc;
      if (bc == INT_MAX) atomicOr(&a.ctr->err, ERR_NO_NN);
    }
  }
  __syncwarp();
  if (lane == 0) {
    atomicAdd(&a.ctr->cluster_pairs, sc[C_CPAIRS]);
    atomicAdd(&a.ctr->point_pairs, sc[C_PPAIRS]);
    atomicAdd(&a.ctr->nodes, sc[C_NODES]);
    atomicAdd(&a.ctr->ltests, sc[C_LTESTS]);
    atomicAdd(&a.ctr->prows, sc[C_PROWS]);
    atomicAdd(&a.ctr->rechecks, sc[C_RECHECKS]);
    atomicAdd(&a.ctr->cache_hits, sc[C_HITS]);
  }
}

template <int LK, int PREC>
cudaError_t launch_lk(const QueryArgs &a, int dp, cudaStream_t s) {
  int blocks = (a.nterm + QWARPS - 1) / QWARPS;
  if (blocks < 1) blocks = 1;
  switch (dp) {
    case 2: k_query<LK, 2, PREC><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    case 4: k_query<LK, 4, PREC><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    case 8: k_query<LK, 8, PREC><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    case 16: k_query<LK, 16, PREC><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

// per-linkage instantiations (hac_query_<linkage>.cu, compiled in parallel)
cudaError_t launch_query_complete(const QueryArgs &a, int dp, int prec, cudaStream_t s);
cudaError_t launch_query_average(const QueryArgs &a, int dp, int prec, cudaStream_t s);
cudaError_t launch_query_ward(const QueryArgs &a, int dp, int prec, cudaStream_t s);
cudaError_t launch_query_avg2(const QueryArgs &a, int dp, int prec, cudaStream_t s);

}  // namespace hacg
