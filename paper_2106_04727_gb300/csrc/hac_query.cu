// Nearest-neighbour search of every terminal cluster (ParChain Algorithms 2-4).
//
// One warp per terminal C_i.  The active clusters sit in spatial order in
// `order`; a 32-ary implicit tree over that order stores, per node, the box of
// its clusters' centroids, the smallest cluster size under it, and (for
// complete linkage) the per-axis min of box-hi / max of box-lo.  The search is
// the paper's range query with the ball radius of Section 4 for each linkage,
// run as branch-and-bound: the radius starts from beta = pred.d (Algorithm 2)
// and shrinks to the best distance found so far, so every cluster that could
// still beat the current best is evaluated and nothing else is.
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
// candidates, never drop the true nearest neighbour.  Candidate distances are
// evaluated exactly as defined (Table 1) in FP64; the nearest neighbour is the
// candidate of least (key, cid) (ties broken lexicographically, Section 1).
//
// Key space: Ward compares D^2 = 2|A||B|/(|A|+|B|) ||c_A - c_B||^2, complete
// compares sqrt(max ||x - y||^2), average compares the mean of ||x - y||.
#include "hac_internal.cuh"

#include <cfloat>
#include <climits>

namespace hacg {

namespace {

constexpr int QWARPS = 4;          // warps per block
constexpr int STK = 256;           // per-warp stack, >= 1 + 31 * (MAXLEV - 1)
constexpr float EPS = 1e-5f;       // relative slack of the FP32 bound tests
constexpr long long SMALLP = 32;   // pairs of at most this many point pairs run per lane

enum { LK_COMPLETE = 0, LK_AVERAGE = 1, LK_WARD = 2 };

__device__ __forceinline__ bool key_less(double k1, int c1, double k2, int c2) {
  return k1 < k2 || (k1 == k2 && c1 < c2);
}

__device__ __forceinline__ void warp_argmin(double &k, int &c) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    double k2 = __shfl_xor_sync(0xffffffffu, k, o);
    int c2 = __shfl_xor_sync(0xffffffffu, c, o);
    if (key_less(k2, c2, k, c)) {
      k = k2;
      c = c2;
    }
  }
}

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

// key -> Euclidean-like distance D (Ward keys are D^2)
template <int LK>
__device__ __forceinline__ double key_to_dist(double k) {
  return LK == LK_WARD ? sqrt(k) : k;
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

// Lower bound on D(C_i, B) for every cluster B under a node, in D units.
template <int LK, int DP>
__device__ __forceinline__ float node_lb(const QueryArgs &a, int node, const float *ci32,
                                         const float *alo, const float *ahi, float na) {
  float lo[DP], hi[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    lo[k] = a.nclo[(size_t)node * DP + k];
    hi[k] = a.nchi[(size_t)node * DP + k];
  }
  float dc = sqrtf(box_d2<DP>(ci32, lo, hi));
  if (LK == LK_WARD) {
    float m = (float)a.nnmin[node];
    return dc * sqrtf(2.f * na * m / (na + m));
  }
  if (LK == LK_COMPLETE) {
    float lb = dc;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      lb = fmaxf(lb, a.nhmin[(size_t)node * DP + k] - alo[k]);
      lb = fmaxf(lb, ahi[k] - a.nlmax[(size_t)node * DP + k]);
    }
    return lb;
  }
  return dc;
}

// Lower bound on D(C_i, B) for the cluster B at position q of the order.
template <int LK, int DP>
__device__ __forceinline__ float cluster_lb(const QueryArgs &a, int q, const float *ci32,
                                            const float *alo, const float *ahi, float na,
                                            float nb) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    float t = ci32[k] - a.q32[(size_t)q * DP + k];
    s = fmaf(t, t, s);
  }
  float dc = sqrtf(s);
  if (LK == LK_WARD) return dc * sqrtf(2.f * na * nb / (na + nb));
  if (LK == LK_COMPLETE) {
    float lb = dc;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      lb = fmaxf(lb, a.qbhi[(size_t)q * DP + k] - alo[k]);
      lb = fmaxf(lb, ahi[k] - a.qblo[(size_t)q * DP + k]);
    }
    return lb;
  }
  return dc;
}

// Ward key 2|A||B|/(|A|+|B|) ||c_A - c_B||^2 in FP64 (Table 1).
template <int DP>
__device__ __forceinline__ double ward_key(const double *cA, const double *cB, int na, int nb) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    double t = cA[k] - cB[k];
    s += t * t;
  }
  return (2.0 * (double)na * (double)nb) / (double)(na + nb) * s;
}

template <int DP>
__device__ __forceinline__ double pt_d2(const double *x, const double *y) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    double t = x[k] - y[k];
    s += t * t;
  }
  return s;
}

// One lane evaluates a whole (small) pair.  Returns the key, or +inf when a
// partial result already exceeds `bound` (then B cannot be the nearest).
template <int LK, int DP>
__device__ double eval_pair_lane(const double *P, int sa, int na, int sb, int nb, double bound,
                                 unsigned long long &pp) {
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
  pp += (unsigned long long)na * nb;
  (void)bound;
  if (LK == LK_COMPLETE) return sqrt(acc);
  return acc / ((double)na * (double)nb);
}

// The whole warp evaluates one pair: lanes stride over the larger cluster's
// points, each lane loops over the smaller cluster (broadcast loads).  Exits
// early once the partial max (complete) or partial sum (average) proves the
// key exceeds `bound`.
template <int LK, int DP>
__device__ double eval_pair_warp(const double *P, int sa, int na, int sb, int nb, double bound,
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
  if (bound < INFINITY) thr = LK == LK_COMPLETE ? bound * bound * (1.0 + 1e-9) : bound * nn * (1.0 + 1e-9);
  double acc = 0.0;
  for (int base = 0; base < nL; base += 32) {
    int l = base + lane;
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
    double tot = LK == LK_COMPLETE ? warp_max(acc) : warp_sum(acc);
    int done = min(nL, base + 32);
    if (tot > thr) {
      if (lane == 0) pp += (unsigned long long)done * nS;
      return INFINITY;
    }
  }
  if (lane == 0) pp += (unsigned long long)nL * nS;
  double tot = LK == LK_COMPLETE ? warp_max(acc) : warp_sum(acc);
  if (LK == LK_COMPLETE) return sqrt(tot);
  return tot / nn;
}

template <int LK, int DP>
struct Searcher {
  const QueryArgs &a;
  int lane, ci, na;
  int sa;
  float fna;
  float ci32[DP], alo[DP], ahi[DP];
  double beta_key;     // pred's key (rounded up) or +inf
  double best_key;
  int best_cid;
  float bd;            // current bound in D units (FP32, rounded up)
  float slack;
  unsigned long long cpairs, ppairs, nodes, ltests, prows;

  __device__ Searcher(const QueryArgs &args, int lane_, int ci_) : a(args), lane(lane_), ci(ci_) {
    na = a.csize[ci];
    fna = (float)na;
    sa = a.seg ? a.seg[ci] : 0;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      ci32[k] = a.cent32[(size_t)ci * DP + k];
      alo[k] = a.blo[(size_t)ci * DP + k];
      ahi[k] = a.bhi[(size_t)ci * DP + k];
    }
    unsigned long long pv = a.pred[ci];
    beta_key = pv == PRED_EMPTY ? INFINITY : (double)__uint_as_float((unsigned)(pv >> 32));
    best_key = INFINITY;
    best_cid = INT_MAX;
    slack = (float)a.abs_slack * (LK == LK_WARD ? sqrtf(2.f * fna) : 2.f);
    cpairs = ppairs = nodes = ltests = prows = 0;
    refresh();
  }

  __device__ double bound_key() const { return fmin(beta_key, best_key); }

  __device__ void refresh() {
    double bk = bound_key();
    bd = bk == INFINITY ? INFINITY : __double2float_ru(key_to_dist<LK>(bk));
  }

  __device__ bool pass(float lb) const { return lb <= bd * (1.f + EPS) + slack; }

  __device__ void offer(double key, int cid) {
    warp_argmin(key, cid);
    if (key_less(key, cid, best_key, best_cid)) {
      best_key = key;
      best_cid = cid;
      refresh();
    }
  }

  __device__ void leaf(int j) {
    const int idx = j * FAN + lane;
    int cb = -1;
    if (idx < a.K) cb = a.order[idx];
    const bool valid = cb >= 0 && cb != ci;
    int nb = valid ? a.qsz[idx] : 1;
    float lb = INFINITY;
    if (valid) {
      lb = cluster_lb<LK, DP>(a, idx, ci32, alo, ahi, fna, (float)nb);
      ltests += 1;
    }
    bool ok = valid && pass(lb);
    if (LK == LK_WARD) {
      double key = INFINITY;
      int c = INT_MAX;
      if (ok) {
        double cA[DP], cB[DP];
#pragma unroll
        for (int k = 0; k < DP; ++k) {
          cA[k] = a.cent[(size_t)ci * DP + k];
          cB[k] = a.q64[(size_t)idx * DP + k];
        }
        key = ward_key<DP>(cA, cB, na, nb);
        c = cb;
      }
      cpairs += __popc(__ballot_sync(0xffffffffu, ok));
      offer(key, c);
      return;
    }
    // complete / average: small pairs one per lane, then the rest one warp each
    const bool small = ok && (long long)na * nb <= SMALLP;
    {
      double key = INFINITY;
      int c = INT_MAX;
      unsigned long long pp = 0;
      if (small) {
        key = eval_pair_lane<LK, DP>(a.p64, sa, na, a.qseg[idx], nb, bound_key(), pp);
        c = cb;
        prows += (unsigned long long)(na + nb);
      }
      ppairs += pp;
      unsigned sm = __ballot_sync(0xffffffffu, small);
      cpairs += __popc(sm);
      if (sm) offer(key, c);
    }
    unsigned big = __ballot_sync(0xffffffffu, ok && !small);
    while (big) {
      float v = (big >> lane) & 1u ? lb : INFINITY;
      int who = lane;
      warp_argmin_f(v, who);
      big &= ~(1u << who);
      if (!pass(v)) break;  // remaining candidates have lb >= v
      int cw = __shfl_sync(0xffffffffu, cb, who);
      int nw = __shfl_sync(0xffffffffu, nb, who);
      int sw = __shfl_sync(0xffffffffu, valid ? a.qseg[idx] : 0, who);
      unsigned long long pp = 0;
      double key = eval_pair_warp<LK, DP>(a.p64, sa, na, sw, nw, bound_key(), lane, pp);
      ppairs += pp;
      cpairs += lane == 0;
      if (lane == 0) prows += (unsigned long long)(na + nw);
      // all lanes hold the same key
      if (key_less(key, cw, best_key, best_cid)) {
        best_key = key;
        best_cid = cw;
        refresh();
      }
    }
  }
};

template <int LK, int DP>
__global__ void __launch_bounds__(QWARPS * 32) k_query64(QueryArgs a) {
  __shared__ uint32_t s_node[QWARPS][STK];
  __shared__ float s_lb[QWARPS][STK];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  uint32_t *sn = s_node[wib];
  float *sl = s_lb[wib];
  const int nlev = tree_levels(a.K);
  unsigned long long cp = 0, pp = 0, nv = 0, lt = 0, pr = 0;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < a.nterm; t += nw) {
    const int ci = a.term[t];
    Searcher<LK, DP> S(a, lane, ci);
    const int own = a.pos[ci] / FAN;
    S.leaf(own);  // seeds the bound with a spatially adjacent cluster (Alg. 2, "nearby cluster")
    int top = 0;
    if (lane == 0) {
      sn[0] = (uint32_t)(nlev - 1) << 27;
      sl[0] = 0.f;
    }
    top = 1;
    __syncwarp();
    while (top > 0) {
      --top;
      const uint32_t e = sn[top];
      const float lb = sl[top];
      __syncwarp();
      if (!S.pass(lb)) continue;
      const int L = (int)(e >> 27), j = (int)(e & ((1u << 27) - 1));
      if (L == 0) {
        if (j != own) S.leaf(j);
        continue;
      }
      const int cnt = level_count(a.K, L - 1);
      const int child = j * FAN + lane;
      float lbc = INFINITY;
      bool ok = false;
      if (child < cnt) {
        lbc = node_lb<LK, DP>(a, a.lvl_base[L - 1] + child, S.ci32, S.alo, S.ahi, S.fna);
        ok = S.pass(lbc);
        S.nodes += 1;
      }
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (m) {
        const int rank = __popc(m & ((1u << lane) - 1u));
        if (ok) {
          sn[top + rank] = ((uint32_t)(L - 1) << 27) | (uint32_t)child;
          sl[top + rank] = lbc;
        }
        float mv = ok ? lbc : INFINITY;
        int ml = lane;
        warp_argmin_f(mv, ml);
        __syncwarp();
        if (lane == 0) {  // nearest child popped first
          const int mp = top + __popc(m & ((1u << ml) - 1u));
          const int last = top + __popc(m) - 1;
          uint32_t tn = sn[mp];
          float tl = sl[mp];
          sn[mp] = sn[last];
          sl[mp] = sl[last];
          sn[last] = tn;
          sl[last] = tl;
        }
        top += __popc(m);
        __syncwarp();
      }
    }
    if (lane == 0) {
      a.Ekey[ci] = S.best_key;
      a.Ecid[ci] = S.best_cid == INT_MAX ? -1 : S.best_cid;
      if (S.best_cid == INT_MAX) atomicOr(&a.ctr->err, ERR_NO_NN);
    }
    cp += S.cpairs;
    pp += S.ppairs;
    nv += S.nodes;
    lt += S.ltests;
    pr += S.prows;
  }
  // per-warp counter totals (lane values differ for nodes; sum them)
  for (int o = 16; o; o >>= 1) {
    nv += __shfl_xor_sync(0xffffffffu, nv, o);
    pp += __shfl_xor_sync(0xffffffffu, pp, o);
    lt += __shfl_xor_sync(0xffffffffu, lt, o);
    pr += __shfl_xor_sync(0xffffffffu, pr, o);
  }
  if (lane == 0) {
    atomicAdd(&a.ctr->cluster_pairs, cp);
    atomicAdd(&a.ctr->point_pairs, pp);
    atomicAdd(&a.ctr->nodes, nv);
    atomicAdd(&a.ctr->ltests, lt);
    atomicAdd(&a.ctr->prows, pr);
  }
}

template <int LK>
cudaError_t launch_lk(const QueryArgs &a, int dp, cudaStream_t s) {
  const int warps = a.nterm;
  int blocks = (warps + QWARPS - 1) / QWARPS;
  if (blocks < 1) blocks = 1;
  switch (dp) {
    case 2: k_query64<LK, 2><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    case 4: k_query64<LK, 4><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    case 8: k_query64<LK, 8><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    case 16: k_query64<LK, 16><<<blocks, QWARPS * 32, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_query(const QueryArgs &a, int dp, int prec, cudaStream_t s) {
  (void)prec;
  if (a.nterm <= 0) return cudaSuccess;
  switch (a.linkage) {
    case LK_COMPLETE: return launch_lk<LK_COMPLETE>(a, dp, s);
    case LK_AVERAGE: return launch_lk<LK_AVERAGE>(a, dp, s);
    case LK_WARD: return launch_lk<LK_WARD>(a, dp, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace hacg
