// Tiled exhaustive nearest-neighbour search for the closed-form linkages
// (Ward, avg-2) in high dimension.
//
// In d > 8 the spatial tree of hac_query.cuh prunes little (most node boxes
// overlap every query ball), and each warp ends up reading most cluster
// records one leaf at a time.  Here a CTA holds BR_T terminals (one per
// thread) and streams the active clusters' FP32 records through shared
// memory in tiles, so each record is read once per BR_T terminals instead of
// once per terminal.  Every candidate is scored in FP32 with the error model
// of the search (|D32 - D| <= delta + rho * D); as in the FP32 pass of the
// tree search, the terminal's FP64 winner is among the candidates whose lower
// bound is at most the least upper bound U:
//   - one such candidate: it wins; its FP64 key is computed directly;
//   - more: the terminal is listed, and a second tiled pass re-scores in FP64
//     every candidate with lower bound <= U and takes the least (key, cid).
// The result is the same (key, cid) the tree search returns.  Single
// instance only (all active clusters are candidates).
#include "hac_query.cuh"

namespace hacg {

namespace {

// tile shape (the tuner's compiled variants override these)
#ifndef HAC_BR_T
#define HAC_BR_T 256
#endif
#ifndef HAC_BR_C
#define HAC_BR_C 128
#endif
constexpr int BR_T = HAC_BR_T;  // terminals per CTA
constexpr int BR_C = HAC_BR_C;  // candidate records per staged tile

template <int LK, int DP>
struct BruteTerm {
  int ci, na, mypos;
  float fna, vA, delta0, rho;
  float x[DP];

  __device__ void init(const QueryArgs &a, int c) {
    ci = c;
    na = a.csize[ci];
    fna = (float)na;
    mypos = a.pos[ci];
    vA = LK == LK_AVG2 ? a.qvar[mypos] : 0.f;
#pragma unroll
    for (int k = 0; k < DP; ++k) x[k] = a.cent32[(size_t)ci * DP + k];
    delta0 = 2.01f * U32 * a.iscale[a.inst[ci]] * sqrtf((float)a.d);
    rho = ((float)a.d + 16.f) * U32;
  }

  // FP32 distance (D units) of the candidate staged at q with size / variance
  // sv, and its absolute error term
  __device__ void score(const float *q, float sv, float &d32, float &dlt) const {
    float dc2 = 0.f;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      const float t = x[k] - q[k];
      dc2 = fmaf(t, t, dc2);
    }
    if (LK == LK_WARD) {
      const float w = ward_w(fna, sv);
      d32 = sqrtf(w * dc2);
      dlt = delta0 * sqrtf(w);
    } else {
      d32 = sqrtf(dc2 + vA + sv);
      dlt = delta0;
    }
  }

  __device__ float lower(float d32, float dlt) const { return fmaxf(d32 - dlt, 0.f) * (1.f - rho); }

  // Cheap test that a candidate's lower bound exceeds u, with no root or
  // division: lo <= u needs D32 <= u / (1 - rho) + dlt, and dlt is at most
  // dmax (Ward: delta0 sqrt(w) with w <= 2|C_i|), so a candidate whose
  // squared FP32 distance exceeds tau = (u / (1 - rho) + dmax)^2 (widened by
  // 1e-5 for the rounding of this test) cannot pass.  Ward compares
  // 2|A||B| dc2 > tau (|A| + |B|) to avoid the division in w.
  __device__ float tau(float u) const {
    if (!(u < INFINITY)) return INFINITY;
    const float dmax = LK == LK_WARD ? delta0 * sqrtf(2.f * fna) : delta0;
    const float r = u / (1.f - rho) + dmax;
    return r * r * (1.f + 1e-5f);
  }

  __device__ bool beyond(const float *q, float sv, float tq) const {
    float dc2 = 0.f;
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      const float t = x[k] - q[k];
      dc2 = fmaf(t, t, dc2);
    }
    if (LK == LK_WARD) return 2.f * fna * sv * dc2 > tq * (fna + sv);
    return dc2 + vA + sv > tq;
  }

  // FP64 key of candidate cb (by cid), as the tree search computes it
  __device__ unsigned long long exact(const QueryArgs &a, int cb) const {
    double cA[DP], cB[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      cA[k] = a.cent[(size_t)ci * DP + k];
      cB[k] = a.cent[(size_t)cb * DP + k];
    }
    const int nb = a.csize[cb];
    if (LK == LK_AVG2) {
      double g2 = 0.0;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        const double t = cA[k] - cB[k];
        g2 += t * t;
      }
      return kbits(g2 + a.sse[ci] / (double)na + a.sse[cb] / (double)nb);
    }
    return kbits(ward_key<DP>(cA, cB, na, nb, DP));
  }
};

// Stage candidate records [p0, p0 + BR_C) of the active order.
template <int LK, int DP>
__device__ __forceinline__ int stage(const QueryArgs &a, int p0, float *sq, float *sv, int *sc) {
  const int cnt = min(BR_C, a.K - p0);
  for (int i = threadIdx.x; i < cnt * DP; i += BR_T) sq[i] = a.q32[(size_t)p0 * DP + i];
  for (int j = threadIdx.x; j < cnt; j += BR_T) {
    sc[j] = a.order[p0 + j];
    sv[j] = LK == LK_WARD ? (float)a.qsz[p0 + j] : a.qvar[p0 + j];
  }
  return cnt;
}

// FP32 pass over every candidate; unique winners are final, the others are
// listed in pend_out with their U kept in Ekey.
template <int LK, int DP>
__global__ void __launch_bounds__(BR_T) k_brute(QueryArgs a) {
  __shared__ float sq[BR_C * DP];
  __shared__ float sv[BR_C];
  __shared__ int sc[BR_C];
  const int t = blockIdx.x * BR_T + threadIdx.x;
  const bool act = t < a.nterm;
  BruteTerm<LK, DP> T;
  if (act) T.init(a, a.term[t]);
  float L1 = INFINITY, L2 = INFINITY, U = INFINITY, d1 = INFINITY, e1 = 0.f, tq = INFINITY;
  int c1 = INT_MAX;
  unsigned long long offered = 0, scanned = 0;
  for (int p0 = 0; p0 < a.K; p0 += BR_C) {
    __syncthreads();
    const int cnt = stage<LK, DP>(a, p0, sq, sv, sc);
    __syncthreads();
    if (!act) continue;
    for (int j = 0; j < cnt; ++j) {
      if (p0 + j == T.mypos || T.beyond(sq + j * DP, sv[j], tq)) continue;
      float d32, dlt;
      T.score(sq + j * DP, sv[j], d32, dlt);
      const float lo = T.lower(d32, dlt);
      if (lo > U) continue;  // cannot be the FP64 winner
      const float up = (d32 + dlt) * (1.f + T.rho);
      const int cb = sc[j];
      ++offered;
      if (lo < L1 || (lo == L1 && cb < c1)) {
        L2 = L1;
        L1 = lo;
        c1 = cb;
        d1 = d32;
        e1 = dlt;
      } else {
        L2 = fminf(L2, lo);
      }
      if (up < U) {
        U = up;
        tq = T.tau(U);
      }
    }
    scanned += cnt;
  }
  if (!act) return;
  const int ci = T.ci;
  if (L2 > U && c1 != INT_MAX) {
    a.Ekey[ci] = __longlong_as_double((long long)T.exact(a, c1));
    a.Ecid[ci] = c1;
  } else {
    a.Ekey[ci] = (double)U;  // the re-score pass reads it back
    a.pend_out[atomicAdd(&a.ctr->npend, 1)] = ci;
  }
  (void)d1;
  (void)e1;
  atomicAdd(&a.ctr->cluster_pairs, offered);
  atomicAdd(&a.ctr->ltests, scanned);
}

// FP64 re-score of the listed terminals: every candidate whose FP32 lower
// bound is within U, least (FP64 key, cid) wins.
template <int LK, int DP>
__global__ void __launch_bounds__(BR_T) k_brute_recheck(QueryArgs a) {
  __shared__ float sq[BR_C * DP];
  __shared__ float sv[BR_C];
  __shared__ int sc[BR_C];
  const int m = a.ctr->npend;
  if ((int)(blockIdx.x * BR_T) >= m) return;  // uniform over the CTA
  const int t = blockIdx.x * BR_T + threadIdx.x;
  const bool act = t < m;
  BruteTerm<LK, DP> T;
  float U = 0.f, tq = 0.f;
  if (act) {
    T.init(a, a.pend_out[t]);
    U = (float)a.Ekey[T.ci];
    tq = T.tau(U);
  }
  unsigned long long bk = KINF, rechecks = 0;
  int bc = INT_MAX;
  for (int p0 = 0; p0 < a.K; p0 += BR_C) {
    __syncthreads();
    const int cnt = stage<LK, DP>(a, p0, sq, sv, sc);
    __syncthreads();
    if (!act) continue;
    for (int j = 0; j < cnt; ++j) {
      if (p0 + j == T.mypos || T.beyond(sq + j * DP, sv[j], tq)) continue;
      float d32, dlt;
      T.score(sq + j * DP, sv[j], d32, dlt);
      if (T.lower(d32, dlt) > U) continue;
      const int cb = sc[j];
      const unsigned long long k = T.exact(a, cb);
      ++rechecks;
      if (kless(k, cb, bk, bc)) {
        bk = k;
        bc = cb;
      }
    }
  }
  if (!act) return;
  a.Ekey[T.ci] = __longlong_as_double((long long)bk);
  a.Ecid[T.ci] = bc == INT_MAX ? -1 : bc;
  if (bc == INT_MAX) atomicOr(&a.ctr->err, ERR_NO_NN);
  atomicAdd(&a.ctr->rechecks, rechecks);
}

// ---------------------------------------------------------------------------
// Candidate lists for average linkage (Euclidean) in high dimension.
//
// Average linkage needs point pairs, so the exhaustive scan cannot score
// candidates itself; it replaces only the tree traversal.  Each terminal (one
// thread) streams every active cluster's FP32 record through shared memory,
// as above, and keeps:
//   U  = the least upper bound on D(C_i, B) over all B: the predecessor bound
//        beta (Algorithm 2) and the Jensen bound of each record,
//        mean ||x - y|| <= sqrt(||c_A - c_B||^2 + var A + var B), with the
//        FP32 centroid distance widened by its error bound;
//   the positions of the clusters whose centroid lower bound
//        ||c_A - c_B|| <= D(A, B) (Section 4.2) is within U (times 1 + 1e-5,
//        plus the search's absolute slack): the only clusters that can be the
//        nearest neighbour.
// The list (sorted by lower bound) and U go to the warp search, which
// evaluates those candidates as it would evaluate a tree leaf.  Tiles start at
// the CTA's own region of the spatial order, so U drops early and the list
// stays short; a list longer than BL_CAP is dropped (count -1) and that
// terminal searches the tree.
// ---------------------------------------------------------------------------
template <int DP>
__global__ void __launch_bounds__(BR_T) k_cand_avg(QueryArgs a, int32_t *lpos, float *llb,
                                                   int32_t *lcnt, float *lub) {
  constexpr int H = DP / 2;
  __shared__ __align__(16) float sq[BR_C * DP];
  __shared__ float sv[BR_C];
  const int t = blockIdx.x * BR_T + threadIdx.x;
  const bool act = t < a.nterm;
  int ci = -1, mypos = -1;
  unsigned long long x[H];
  float vA = 0.f, U = INFINITY, delta0 = 0.f, rho = 0.f, slack = 0.f;
  if (act) {
    ci = a.term[t];
    mypos = a.pos[ci];
    vA = a.qvar[mypos];
#pragma unroll
    for (int h = 0; h < H; ++h)
      x[h] = ((const unsigned long long *)(a.cent32 + (size_t)ci * DP))[h];
    const unsigned long long pv = a.pred[ci];
    if (pv != PRED_EMPTY) U = __uint_as_float((unsigned)(pv >> 32));
    const int ins = a.inst[ci];
    delta0 = 2.01f * U32 * a.iscale[ins] * sqrtf((float)a.d);
    rho = ((float)a.d + 16.f) * U32 + 32.f * U32;
    slack = a.islack[ins] * 2.f;
  }
  // candidate threshold on the squared centroid distance for the current U
  auto thr2 = [&](float u) {
    if (!(u < INFINITY)) return INFINITY;
    const float tt = u * (1.f + EPS) + slack;
    return tt * tt * (1.f + 1e-6f);
  };
  float T2 = thr2(U);
  int32_t *L = act ? lpos + (size_t)mypos * BL_CAP : nullptr;
  float *LB = act ? llb + (size_t)mypos * BL_CAP : nullptr;
  int cnt = 0;
  bool over = false;
  const int nt = (a.K + BR_C - 1) / BR_C;
  const int k0 = a.pos[a.term[blockIdx.x * BR_T]] / BR_C;  // the CTA's own region first
  unsigned long long scanned = 0;
  for (int it = 0; it < nt; ++it) {
    const int p0 = ((k0 + it) % nt) * BR_C;
    const int n_here = min(BR_C, a.K - p0);
    __syncthreads();
    for (int i = threadIdx.x; i < n_here * DP; i += BR_T) sq[i] = a.q32[(size_t)p0 * DP + i];
    for (int j = threadIdx.x; j < n_here; j += BR_T) sv[j] = a.qvar[p0 + j];
    __syncthreads();
    if (!act || over) continue;
    scanned += n_here;
    for (int j = 0; j < n_here; ++j) {
      if (p0 + j == mypos) continue;
      const unsigned long long *y = (const unsigned long long *)(sq + j * DP);
      unsigned long long tt = f2_sub(x[0], y[0]);
      unsigned long long d2 = f2_mul(tt, tt);
#pragma unroll
      for (int h = 1; h < H; ++h) {
        tt = f2_sub(x[h], y[h]);
        d2 = f2_fma(tt, tt, d2);
      }
      const float dc2 = f2_hsum(d2);
      if (dc2 <= T2) {
        if (cnt == BL_CAP) {  // full: keep only what the current U still admits
          const float tl = sqrtf(T2);
          int k = 0;
          for (int q = 0; q < cnt; ++q)
            if (LB[q] <= tl) {
              L[k] = L[q];
              LB[k] = LB[q];
              ++k;
            }
          cnt = k;
        }
        if (cnt < BL_CAP) {
          L[cnt] = p0 + j;
          LB[cnt] = sqrtf(dc2);
          ++cnt;
        } else {
          over = true;
          break;
        }
      }
      // Jensen upper bound (rounded up), only when it can lower U
      const float vB = sv[j];
      if (dc2 + vA + vB < U * U) {
        const float r = __fadd_ru(__fmul_ru(__fsqrt_ru(dc2), 1.f + rho), delta0);
        const float ub = __fsqrt_ru(__fadd_ru(__fadd_ru(__fmul_ru(r, r), vA), vB));
        if (ub < U) {
          U = ub;
          T2 = thr2(U);
        }
      }
    }
  }
  if (!act) return;
  if (!over) {
    // final filter, then insertion sort by lower bound
    const float tl = sqrtf(T2);
    int k = 0;
    for (int q = 0; q < cnt; ++q)
      if (LB[q] <= tl) {
        const int pq = L[q];
        const float lq = LB[q];
        int w = k++;
        while (w > 0 && LB[w - 1] > lq) {
          L[w] = L[w - 1];
          LB[w] = LB[w - 1];
          --w;
        }
        L[w] = pq;
        LB[w] = lq;
      }
    cnt = k;
  }
  lcnt[mypos] = over ? -1 : cnt;
  lub[mypos] = U;
  atomicAdd(&a.ctr->ltests, scanned);
}

template <int LK>
cudaError_t launch_brute_lk(const QueryArgs &a, int dp, cudaStream_t s) {
  const int blocks = (a.nterm + BR_T - 1) / BR_T;
  switch (dp) {
    case 8:
      k_brute<LK, 8><<<blocks, BR_T, 0, s>>>(a);
      k_brute_recheck<LK, 8><<<blocks, BR_T, 0, s>>>(a);
      break;
    case 16:
      k_brute<LK, 16><<<blocks, BR_T, 0, s>>>(a);
      k_brute_recheck<LK, 16><<<blocks, BR_T, 0, s>>>(a);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cand_avg(const QueryArgs &a, int32_t *lpos, float *llb, int32_t *lcnt,
                            float *lub, int dp, cudaStream_t s) {
  if (a.nterm <= 0) return cudaSuccess;
  const int blocks = (a.nterm + BR_T - 1) / BR_T;
  switch (dp) {
    case 8: k_cand_avg<8><<<blocks, BR_T, 0, s>>>(a, lpos, llb, lcnt, lub); break;
    case 16: k_cand_avg<16><<<blocks, BR_T, 0, s>>>(a, lpos, llb, lcnt, lub); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// The exhaustive search of every terminal (closed-form linkages, FP32 bulk
// with FP64 re-score, one instance); pend_out must hold nterm entries and
// ctr->npend must be 0.
cudaError_t launch_brute(const QueryArgs &a, int dp, cudaStream_t s) {
  if (a.nterm <= 0) return cudaSuccess;
  if (a.linkage == LK_WARD) return launch_brute_lk<LK_WARD>(a, dp, s);
  if (a.linkage == LK_AVG2) return launch_brute_lk<LK_AVG2>(a, dp, s);
  return cudaErrorInvalidValue;
}

}  // namespace hacg
