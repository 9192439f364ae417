// Dense phase of average linkage (avg-1): the whole matrix of pair distances
// once the active clusters fit.
//
// Section 5 keeps, per cluster, a table of up to s cached distances that
// Algorithm 5 updates by Lance-Williams after every merge.  When s reaches
// the number K of active clusters the table is the full K x K matrix, and no
// distance ever has to be evaluated twice.  On a GB300 that matrix fits for K
// in the tens of thousands (8 GiB at K = 32,768), so once K drops to that
// size this instance switches to it:
//
//   * one all-pairs sweep of the points fills it: every pair of points in
//     different clusters is visited once (the points are laid out in
//     cluster-contiguous segments in position order, so a tile of 1,024 x
//     1,024 points covers a handful of cluster pairs), and the sums of point
//     distances are accumulated per cluster pair.  For average linkage every
//     such point pair enters exactly one later merge distance, so the sweep
//     does no work the exact answer does not need;
//   * every later round finds each terminal's nearest neighbour by a scan of
//     its row (Algorithm 2 without a range query: the matrix holds every
//     candidate), and after the merges the rows and columns of the merged
//     clusters are updated by the average-linkage Lance-Williams formula
//     (Table 2: D(A u B, C) = (|A| D(A, C) + |B| D(B, C)) / (|A| + |B|));
//   * the chain update, reciprocal-pair filter, merges and compaction are the
//     ordinary round's kernels, so the rounds are those of Algorithm 1.
//
// Exact sums.  Every entry is kept as the sum of its point distances in
// 128-bit fixed point (unit 2^e, chosen per instance so that (n/2)^2 times the
// largest point distance stays below 2^126 units; stored as four 32-bit limbs
// in 64-bit words, so atomic additions need no carry), next to the mean
// distance that sum gives in FP64.  Integer addition is exact and associative, so:
//   * tiles can add into a cell with atomics in any order and the run is
//     deterministic;
//   * the Lance-Williams update of average linkage is the exact addition of
//     the sums (S(A u B, C) = S(A, C) + S(B, C)), with no rounding drift;
//   * in the FP64 mode a cell's sum is the exact sum of the FP64 point
//     distances of its pairs (each converts exactly), whatever the grouping,
//     so an FP64 re-score from the points in the FP32 mode reproduces the
//     FP64 mode's entry bit for bit, and both modes break exact ties alike.
//
// Precision.  FP64 mode: point distances in FP64, every entry exact.  FP32
// mode: the sweep uses the FP32 point copy and the stated error model of an
// FP32 point distance, |D32 - D| <= delta + rho D with rho = (d + 16) u + 32 u
// (FP32 partial sums of at most 32 terms), which sums and weighted means
// preserve; such an entry is an estimate.  A terminal's FP64 nearest
// neighbour is among the entries whose lower bound is within the least upper
// bound U; if that window holds estimates they are re-scored in FP64 from the
// points (GPU-wide) and the search is repeated, so the nearest neighbour,
// hence the tree, is the FP64 one.  A lone estimate whose bound is within
// 4e-6 relative keeps its upper bound as the height, as in the tree search.
#include "hac_impl.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

namespace hacg {

namespace {

constexpr unsigned long long KINF_D = 0x7ff0000000000000ull;  // bits of +inf
constexpr unsigned long long SIGN = 0x8000000000000000ull;

// ---------------------------------------------------------------------------
// 128-bit fixed-point sums: value = (hi * 2^64 + lo) * 2^e; the top bit of hi
// marks an estimate (sums stay below 2^126 units, so it never carries)
// ---------------------------------------------------------------------------
constexpr unsigned long long TOP = 0x8000000000000000ull;

struct U128 {
  unsigned long long lo, hi;
};

// fixed-point value of v >= 0 (exact for v >= 2^(e+52), truncated below 2^e)
__device__ __forceinline__ U128 fx_of(double v, int e) {
  U128 r{0ull, 0ull};
  if (!(v > 0.0)) return r;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  int E = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & 0xfffffffffffffull;
  if (E == 0)
    E = 1;  // subnormal
  else
    m |= 1ull << 52;
  int sh = E - 1075 - e;  // v = m * 2^(sh + e)
  if (sh > 74) sh = 74;   // cannot happen: every sum stays below 2^126 units
  if (sh >= 64) {
    r.hi = m << (sh - 64);
  } else if (sh > 0) {
    r.lo = m << sh;
    r.hi = m >> (64 - sh);
  } else if (sh == 0) {
    r.lo = m;
  } else if (sh > -64) {
    r.lo = m >> (-sh);
  }
  return r;
}

__device__ __forceinline__ void u128_add(U128 &a, const U128 &b) {
  const unsigned long long lo = a.lo + b.lo;
  a.hi += b.hi + (lo < a.lo ? 1ull : 0ull);
  a.lo = lo;
}

// A stored sum is four 64-bit words, each the sum of one 32-bit limb of
// every addend (w0 + w1 2^32 + w2 2^64 + w3 2^96), so additions need no
// carries and go out as fire-and-forget atomics; 2^32 additions per word
// cannot overflow.  The estimate flag is the top bit of w3 (sums stay below
// 2^126 units, so w3 < 2^30).
constexpr int LIMBS = 4;

// the pair i < j of a k x k matrix in the packed upper triangle
__host__ __device__ __forceinline__ size_t tri(long long i, long long j, long long k) {
  return (size_t)(i * k - i * (i + 1) / 2 + (j - i - 1));
}

__device__ __forceinline__ void limbs_atomic(unsigned long long *w, const U128 &b) {
  if (!(b.lo | b.hi)) return;
  const unsigned long long l0 = b.lo & 0xffffffffull, l1 = b.lo >> 32;
  const unsigned long long l2 = b.hi & 0xffffffffull, l3 = b.hi >> 32;
  if (l0) atomicAdd(w, l0);
  if (l1) atomicAdd(w + 1, l1);
  if (l2) atomicAdd(w + 2, l2);
  if (l3) atomicAdd(w + 3, l3);
}

// the 128-bit value of four limb words (flag bit dropped) and the flag
__device__ __forceinline__ U128 limbs_value(const unsigned long long *w) {
  const unsigned long long w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3] & ~TOP;
  U128 r;
  r.lo = w0 + (w1 << 32);
  const unsigned long long c = r.lo < w0 ? 1ull : 0ull;
  r.hi = (w1 >> 32) + w2 + (w3 << 32) + c;
  return r;
}

// fixed-point value of a non-negative float (exact above 2^(e+23))
__device__ __forceinline__ U128 fx_of_f(float v, int e) {
  U128 r{0ull, 0ull};
  if (!(v > 0.f)) return r;
  const unsigned bits = __float_as_uint(v);
  int E = (int)((bits >> 23) & 0xff);
  unsigned long long m = bits & 0x7fffffu;
  if (E == 0)
    E = 1;
  else
    m |= 1ull << 23;
  int sh = E - 150 - e;  // v = m * 2^(sh + e)
  if (sh > 102) sh = 102;
  if (sh >= 64) {
    r.hi = m << (sh - 64);
  } else if (sh > 0) {
    r.lo = m << sh;
    r.hi = sh > 40 ? m >> (64 - sh) : 0ull;
  } else if (sh == 0) {
    r.lo = m;
  } else if (sh > -64) {
    r.lo = m >> (-sh);
  }
  return r;
}

__device__ __forceinline__ U128 u128_shfl_down(const U128 &v, int o) {
  return U128{__shfl_down_sync(0xffffffffu, v.lo, o), __shfl_down_sync(0xffffffffu, v.hi, o)};
}

__device__ __forceinline__ U128 u128_shfl_xor(const U128 &v, int o) {
  return U128{__shfl_xor_sync(0xffffffffu, v.lo, o), __shfl_xor_sync(0xffffffffu, v.hi, o)};
}

// The mean distance of an entry, one function everywhere so that equal sums
// and sizes give equal means: the 128-bit sum as an FP64 number (the words
// scaled by 2^e and 2^(64+e)), times 1 / size of the cluster with the lower
// matrix index, times 1 / size of the other (reciprocals kept per matrix
// index: no FP64 division); the sign bit set for an estimate.
__device__ __forceinline__ double entry_mean(const unsigned long long *w, double sl, double sh,
                                             double inv_lo, double inv_hi) {
  const U128 v = limbs_value(w);
  const double S = fma((double)v.hi, sh, (double)v.lo * sl);
  const double m = S * inv_lo * inv_hi;
  const unsigned long long b = (unsigned long long)__double_as_longlong(m);
  return __longlong_as_double((long long)((w[3] & TOP) ? (b | SIGN) : b));
}

__device__ __forceinline__ bool is_est(double x) {
  return ((unsigned long long)__double_as_longlong(x) & SIGN) != 0;
}
__device__ __forceinline__ double mag(double x) { return fabs(x); }

// ---------------------------------------------------------------------------
// the all-pairs sweep
// ---------------------------------------------------------------------------
constexpr int DS_TPB = 256;  // threads per tile
constexpr int DS_CH = 256;   // columns per staged chunk
// FP32 sweep shape: rows per thread for d <= 8 (2 above), and the resident
// tiles per SM the register budget is cut for (the shape tuner's best at
// 10^6 points, 5-D: 4 and 4)
#ifndef HAC_DS_PPT8
#define HAC_DS_PPT8 4
#endif
#ifndef HAC_DS_MINB
#define HAC_DS_MINB 4
#endif
struct SweepArgs {
  const float *p32;
  const double *p64;
  const int32_t *plab;
  const int32_t *didx;
  int64_t N;  // points in the layout
  int dk, e;
  // FP32 sweep: coordinates times scl = 2^k (exact), so that squared
  // distances flushed to zero by the square root (below 2^-126) are below
  // 2^(-126-2k) unscaled; sums of scaled distances convert with unit 2^es,
  // es = e + k, to the same fixed-point values
  float scl;
  int es;
  unsigned long long *sum;  // the packed upper triangle of sums (LIMBS words per pair)
  long long nb;             // blocks of TI points along each axis
  Counters *ctr;
};

__device__ __forceinline__ void tile_of(long long t, long long &bi, long long &bj) {
  long long j = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (j * (j + 1) / 2 > t) --j;
  while ((j + 1) * (j + 2) / 2 <= t) ++j;
  bj = j;
  bi = t - j * (j + 1) / 2;
}

// Per chunk: segment starts of equal keys (cluster matrix indices) among the
// staged columns; returns the count, sstart[count] = cnt.
__device__ __forceinline__ int chunk_segments(const int *skey, int cnt, int *sstart, int *wtot) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const bool flag = t < cnt && (t == 0 || skey[t] != skey[t - 1]);
  const unsigned b = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) wtot[w] = __popc(b);
  __syncthreads();
  int before = 0, total = 0;
  for (int i = 0; i < DS_TPB / 32; ++i) {
    before += i < w ? wtot[i] : 0;
    total += wtot[i];
  }
  if (flag) sstart[before + __popc(b & ((1u << lane) - 1u))] = t;
  if (t == 0) sstart[total] = cnt;
  __syncthreads();
  return total;
}

// Keys of a warp's rows are non-decreasing along the lanes, so equal keys
// form contiguous runs.  `same` holds, per step o = 1, 2, 4, 8, 16, whether
// lane + o has this lane's key; after seg_sum the first lane of each run
// holds the run's total.
__device__ __forceinline__ unsigned seg_mask(int k, int lane) {
  unsigned m = 0;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int k2 = __shfl_down_sync(0xffffffffu, k, 1 << i);
    if (lane + (1 << i) < 32 && k2 == k) m |= 1u << i;
  }
  return m;
}

__device__ __forceinline__ U128 seg_sum(U128 v, unsigned same) {
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const U128 v2 = u128_shfl_down(v, 1 << i);
    if ((same >> i) & 1u) u128_add(v, v2);
  }
  return v;
}

// Row layout of a warp: lane l holds PPT consecutive rows, r0 + l * PPT + r,
// so a lane's rows mostly share one key (cluster), and keys are
// non-decreasing along (lane, r).  Per lane: its head run (key of row 0), its
// tail run (key of row PPT - 1), and any runs wholly inside the lane.
struct RowKeys {
  int head, tail;
  unsigned same;  // seg_mask of the tail keys
  bool lead;      // first lane of its tail run
  bool absorbed;  // the head run continues the previous lane's tail run
  bool split;     // head != tail
};

// Row setup shared by both sweeps; returns whether all rows of the warp
// share one key.
template <int PPT>
__device__ __forceinline__ bool row_keys(const SweepArgs &a, long long r0, int lane,
                                         int (&krow)[PPT], RowKeys &rk, int &kfirst) {
#pragma unroll
  for (int r = 0; r < PPT; ++r) {
    const long long row = r0 + (long long)lane * PPT + r;
    krow[r] = row < a.N ? a.didx[a.plab[row]] : INT_MAX;
  }
  rk.head = krow[0];
  rk.tail = krow[PPT - 1];
  rk.split = rk.head != rk.tail;
  rk.same = seg_mask(rk.tail, lane);
  const int pt = __shfl_up_sync(0xffffffffu, rk.tail, 1);
  rk.lead = lane == 0 || pt != rk.tail;
  rk.absorbed = lane > 0 && rk.split && pt == rk.head;
  kfirst = __shfl_sync(0xffffffffu, rk.head, 0);
  const int klast = __shfl_sync(0xffffffffu, rk.tail, 31);
  return kfirst == klast;
}

// Flush one column segment (key qj) of every row: cell (key, qj) gets the
// sum of the rows with that key when key < qj (each unordered cluster pair
// once, its lower matrix index first).  Runs inside a lane are summed there;
// a head run that continues the previous lane's tail is handed to it; the
// tails are summed over each run of lanes by one segmented reduction.
template <int PPT>
__device__ __forceinline__ void flush(const SweepArgs &a, const U128 (&acc)[PPT],
                                      const int (&krow)[PPT], const RowKeys &rk, bool uniform,
                                      int qj, int lane) {
  if (uniform) {  // every row of the warp in one cluster
    if (!(krow[0] < qj)) return;
    U128 v = acc[0];
#pragma unroll
    for (int r = 1; r < PPT; ++r) u128_add(v, acc[r]);
#pragma unroll
    for (int o = 16; o; o >>= 1) u128_add(v, u128_shfl_xor(v, o));
    if (lane == 0) limbs_atomic(&a.sum[LIMBS * tri(krow[0], qj, a.dk)], v);
    return;
  }
  U128 vh{0ull, 0ull}, vt{0ull, 0ull};
#pragma unroll
  for (int r = 0; r < PPT; ++r) {
    if (krow[r] == rk.tail)
      u128_add(vt, acc[r]);
    else if (krow[r] == rk.head)
      u128_add(vh, acc[r]);
  }
  if (rk.split) {
    // runs wholly inside this lane (a cluster of fewer than PPT points here)
    int k = -1;
    U128 m{0ull, 0ull};
#pragma unroll
    for (int r = 0; r < PPT; ++r) {
      const int kr = krow[r];
      if (kr == rk.head || kr == rk.tail) continue;
      if (kr != k) {
        if (k >= 0 && k < qj) limbs_atomic(&a.sum[LIMBS * tri(k, qj, a.dk)], m);
        k = kr;
        m = U128{0ull, 0ull};
      }
      u128_add(m, acc[r]);
    }
    if (k >= 0 && k < qj) limbs_atomic(&a.sum[LIMBS * tri(k, qj, a.dk)], m);
  }
  // the next lane's head joins this tail when it continues the run
  const U128 nh = u128_shfl_down(vh, 1);
  const bool nabs = __shfl_down_sync(0xffffffffu, rk.absorbed, 1);
  if (lane < 31 && nabs) u128_add(vt, nh);
  if (rk.split && !rk.absorbed && rk.head < qj)
    limbs_atomic(&a.sum[LIMBS * tri(rk.head, qj, a.dk)], vh);
  vt = seg_sum(vt, rk.same);
  if (rk.lead && rk.tail < qj) limbs_atomic(&a.sum[LIMBS * tri(rk.tail, qj, a.dk)], vt);
}

// FP32 sweep, specialised on the true dimension D (rows of stride DP
// floats), PPT rows per thread; a tile is TI x TI points, TI = 256 * PPT.
// Two of a thread's rows share each f32x2 word (one coordinate of each) and
// every staged column is duplicated into both halves, so one packed subtract
// and one packed multiply-add advance two point pairs by one coordinate.  Per
// row and column segment: FP32 partial sums of at most 32 terms, each
// converted to fixed point exactly and added as integers (no FP64 work).
template <int D, int DP, int PPT>
__global__ void __launch_bounds__(DS_TPB, HAC_DS_MINB) k_dense_sweep32(SweepArgs a) {
  constexpr int TI = DS_TPB * PPT, NP = PPT / 2;
  __shared__ unsigned long long sy[DS_CH * D];
  __shared__ int skey[DS_CH];
  __shared__ int sstart[DS_CH + 1];
  __shared__ int wtot[DS_TPB / 32];
  long long bi, bj;
  tile_of(blockIdx.x + (long long)gridDim.x * blockIdx.y, bi, bj);
  if (bi >= a.nb || bj >= a.nb) return;  // uniform over the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r0 = bi * TI + (long long)w * 32 * PPT;
  unsigned long long x[NP][D];
  int krow[PPT];
  RowKeys rk;
  int kfirst;
  const bool uniform = row_keys<PPT>(a, r0, lane, krow, rk, kfirst);
#pragma unroll
  for (int h = 0; h < NP; ++h) {
    const long long ra = r0 + (long long)lane * PPT + 2 * h, rb = ra + 1;
#pragma unroll
    for (int k = 0; k < D; ++k)
      x[h][k] = f2_pack(ra < a.N ? a.p32[(size_t)ra * DP + k] * a.scl : 0.f,
                        rb < a.N ? a.p32[(size_t)rb * DP + k] * a.scl : 0.f);
  }
  unsigned long long pairs = 0;
  for (int ch = 0; ch < PPT; ++ch) {  // TI columns in chunks of DS_CH
    const long long c0 = bj * TI + (long long)ch * DS_CH;
    if (c0 >= a.N) break;  // uniform
    const int cnt = (int)min((long long)DS_CH, a.N - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * D; i += DS_TPB) {
      const int c = i / D, k = i - c * D;
      const float y = a.p32[(size_t)(c0 + c) * DP + k] * a.scl;
      sy[i] = f2_pack(y, y);
    }
    if (threadIdx.x < DS_CH)
      skey[threadIdx.x] = threadIdx.x < cnt ? a.didx[a.plab[c0 + threadIdx.x]] : -1;
    __syncthreads();
    const int nseg = chunk_segments(skey, cnt, sstart, wtot);
    for (int sg = 0; sg < nseg; ++sg) {
      const int cb = sstart[sg], ce = sstart[sg + 1];
      const int qj = skey[cb];
      if (qj <= kfirst) continue;  // no row of this warp pairs with it (uniform)
      U128 acc[PPT];
#pragma unroll
      for (int r = 0; r < PPT; ++r) acc[r] = U128{0ull, 0ull};
      for (int c1 = cb; c1 < ce; c1 += 32) {
        const int c2 = min(c1 + 32, ce);
        float part[PPT];
#pragma unroll
        for (int r = 0; r < PPT; ++r) part[r] = 0.f;
#pragma unroll 2
        for (int c = c1; c < c2; ++c) {
          unsigned long long y[D];
#pragma unroll
          for (int k = 0; k < D; ++k) y[k] = sy[c * D + k];
#pragma unroll
          for (int h = 0; h < NP; ++h) {
            unsigned long long t = f2_sub(x[h][0], y[0]);
            unsigned long long d2 = f2_mul(t, t);
#pragma unroll
            for (int k = 1; k < D; ++k) {
              t = f2_sub(x[h][k], y[k]);
              d2 = f2_fma(t, t, d2);
            }
            float s0, s1;
            f2_unpack(d2, s0, s1);
            part[2 * h] += sqrt_approx_ftz(s0);
            part[2 * h + 1] += sqrt_approx_ftz(s1);
          }
        }
#pragma unroll
        for (int r = 0; r < PPT; ++r) u128_add(acc[r], fx_of_f(part[r], a.es));
      }
      int below = 0;
#pragma unroll
      for (int r = 0; r < PPT; ++r) below += krow[r] < qj;
      pairs += (unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)below) * (ce - cb);
      flush<PPT>(a, acc, krow, rk, uniform, qj, lane);
    }
  }
  if (lane == 0 && pairs) atomicAdd(&a.ctr->dense_pp, pairs);
}

// FP64 sweep: the same tiles, FP64 coordinates; every point distance is
// added to the row's 128-bit sum exactly.
template <int DP, int PPT>
__global__ void __launch_bounds__(DS_TPB) k_dense_sweep64(SweepArgs a) {
  constexpr int TI = DS_TPB * PPT;
  __shared__ double sy[DS_CH * DP];
  __shared__ int skey[DS_CH];
  __shared__ int sstart[DS_CH + 1];
  __shared__ int wtot[DS_TPB / 32];
  long long bi, bj;
  tile_of(blockIdx.x + (long long)gridDim.x * blockIdx.y, bi, bj);
  if (bi >= a.nb || bj >= a.nb) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r0 = bi * TI + (long long)w * 32 * PPT;
  double x[PPT][DP];
  int krow[PPT];
  RowKeys rk;
  int kfirst;
  const bool uniform = row_keys<PPT>(a, r0, lane, krow, rk, kfirst);
#pragma unroll
  for (int r = 0; r < PPT; ++r) {
    const long long row = r0 + (long long)lane * PPT + r;
#pragma unroll
    for (int k = 0; k < DP; ++k) x[r][k] = row < a.N ? a.p64[(size_t)row * DP + k] : 0.0;
  }
  unsigned long long pairs = 0;
  for (int ch = 0; ch < PPT; ++ch) {
    const long long c0 = bj * TI + (long long)ch * DS_CH;
    if (c0 >= a.N) break;
    const int cnt = (int)min((long long)DS_CH, a.N - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt * DP; i += DS_TPB) sy[i] = a.p64[(size_t)c0 * DP + i];
    if (threadIdx.x < DS_CH)
      skey[threadIdx.x] = threadIdx.x < cnt ? a.didx[a.plab[c0 + threadIdx.x]] : -1;
    __syncthreads();
    const int nseg = chunk_segments(skey, cnt, sstart, wtot);
    for (int sg = 0; sg < nseg; ++sg) {
      const int cb = sstart[sg], ce = sstart[sg + 1];
      const int qj = skey[cb];
      if (qj <= kfirst) continue;
      U128 acc[PPT];
#pragma unroll
      for (int r = 0; r < PPT; ++r) acc[r] = U128{0ull, 0ull};
      for (int c = cb; c < ce; ++c) {
        const double *y = sy + c * DP;
#pragma unroll
        for (int r = 0; r < PPT; ++r) {
          double d2 = 0.0;
#pragma unroll
          for (int k = 0; k < DP; ++k) {
            const double t = x[r][k] - y[k];
            d2 = fma(t, t, d2);
          }
          u128_add(acc[r], fx_of(sqrt(d2), a.e));
        }
      }
      int below = 0;
#pragma unroll
      for (int r = 0; r < PPT; ++r) below += krow[r] < qj;
      pairs += (unsigned long long)__reduce_add_sync(0xffffffffu, (unsigned)below) * (ce - cb);
      flush<PPT>(a, acc, krow, rk, uniform, qj, lane);
    }
  }
  if (lane == 0 && pairs) atomicAdd(&a.ctr->dense_pp, pairs);
}

// Sums -> means: both triangles of the mean matrix (+inf on the diagonal);
// an estimate (FP32 mode) gets its flag in the sum.  32 x 32 tiles of the
// upper triangle with their mirror tile, written through shared memory so
// every global access is a row segment.
__global__ void k_dense_fin(State s, int dk, bool est) {
  __shared__ double Mv[32][33];
  const int nt = (dk + 31) / 32;
  long long ti, tj;
  tile_of(blockIdx.x + (long long)gridDim.x * blockIdx.y, ti, tj);
  if (ti >= nt || tj >= nt) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int k = ty; k < 32; k += 8) {
    const long long i = ti * 32 + k, j = tj * 32 + tx;  // the upper tile
    double v = 0.0;
    if (i < dk && j < dk) {
      if (i == j) {
        v = __longlong_as_double((long long)KINF_D);
      } else if (i < j) {
        unsigned long long *c = s.dsum + LIMBS * tri(i, j, dk);
        if (est) c[3] |= TOP;
        v = entry_mean(c, s.dsl, s.dsh, s.dinv[i], s.dinv[j]);
      }
    }
    Mv[k][tx] = v;
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const long long i = ti * 32 + k, j = tj * 32 + tx;
    if (i < dk && j < dk)  // diagonal tile: the lower cells take the upper cells' means
      s.dmat[(size_t)i * dk + j] = ti == tj && i > j ? Mv[tx][k] : Mv[k][tx];
    if (ti != tj) {  // mirror tile: row tj*32+k, column ti*32+tx = upper cell (tx, k)
      const long long i2 = tj * 32 + k, j2 = ti * 32 + tx;
      if (i2 < dk && j2 < dk) s.dmat[(size_t)i2 * dk + j2] = Mv[tx][k];
    }
  }
}

__global__ void k_dense_init(State s, const int32_t *order, int K) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < K; p += gridDim.x * blockDim.x) {
    const int c = order[p];
    s.didx[c] = p;
    s.dcid[p] = c;
    s.dinv[p] = 1.0 / (double)s.qsz[p];
  }
}

// ---------------------------------------------------------------------------
// nearest neighbours on the matrix: one warp per terminal, a scan of its row
// ---------------------------------------------------------------------------
struct NNArgs {
  const double *dmat;
  int dk, K, nlist;
  const int32_t *order, *didx, *list, *dq;
  // FP32 mode: error model of an estimate x of the FP64 value D,
  // |x - D| <= delta + rho D + eta; eta (absolute) covers the sums' fixed-
  // point truncation (below one unit 2^e per partial sum, on both sides)
  // and the square roots' flush of squared distances below 2^-126 (scaled)
  double delta, rho, eta;
  // FP32 mode with delta = 0: the bounds as steps of the FP64 bit pattern
  // (adding N ulps to a non-negative double multiplies it by at least
  // 1 + N 2^-53): for x >= m0 (so eta <= 2^-30 x) up = x + nu ulps >=
  // (x + eta) / (1 - rho) and lo = x - nl ulps <= (x - eta) / (1 + rho) (nl
  // doubled for a step down across a power of two); an estimate below m0
  // spans [0, m0up] (m0up = 2 m0 >= its upper bound)
  unsigned long long nu, nl, m0, m0up;
  double *Ekey;
  int32_t *Ecid;
  int32_t *drq_a, *drq_b;
  int drq_cap;
  int32_t *pend_out;
  Counters *ctr;
};

__device__ __forceinline__ bool kless_d(unsigned long long k1, int c1, unsigned long long k2,
                                        int c2) {
  return k1 < k2 || (k1 == k2 && c1 < c2);
}

__device__ __forceinline__ void warp_argmin_kc(unsigned long long &k, int &c) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
    const int c2 = __shfl_xor_sync(0xffffffffu, c, o);
    if (kless_d(k2, c2, k, c)) {
      k = k2;
      c = c2;
    }
  }
}

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// One warp per terminal; each lane has NN_U loads of the row in flight.
constexpr int NN_U = 4;

template <int F32>
__global__ void k_dense_nn(NNArgs a) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long tests = 0;
  for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < a.nlist; t += nw) {
    const int ci = a.list[t];
    const int qi = a.didx[ci];
    const double *row = a.dmat + (size_t)qi * a.dk;
    tests += (unsigned long long)(a.K - 1);
    if (!F32) {
      unsigned long long bk = KINF_D;
      int bc = INT_MAX;
      for (int p0 = 0; p0 < a.K; p0 += 32 * NN_U) {
        unsigned long long k[NN_U];
        int c[NN_U];
#pragma unroll
        for (int u = 0; u < NN_U; ++u) {
          const int p = p0 + u * 32 + lane;
          c[u] = p < a.K ? a.order[p] : ci;
          k[u] = p < a.K ? (unsigned long long)__double_as_longlong(row[a.dq[p]]) : KINF_D;
        }
#pragma unroll
        for (int u = 0; u < NN_U; ++u)
          if (c[u] != ci && kless_d(k[u], c[u], bk, bc)) {
            bk = k[u];
            bc = c[u];
          }
      }
      warp_argmin_kc(bk, bc);
      if (lane == 0) {
        a.Ekey[ci] = __longlong_as_double((long long)bk);
        a.Ecid[ci] = bc == INT_MAX ? -1 : bc;
        if (bc == INT_MAX) atomicOr(&a.ctr->err, ERR_NO_NN);
      }
      continue;
    }
    if (F32 == 2) {
      // FP32 mode, integer bounds (no FP64 arithmetic in the scan)
      unsigned long long U = ~0ull;
      for (int p0 = 0; p0 < a.K; p0 += 32 * NN_U) {
        unsigned long long x[NN_U];
        int c[NN_U];
#pragma unroll
        for (int u = 0; u < NN_U; ++u) {
          const int p = p0 + u * 32 + lane;
          c[u] = p < a.K ? a.order[p] : ci;
          x[u] = p < a.K ? (unsigned long long)__double_as_longlong(row[a.dq[p]]) : KINF_D;
        }
#pragma unroll
        for (int u = 0; u < NN_U; ++u) {
          if (c[u] == ci) continue;
          const unsigned long long m = x[u] & ~SIGN;
          const unsigned long long up = (x[u] & SIGN) ? (m < a.m0 ? a.m0up : m + a.nu) : m;
          U = up < U ? up : U;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const unsigned long long u2 = __shfl_xor_sync(0xffffffffu, U, o);
        U = u2 < U ? u2 : U;
      }
      unsigned long long bk = KINF_D, ev = 0;
      int bc = INT_MAX, nW = 0, nE = 0, ec = INT_MAX;
      for (int p0 = 0; p0 < a.K; p0 += 32 * NN_U) {
        unsigned long long x[NN_U];
        int c[NN_U];
#pragma unroll
        for (int u = 0; u < NN_U; ++u) {
          const int p = p0 + u * 32 + lane;
          c[u] = p < a.K ? a.order[p] : ci;
          x[u] = p < a.K ? (unsigned long long)__double_as_longlong(row[a.dq[p]]) : KINF_D;
        }
#pragma unroll
        for (int u = 0; u < NN_U; ++u) {
          if (c[u] == ci) continue;
          const unsigned long long m = x[u] & ~SIGN;
          const bool exact = !(x[u] & SIGN);
          const unsigned long long lo = exact ? m : (m < a.m0 ? 0ull : m - a.nl);
          if (lo > U) continue;
          ++nW;
          if (exact) {
            if (kless_d(m, c[u], bk, bc)) {
              bk = m;
              bc = c[u];
            }
          } else {
            ++nE;
            ec = c[u];
            ev = m;
          }
        }
      }
      warp_argmin_kc(bk, bc);
      const int totW = __reduce_add_sync(0xffffffffu, (unsigned)nW);
      const int totE = __reduce_add_sync(0xffffffffu, (unsigned)nE);
      if (totE == 0) {
        if (lane == 0) {
          a.Ekey[ci] = __longlong_as_double((long long)bk);
          a.Ecid[ci] = bc == INT_MAX ? -1 : bc;
          if (bc == INT_MAX) atomicOr(&a.ctr->err, ERR_NO_NN);
        }
        continue;
      }
      if (totW == 1) {
        // the lone candidate is an estimate; rho <= 4e-6 here (checked by the
        // host), so its upper bound stands in for the FP64 value, unless the
        // absolute term dominates it (below m0: re-scored)
        const unsigned holder = __ballot_sync(0xffffffffu, nE > 0);
        const int hl = __ffs(holder) - 1;
        const unsigned long long v = __shfl_sync(0xffffffffu, ev, hl);
        const int c = __shfl_sync(0xffffffffu, ec, hl);
        if (v >= a.m0) {
          if (lane == 0) {
            a.Ekey[ci] = __longlong_as_double((long long)(v + a.nu));
            a.Ecid[ci] = c;
          }
          continue;
        }
      }
      // several candidates in the window: re-score its estimates in FP64
      for (int p = lane; p < a.K; p += 32) {
        const int c = a.order[p];
        if (c == ci) continue;
        const int q = a.dq[p];
        const unsigned long long xb = (unsigned long long)__double_as_longlong(row[q]);
        const unsigned long long m = xb & ~SIGN;
        if (!(xb & SIGN) || (m < a.m0 ? 0ull : m - a.nl) > U) continue;
        const int r = atomicAdd(&a.ctr->nrq, 1);
        if (r < a.drq_cap) {
          a.drq_a[r] = min(qi, q);
          a.drq_b[r] = max(qi, q);
        }
      }
      if (lane == 0) a.pend_out[atomicAdd(&a.ctr->npend, 1)] = ci;
      continue;
    }
    // FP32 mode.  Bounds of an estimate x on the FP64 value D:
    // (x - delta - eta) / (1 + rho) <= D <= (x + delta + eta) / (1 - rho),
    // widened by 1e-12 for the rounding of these FP64 operations.
    const double dl = a.delta + a.eta;
    // x - dl rounds by up to 2^-52 max(x, dl): when x is close to dl that is
    // not within the relative 1e-12, so the lower bound subtracts a little more
    const double dlo = dl * (1.0 + 0x1p-50);
    const double lo_f = (1.0 - 1e-12) / (1.0 + a.rho), up_f = (1.0 + 1e-12) / (1.0 - a.rho);
    double U = INFINITY;
    for (int p0 = 0; p0 < a.K; p0 += 32 * NN_U) {
      double x[NN_U];
      int c[NN_U];
#pragma unroll
      for (int u = 0; u < NN_U; ++u) {
        const int p = p0 + u * 32 + lane;
        c[u] = p < a.K ? a.order[p] : ci;
        x[u] = p < a.K ? row[a.dq[p]] : INFINITY;
      }
#pragma unroll
      for (int u = 0; u < NN_U; ++u) {
        if (c[u] == ci) continue;
        const double m = mag(x[u]);
        const bool exact = !is_est(x[u]);
        U = fmin(U, exact ? m : (m + dl) * up_f);
      }
    }
    U = warp_min_d(U);
    unsigned long long bk = KINF_D;
    int bc = INT_MAX, nW = 0, nE = 0, ec = INT_MAX;
    double ev = 0.0;
    for (int p0 = 0; p0 < a.K; p0 += 32 * NN_U) {
      double x[NN_U];
      int c[NN_U];
#pragma unroll
      for (int u = 0; u < NN_U; ++u) {
        const int p = p0 + u * 32 + lane;
        c[u] = p < a.K ? a.order[p] : ci;
        x[u] = p < a.K ? row[a.dq[p]] : INFINITY;
      }
#pragma unroll
      for (int u = 0; u < NN_U; ++u) {
        if (c[u] == ci) continue;
        const double m = mag(x[u]);
        const bool exact = !is_est(x[u]);
        const double lo = exact ? m : fmax(m - dlo, 0.0) * lo_f;
        if (!(lo <= U)) continue;
        ++nW;
        if (exact) {
          const unsigned long long k = (unsigned long long)__double_as_longlong(m);
          if (kless_d(k, c[u], bk, bc)) {
            bk = k;
            bc = c[u];
          }
        } else {
          ++nE;
          ec = c[u];
          ev = m;
        }
      }
    }
    warp_argmin_kc(bk, bc);
    const int totW = __reduce_add_sync(0xffffffffu, (unsigned)nW);
    const int totE = __reduce_add_sync(0xffffffffu, (unsigned)nE);
    if (totE == 0) {
      if (lane == 0) {
        a.Ekey[ci] = __longlong_as_double((long long)bk);
        a.Ecid[ci] = bc == INT_MAX ? -1 : bc;
        if (bc == INT_MAX) atomicOr(&a.ctr->err, ERR_NO_NN);
      }
      continue;
    }
    if (totW == 1) {
      // the lone candidate is an estimate: its upper bound stands in for
      // the FP64 value when the stated bound is within 4e-6 relative
      const unsigned holder = __ballot_sync(0xffffffffu, nE > 0);
      const int hl = __ffs(holder) - 1;
      const double v = __shfl_sync(0xffffffffu, ev, hl);
      const int c = __shfl_sync(0xffffffffu, ec, hl);
      if (dl + a.rho * v <= 4e-6 * v) {
        if (lane == 0) {
          a.Ekey[ci] = (v + dl) * up_f;
          a.Ecid[ci] = c;
        }
        continue;
      }
      if (lane == hl) {
        const int r = atomicAdd(&a.ctr->nrq, 1);
        if (r < a.drq_cap) {
          const int q = a.didx[c];
          a.drq_a[r] = min(qi, q);
          a.drq_b[r] = max(qi, q);
        }
      }
    } else {
      // several candidates in the window: re-score its estimates in FP64
      for (int p = lane; p < a.K; p += 32) {
        const int c = a.order[p];
        if (c == ci) continue;
        const int q = a.dq[p];
        const double x = row[q];
        const double m = mag(x);
        const bool exact = !is_est(x);
        if (exact || !(fmax(m - dlo, 0.0) * lo_f <= U)) continue;
        const int r = atomicAdd(&a.ctr->nrq, 1);
        if (r < a.drq_cap) {
          a.drq_a[r] = min(qi, q);
          a.drq_b[r] = max(qi, q);
        }
      }
    }
    if (lane == 0) a.pend_out[atomicAdd(&a.ctr->npend, 1)] = ci;
  }
  for (int o = 16; o; o >>= 1) tests += __shfl_xor_sync(0xffffffffu, tests, o);
  if (lane == 0 && tests) atomicAdd(&a.ctr->ltests, tests);
}

// ---------------------------------------------------------------------------
// FP64 re-score of listed pairs from the points (GPU-wide)
// ---------------------------------------------------------------------------
constexpr int RQ_TPB = 256;   // rows (points of the first cluster) per tile
constexpr int RQ_COLS = 1024; // points of the second cluster per tile
constexpr int RQ_CH = 128;    // staged per chunk

__global__ void k_drq_count(State s, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int A = s.dcid[s.drq_a[i]], B = s.dcid[s.drq_b[i]];
    const long long na = s.csize[A], nb = s.csize[B];
    s.drq_pre[i] = (int32_t)(((na + RQ_TPB - 1) / RQ_TPB) * ((nb + RQ_COLS - 1) / RQ_COLS));
  }
}

// exclusive scan of m tile counts into drq_pre (one block; total at [m])
__global__ void k_drq_scan(State s, int m) {
  __shared__ long long part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (m + T - 1) / T, b0 = t * per;
  long long sum = 0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < m) sum += s.drq_pre[b0 + i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int i = 0; i < T; ++i) {
      const long long v = part[i];
      part[i] = run;
      run += v;
    }
    s.drq_pre[m] = (int32_t)min(run, (long long)INT_MAX);
    if (run > INT_MAX) atomicOr(&s.ctr->err, ERR_WINDOW);  // far beyond any real queue
  }
  __syncthreads();
  long long run = part[t];
  for (int i = 0; i < per; ++i)
    if (b0 + i < m) {
      const long long v = s.drq_pre[b0 + i];
      s.drq_pre[b0 + i] = (int32_t)run;
      run += v;
    }
}

template <int DP>
__global__ void __launch_bounds__(RQ_TPB) k_drq_eval(State s, int m, int cur) {
  __shared__ double sy[RQ_CH * DP];
  __shared__ unsigned long long rlo[RQ_TPB / 32], rhi[RQ_TPB / 32];
  const int total = s.drq_pre[m];
  const double *P = s.p64[cur];
  const int32_t *seg = s.seg[cur];
  for (int t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = m - 1;  // last i with pre[i] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s.drq_pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int i = lo;
    const int A = s.dcid[s.drq_a[i]], B = s.dcid[s.drq_b[i]];
    const int na = s.csize[A], nb = s.csize[B];
    const int tbn = (nb + RQ_COLS - 1) / RQ_COLS;
    const int j = t - s.drq_pre[i];
    const int ta = j / tbn, tb = j - ta * tbn;
    const int row = ta * RQ_TPB + threadIdx.x;
    double x[DP];
    const bool act = row < na;
#pragma unroll
    for (int k = 0; k < DP; ++k) x[k] = act ? P[(size_t)(seg[A] + row) * DP + k] : 0.0;
    U128 acc{0ull, 0ull};
    const int cbeg = tb * RQ_COLS, cend = min(nb, cbeg + RQ_COLS);
    for (int c0 = cbeg; c0 < cend; c0 += RQ_CH) {
      const int cnt = min(RQ_CH, cend - c0);
      __syncthreads();
      for (int q = threadIdx.x; q < cnt * DP; q += RQ_TPB)
        sy[q] = P[(size_t)(seg[B] + c0) * DP + q];
      __syncthreads();
      if (act)
        for (int c = 0; c < cnt; ++c) {
          double d2 = 0.0;
#pragma unroll
          for (int k = 0; k < DP; ++k) {
            const double u = x[k] - sy[c * DP + k];
            d2 = fma(u, u, d2);
          }
          u128_add(acc, fx_of(sqrt(d2), s.dexp));  // exactly as the FP64 sweep
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) u128_add(acc, u128_shfl_xor(acc, o));
    if ((threadIdx.x & 31) == 0) {
      rlo[threadIdx.x >> 5] = acc.lo;
      rhi[threadIdx.x >> 5] = acc.hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      U128 v{0ull, 0ull};
      for (int w = 0; w < RQ_TPB / 32; ++w) u128_add(v, U128{rlo[w], rhi[w]});
      limbs_atomic(&s.drq_acc[LIMBS * (size_t)i], v);
      const long long rows = min(RQ_TPB, na - ta * RQ_TPB);
      atomicAdd(&s.ctr->dense_rq_pp, (unsigned long long)(rows * (cend - cbeg)));
    }
  }
}

// the re-scored sums replace both entries (exact: no flag)
__global__ void k_drq_fin(State s, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int qa = s.drq_a[i], qb = s.drq_b[i];
    const unsigned long long *w = s.drq_acc + LIMBS * (size_t)i;
    const double v = entry_mean(w, s.dsl, s.dsh, s.dinv[qa], s.dinv[qb]);  // qa < qb
    unsigned long long *c = s.dsum + LIMBS * tri(qa, qb, s.dk);  // qa < qb
#pragma unroll
    for (int l = 0; l < LIMBS; ++l) c[l] = w[l];
    s.dmat[(size_t)qa * s.dk + qb] = v;
    s.dmat[(size_t)qb * s.dk + qa] = v;
  }
}

// ---------------------------------------------------------------------------
// Lance-Williams update of the matrix after the round's merges: for average
// linkage the sum of A u B with C is the sum of A's and B's (exact), the mean
// follows from the new sizes
// ---------------------------------------------------------------------------
struct Limbs {
  unsigned long long w[LIMBS];
};

__device__ __forceinline__ Limbs sum_at(const State &s, int i, int j) {  // the pair {i, j}
  const unsigned long long *c = s.dsum + LIMBS * (i < j ? tri(i, j, s.dk) : tri(j, i, s.dk));
  Limbs r;
#pragma unroll
  for (int l = 0; l < LIMBS; ++l) r.w[l] = c[l];
  return r;
}

// limb-wise sum (the flags OR)
__device__ __forceinline__ Limbs sum_add(const Limbs &x, const Limbs &y) {
  Limbs r;
#pragma unroll
  for (int l = 0; l < LIMBS - 1; ++l) r.w[l] = x.w[l] + y.w[l];
  r.w[3] = ((x.w[3] & ~TOP) + (y.w[3] & ~TOP)) | ((x.w[3] | y.w[3]) & TOP);
  return r;
}

__device__ __forceinline__ void sum_put(const State &s, int i, int j, const Limbs &v) {
  unsigned long long *c = s.dsum + LIMBS * (i < j ? tri(i, j, s.dk) : tri(j, i, s.dk));
#pragma unroll
  for (int l = 0; l < LIMBS; ++l) c[l] = v.w[l];
}

// the round's positions after the merges: size of each cluster and whether
// it merged (the order is the one of the start of the round)
__global__ void k_dense_cols(State s, const int32_t *order_old, int Kold, int round, int npairs) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Kold; j += gridDim.x * blockDim.x)
    s.dqm[j] = s.mround[order_old[j]] == round ? 1 : 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
    const int lo = s.pair_lo[p];
    s.dinv[s.didx[lo]] = 1.0 / (double)s.csize[lo];  // the merged cluster's size
  }
}

// 1. rows: the survivor's sum with every cluster that did not merge this
//    round adds its partner's; means in the survivor's row
__global__ void k_dense_row(State s, int Kold, int npairs) {
  const int dk = s.dk;
  for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
    const int lo = s.pair_lo[p], hi = s.pair_hi[p];
    const int qa = s.didx[lo], qb = s.didx[hi];
    const double ia = s.dinv[qa];  // already the merged cluster's
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Kold; j += gridDim.x * blockDim.x) {
      if (s.dqm[j]) continue;  // pairs of two merged clusters: k_dense_fix
      const int q = s.dq[j];
      const Limbs v = sum_add(sum_at(s, qa, q), sum_at(s, qb, q));
      sum_put(s, qa, q, v);
      const double iq = s.dinv[q];
      s.dmat[(size_t)qa * dk + q] = qa < q ? entry_mean(v.w, s.dsl, s.dsh, ia, iq)
                                           : entry_mean(v.w, s.dsl, s.dsh, iq, ia);
    }
  }
}

// 2. pairs of clusters that both merged this round: the four old sums, once
//    per unordered pair (the lower index writes both means)
__global__ void k_dense_fix(State s, int npairs) {
  const long long tot = (long long)npairs * npairs;
  const int dk = s.dk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot;
       t += (long long)gridDim.x * blockDim.x) {
    const int p1 = (int)(t / npairs), p2 = (int)(t - (long long)p1 * npairs);
    if (p1 == p2) continue;
    const int a = s.pair_lo[p1], b = s.pair_hi[p1];
    const int c = s.pair_lo[p2], d = s.pair_hi[p2];
    const int qa = s.didx[a], qb = s.didx[b], qc = s.didx[c], qd = s.didx[d];
    if (qa > qc) continue;
    const Limbs v = sum_add(sum_add(sum_at(s, qa, qc), sum_at(s, qa, qd)),
                            sum_add(sum_at(s, qb, qc), sum_at(s, qb, qd)));
    sum_put(s, qa, qc, v);
    const double m = entry_mean(v.w, s.dsl, s.dsh, s.dinv[qa], s.dinv[qc]);  // qa < qc
    s.dmat[(size_t)qa * dk + qc] = m;
    s.dmat[(size_t)qc * dk + qa] = m;
  }
}

// 3. columns: every cluster that did not merge gets the survivor's mean in
//    its own row (the mean matrix stays exactly symmetric)
__global__ void k_dense_col(State s, int Kold, int npairs) {
  const int dk = s.dk;
  for (int p = blockIdx.y; p < npairs; p += gridDim.y) {
    const int qa = s.didx[s.pair_lo[p]];
    const double *ra = s.dmat + (size_t)qa * dk;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Kold; j += gridDim.x * blockDim.x) {
      if (s.dqm[j]) continue;
      const int r = s.dq[j];
      s.dmat[(size_t)r * dk + qa] = ra[r];
    }
  }
}

// matrix index of every active position (the search's column list)
__global__ void k_dense_q(State s, const int32_t *order, int K) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < K; p += gridDim.x * blockDim.x)
    s.dq[p] = s.didx[order[p]];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename F>
void launch_2d_tiles(F kernel, long long tiles, int threads_x, cudaStream_t st,
                     const SweepArgs &a) {
  const unsigned gx = (unsigned)std::min<long long>(tiles, 65535);
  const unsigned gy = (unsigned)((tiles + gx - 1) / gx);
  kernel<<<dim3(gx, gy), threads_x, 0, st>>>(a);
}

int sweep(hac_ctx *h, cudaStream_t st, const SweepArgs &a) {
  const State &s = h->s;
  const bool f32 = s.prec == HAC_PREC_F32_RECHECK;
  // rows per thread: 4 (2 for 16-wide FP32 rows and for FP64), for 2-3
  // resident tiles per SM
  const int ppt = f32 && s.dp <= 8 ? HAC_DS_PPT8 : 2;
  const long long TI = (long long)DS_TPB * ppt;
  SweepArgs b = a;
  b.nb = (a.N + TI - 1) / TI;
  const long long tiles = b.nb * (b.nb + 1) / 2;
  if (f32) {
    constexpr int P8 = HAC_DS_PPT8;
    switch (s.d) {  // specialised on the true dimension
      case 1: launch_2d_tiles(k_dense_sweep32<1, 2, P8>, tiles, DS_TPB, st, b); break;
      case 2: launch_2d_tiles(k_dense_sweep32<2, 2, P8>, tiles, DS_TPB, st, b); break;
      case 3: launch_2d_tiles(k_dense_sweep32<3, 4, P8>, tiles, DS_TPB, st, b); break;
      case 4: launch_2d_tiles(k_dense_sweep32<4, 4, P8>, tiles, DS_TPB, st, b); break;
      case 5: launch_2d_tiles(k_dense_sweep32<5, 8, P8>, tiles, DS_TPB, st, b); break;
      case 6: launch_2d_tiles(k_dense_sweep32<6, 8, P8>, tiles, DS_TPB, st, b); break;
      case 7: launch_2d_tiles(k_dense_sweep32<7, 8, P8>, tiles, DS_TPB, st, b); break;
      case 8: launch_2d_tiles(k_dense_sweep32<8, 8, P8>, tiles, DS_TPB, st, b); break;
      case 9: launch_2d_tiles(k_dense_sweep32<9, 16, 2>, tiles, DS_TPB, st, b); break;
      case 10: launch_2d_tiles(k_dense_sweep32<10, 16, 2>, tiles, DS_TPB, st, b); break;
      case 11: launch_2d_tiles(k_dense_sweep32<11, 16, 2>, tiles, DS_TPB, st, b); break;
      case 12: launch_2d_tiles(k_dense_sweep32<12, 16, 2>, tiles, DS_TPB, st, b); break;
      case 13: launch_2d_tiles(k_dense_sweep32<13, 16, 2>, tiles, DS_TPB, st, b); break;
      case 14: launch_2d_tiles(k_dense_sweep32<14, 16, 2>, tiles, DS_TPB, st, b); break;
      case 15: launch_2d_tiles(k_dense_sweep32<15, 16, 2>, tiles, DS_TPB, st, b); break;
      default: launch_2d_tiles(k_dense_sweep32<16, 16, 2>, tiles, DS_TPB, st, b);
    }
  } else {
    switch (s.dp) {
      case 2: launch_2d_tiles(k_dense_sweep64<2, 2>, tiles, DS_TPB, st, b); break;
      case 4: launch_2d_tiles(k_dense_sweep64<4, 2>, tiles, DS_TPB, st, b); break;
      case 8: launch_2d_tiles(k_dense_sweep64<8, 2>, tiles, DS_TPB, st, b); break;
      default: launch_2d_tiles(k_dense_sweep64<16, 2>, tiles, DS_TPB, st, b);
    }
  }
  CK(cudaGetLastError());
  return HAC_OK;
}

int64_t dense_threshold(const hac_ctx *h) {
  return h->dense_k >= 0 ? h->dense_k : h->dense_def;
}

// FP64 re-score of the first m listed pairs (they then hold exact values)
int recheck(hac_ctx *h, cudaStream_t st, int m) {
  State &s = h->s;
  if (m <= 0) return HAC_OK;
  CK(cudaMemsetAsync(s.drq_acc, 0, (size_t)m * LIMBS * sizeof(unsigned long long), st));
  k_drq_count<<<grid_for(m, TPB), TPB, 0, st>>>(s, m);
  k_drq_scan<<<1, 1024, 0, st>>>(s, m);
  const int g = device_sms() * 4;
  switch (s.dp) {
    case 2: k_drq_eval<2><<<g, RQ_TPB, 0, st>>>(s, m, h->pcur); break;
    case 4: k_drq_eval<4><<<g, RQ_TPB, 0, st>>>(s, m, h->pcur); break;
    case 8: k_drq_eval<8><<<g, RQ_TPB, 0, st>>>(s, m, h->pcur); break;
    default: k_drq_eval<16><<<g, RQ_TPB, 0, st>>>(s, m, h->pcur);
  }
  k_drq_fin<<<grid_for(m, TPB), TPB, 0, st>>>(s, m);
  h->launches += 4;
  CK(cudaGetLastError());
  return HAC_OK;
}

}  // namespace

// Default switch-over for a run: the tree search prunes well in low
// dimension and poorly above 8, so the matrix pays off later (smaller K) in
// 2-D and much earlier in 16-D.  Measured at 10^6 points (whole average run,
// ms at 8,192 / 16,384 / 32,768): 2-D uniform 171 / 186 / 241, 2-D Gaussian
// disc 174 / 185 / 250; 5-D mixture 438 / 432 / 472, 5-D uniform
// 368 (12,288) / 374 / 429, 5-D Gaussian disc 778 / 521 / 518; 16-D lattice
// 21.4 s / 11.5 s (32,768) / 9.0 s (49,152) / 8.3 s (65,536).  The two
// matrices (24 B per entry of the K x K matrix) take at most half of the
// device memory free at the start of the run.
int64_t dense_default(int d) {
  int64_t k = d <= 3 ? 8192 : d <= 8 ? 16384 : 65536;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
    k = std::min<int64_t>(k, (int64_t)std::sqrt(0.5 * (double)fr / 24.0));
  else
    cudaGetLastError();
  return k;
}

int dense_maybe_enter(hac_ctx *h, cudaStream_t st, int K, RoundCtl &ctl) {
  State &s = h->s;
  if (s.dense) return 1;
  if (s.linkage != LK_AVERAGE || s.max_inst != 1 || s.noprune || K < 2) return 0;
  if ((int64_t)K > dense_threshold(h)) return 0;
  // buffers, sized once per handle for the largest matrix it can need
  if (h->dense_cap < K) {
    const int64_t cap = std::min<int64_t>(dense_threshold(h), h->n);
    const int rqcap = (int)std::min<int64_t>(std::max<int64_t>(4 * cap, 1 << 16), 1 << 22);
    int rc = 0;
    if ((rc = dalloc(h, &s.didx, h->n)) || (rc = dalloc(h, &s.dcid, cap)) ||
        (rc = dalloc(h, &s.dq, cap)) || (rc = dalloc(h, &s.dinv, cap)) ||
        (rc = dalloc(h, &s.dqm, cap)) ||
        (rc = dalloc(h, &s.drq_a, rqcap)) || (rc = dalloc(h, &s.drq_b, rqcap)) ||
        (rc = dalloc(h, &s.drq_pre, rqcap + 1)) ||
        (rc = dalloc(h, &s.drq_acc, LIMBS * (size_t)rqcap)) || (rc = dalloc(h, &s.dpend[0], cap)) ||
        (rc = dalloc(h, &s.dpend[1], cap)))
      return rc;
    s.drq_cap = rqcap;
    // the matrices last: without room for them the instance stays on the
    // range-query search (same result)
    if (dalloc(h, &s.dmat, (size_t)cap * cap) != HAC_OK ||
        dalloc(h, &s.dsum, LIMBS * (size_t)cap * (cap - 1) / 2 + 1) != HAC_OK) {
      h->dense_k = 0;
      return 0;
    }
    h->dense_cap = cap;
  }
  s.dk = K;
  // unit of the fixed-point sums: (n/2)^2 x the largest point distance < 2^126 units
  const double dmax = 2.0 * (double)s.coord_scale * std::sqrt((double)s.d) * (1.0 + 1e-5);
  const double smax = 0.25 * (double)h->lay_n * (double)h->lay_n * dmax;
  s.dexp = smax > 0.0 ? (int)std::floor(std::log2(smax)) + 1 - 126 : -1000;
  s.dsl = std::ldexp(1.0, s.dexp);
  s.dsh = std::ldexp(1.0, 64 + s.dexp);
  k_dense_init<<<grid_for(K, TPB), TPB, 0, st>>>(s, s.order[h->ocur], K);
  CK(cudaMemsetAsync(s.dsum, 0, (size_t)K * (K - 1) / 2 * LIMBS * sizeof(unsigned long long),
                     st));
  SweepArgs a{};
  a.p32 = s.p32[h->pcur];
  a.p64 = s.p64[h->pcur];
  a.plab = s.plab[h->pcur];
  a.didx = s.didx;
  a.N = h->lay_n;
  a.dk = K;
  a.e = s.dexp;
  // the FP32 copy scaled by 2^k toward |coordinate| <= 2^40 (squared
  // distances stay below 2^86 for d <= 16; k >= 0 keeps the scaling exact)
  {
    int k = 0;
    if (s.p32_max > 0.0)
      k = std::max(0, std::min(100, 40 - (int)std::ceil(std::log2(s.p32_max))));
    s.dsk = k;
    a.scl = std::ldexp(1.0f, k);
    a.es = s.dexp + k;
  }
  a.sum = s.dsum;
  a.ctr = s.ctr;
  if (ctl.eb0) cudaEventRecord(ctl.eb0, st);
  int rc = sweep(h, st, a);
  if (rc) return rc;
  if (ctl.eb1) cudaEventRecord(ctl.eb1, st);
  const long long nt = (K + 31) / 32, tiles = nt * (nt + 1) / 2;
  const unsigned gx = (unsigned)std::min<long long>(tiles, 65535);
  const unsigned gy = (unsigned)((tiles + gx - 1) / gx);
  k_dense_fin<<<dim3(gx, gy), dim3(32, 8), 0, st>>>(s, K, s.prec == HAC_PREC_F32_RECHECK);
  CK(cudaGetLastError());
  if (ctl.eb0) {
    CK(cudaEventSynchronize(ctl.eb1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctl.eb0, ctl.eb1);
    ctl.ms_dense += ms;
  }
  h->launches += 3;
  ctl.dense_launches += 3;
  s.dense = 1;
  return 1;
}

int dense_search(hac_ctx *h, cudaStream_t st, int K, int nterm, RoundCtl &ctl) {
  State &s = h->s;
  NNArgs a{};
  a.dmat = s.dmat;
  a.dk = s.dk;
  a.K = K;
  a.order = s.order[h->ocur];
  a.didx = s.didx;
  a.dq = s.dq;
  a.list = s.term;
  k_dense_q<<<grid_for(K, TPB), TPB, 0, st>>>(s, a.order, K);
  h->launches += 1;
  a.nlist = nterm;
  a.delta = (double)s.delta_pts;
  a.rho = ((double)s.d + 48.0) * 5.9604644775390625e-8;
  a.Ekey = s.Ekey;
  a.Ecid = s.Ecid;
  a.drq_a = s.drq_a;
  a.drq_b = s.drq_b;
  a.drq_cap = s.drq_cap;
  a.ctr = s.ctr;
  // absolute term: a truncation below one unit 2^dexp on each side (the FP32
  // partial sums and the FP64 re-score's distances) and the flush of scaled
  // squared distances below 2^-126 (distances below 2^(-63-dsk))
  a.eta = (2.0 * std::ldexp(1.0, s.dexp) + std::ldexp(1.0, -63 - s.dsk)) * (1.0 + 1e-9);
  const bool f32 = s.prec == HAC_PREC_F32_RECHECK;
  // integer bounds when the estimates carry no relative-to-scale absolute
  // term and the lone estimate's bound is within the 4e-6 the height
  // convention allows; above m0 = 2^30 eta the absolute term is within
  // 2^-30 of an entry and joins rho
  const double rho_i = a.rho + std::ldexp(1.0, -30);
  const bool intb = f32 && a.delta == 0.0 && rho_i <= 4e-6;
  a.nu = (unsigned long long)std::ceil(std::ldexp(rho_i / (1.0 - rho_i), 53) * (1.0 + 1e-6)) + 2;
  a.nl = 2 * ((unsigned long long)std::ceil(std::ldexp(rho_i, 53) * (1.0 + 1e-6)) + 2);
  {
    const double m0 = std::ldexp(a.eta, 30);
    memcpy(&a.m0, &m0, 8);
    const double m0up = 2.0 * m0;
    memcpy(&a.m0up, &m0up, 8);
  }
  for (int it = 0;; ++it) {
    if (it >= 64) return HAC_EINTERNAL;
    CK(cudaMemsetAsync(&s.ctr->npend, 0, sizeof(int32_t), st));
    CK(cudaMemsetAsync(&s.ctr->nrq, 0, sizeof(int32_t), st));
    a.pend_out = s.dpend[it & 1];
    const int blocks = std::max(1, std::min(cdiv(a.nlist, 8), device_sms() * 16));
    if (intb)
      k_dense_nn<2><<<blocks, 256, 0, st>>>(a);
    else if (f32)
      k_dense_nn<1><<<blocks, 256, 0, st>>>(a);
    else
      k_dense_nn<0><<<blocks, 256, 0, st>>>(a);
    CK(cudaGetLastError());
    h->launches += 1;
    ctl.searches += a.nlist;
    if (!f32) break;
    int cnt[2];  // npend, nrq are not adjacent: two reads
    CK(cudaMemcpyAsync(&cnt[0], &s.ctr->npend, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&cnt[1], &s.ctr->nrq, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (cnt[0] == 0) break;
    const int m = std::min(cnt[1], s.drq_cap);
    ctl.dense_launches += 4;
    int rc = recheck(h, st, m);
    if (rc) return rc;
    ctl.dense_rechecks += m;
    a.list = s.dpend[it & 1];
    a.nlist = cnt[0];
  }
  return HAC_OK;
}

int dense_update(hac_ctx *h, cudaStream_t st, int round, int K, int npairs) {
  State &s = h->s;
  if (npairs <= 0) return HAC_OK;
  // s.dq holds this round's positions (the order before the compaction)
  k_dense_cols<<<grid_for(K, TPB), TPB, 0, st>>>(s, s.order[h->ocur], K, round, npairs);
  const int gx = std::max(1, std::min(cdiv(K, TPB), 64));
  const int gy = std::min(npairs, 65535);
  k_dense_row<<<dim3(gx, gy), TPB, 0, st>>>(s, K, npairs);
  if (npairs > 1) {
    const long long tot = (long long)npairs * npairs;
    k_dense_fix<<<grid_for(tot, TPB), TPB, 0, st>>>(s, npairs);
    h->launches += 1;
  }
  k_dense_col<<<dim3(gx, gy), TPB, 0, st>>>(s, K, npairs);
  h->launches += 3;
  CK(cudaGetLastError());
  return HAC_OK;
}

}  // namespace hacg
