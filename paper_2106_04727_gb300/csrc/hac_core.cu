// GB300 nearest-neighbor-chain HAC: initial layout, the per-round kernels of
// ParChain Algorithm 1 around the nearest-neighbour search, and the C ABI.
//
// Round r (Algorithm 1):
//   find_nearest_neighbors      k_query (hac_query.cu), one warp per terminal
//   succ / WriteMin(pred)       k_chain: packed (f32 key, cid) 64-bit atomicMin
//   R-NN parallel filter        k_rnn: terminal i with succ(succ(i)) == i
//   merge                       k_merge: size, FP64 coordinate sums, box union
//   D.update / active / terms   k_cmp_*: chain repair, stable compaction of the
//                               active order, new terminal list, new segment
//                               offsets; k_relayout moves points so every
//                               cluster stays one contiguous segment;
//                               k_tree_*: rebuild the range-query tree
#include "hac.h"
#include "hac_internal.cuh"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <type_traits>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using namespace hacg;

namespace {

constexpr int TPB = 256;

enum { LK_COMPLETE = 0, LK_AVERAGE = 1, LK_WARD = 2, LK_AVG2 = 3 };

__host__ __device__ inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// block-wide helpers (256 threads)
// ---------------------------------------------------------------------------

// exclusive scan of one int per thread; returns the block total in *total
__device__ int block_excl_scan(int v, int *total) {
  __shared__ int ws[TPB / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < TPB / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < TPB / 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < TPB / 32) ws[lane] = t;
  }
  __syncthreads();
  const int pre = w ? ws[w - 1] : 0;
  *total = ws[TPB / 32 - 1];
  __syncthreads();
  return pre + x - v;
}

__device__ int block_sum(int v) {
  int t;
  block_excl_scan(v, &t);
  return t;
}

// ---------------------------------------------------------------------------
// generic exclusive scan of an int array (3 phases)
// ---------------------------------------------------------------------------
constexpr int SC_ITEMS = 8, SC_TILE = TPB * SC_ITEMS;

__global__ void k_scan_reduce(const int32_t *in, int m, int32_t *bs) {
  int s = 0;
  const int base = blockIdx.x * SC_TILE;
  for (int i = threadIdx.x; i < SC_TILE; i += TPB)
    if (base + i < m) s += in[base + i];
  s = block_sum(s);
  if (threadIdx.x == 0) bs[blockIdx.x] = s;
}

// one block: exclusive scan of `nb` values in place; total to *tot
__global__ void k_scan_top(int32_t *bs, int nb, int32_t *tot) {
  const int per = cdiv(nb, TPB);
  const int b0 = threadIdx.x * per;
  int s = 0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < nb) s += bs[b0 + i];
  int t;
  int pre = block_excl_scan(s, &t);
  for (int i = 0; i < per; ++i)
    if (b0 + i < nb) {
      int v = bs[b0 + i];
      bs[b0 + i] = pre;
      pre += v;
    }
  if (threadIdx.x == 0 && tot) *tot = t;
}

__global__ void k_scan_down(const int32_t *in, int32_t *out, int m, const int32_t *bs) {
  const int base = blockIdx.x * SC_TILE + threadIdx.x * SC_ITEMS;
  int v[SC_ITEMS];
  int s = 0;
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    v[i] = base + i < m ? in[base + i] : 0;
    s += v[i];
  }
  int t;
  int pre = block_excl_scan(s, &t) + bs[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SC_ITEMS; ++i) {
    if (base + i < m) out[base + i] = pre;
    pre += v[i];
  }
}

// ---------------------------------------------------------------------------
// LSD radix sort of (u64 key, i32 value), 8-bit digits, stable
// ---------------------------------------------------------------------------
constexpr int RS_ITEMS = 8, RS_TILE = TPB * RS_ITEMS;

__global__ void k_rs_hist(const uint64_t *keys, int n, int shift, int32_t *hist, int ntiles) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int base = blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += TPB)
    if (base + i < n) atomicAdd(&h[(keys[base + i] >> shift) & 255], 1);
  __syncthreads();
  hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t *kin, const int32_t *vin, uint64_t *kout,
                             int32_t *vout, int n, int shift, const int32_t *hscan, int ntiles) {
  __shared__ int run[256];
  __shared__ int wcnt[TPB / 32][257];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  run[tid] = hscan[tid * ntiles + blockIdx.x];
  const int base = blockIdx.x * RS_TILE;
  for (int c = 0; c < RS_ITEMS; ++c) {
    for (int i = tid; i < (TPB / 32) * 257; i += TPB) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int p = base + c * TPB + tid;
    const bool v = p < n;
    const uint64_t k = v ? kin[p] : 0;
    const int val = v ? vin[p] : 0;
    const int dig = v ? (int)((k >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) wcnt[w][dig] = __popc(peers);
    __syncthreads();
    if (v) {
      int off = run[dig];
      for (int ww = 0; ww < w; ++ww) off += wcnt[ww][dig];
      kout[off + rank] = k;
      vout[off + rank] = val;
    }
    __syncthreads();
    int s = 0;
    for (int ww = 0; ww < TPB / 32; ++ww) s += wcnt[ww][tid];
    run[tid] += s;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// init: bounding box, Morton keys, layout
// ---------------------------------------------------------------------------

// order-preserving map of doubles to u64 (for atomicMin/Max)
__device__ __forceinline__ unsigned long long ord_enc(double x) {
  unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <typename T>
__global__ void k_bbox(const T *X, int64_t n, int d, unsigned long long *mn,
                       unsigned long long *mx, Counters *ctr) {
  double lo[MAXD], hi[MAXD];
  for (int k = 0; k < d; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < d; ++k) {
      double x = (double)X[i * d + k];
      if (!isfinite(x)) bad = true;
      lo[k] = fmin(lo[k], x);
      hi[k] = fmax(hi[k], x);
    }
  if (bad) atomicOr(&ctr->err, ERR_NONFINITE);
  for (int k = 0; k < d; ++k) {
    double a = lo[k], b = hi[k];
    for (int o = 16; o; o >>= 1) {
      a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(mn + k, ord_enc(a));
      atomicMax(mx + k, ord_enc(b));
    }
  }
}

struct MortonParams {
  double lo[MAXD], inv[MAXD];
  int bits;
};

template <typename T>
__global__ void k_morton(const T *X, int64_t n, int d, MortonParams mp, uint64_t *keys,
                         int32_t *vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t q[MAXD];
    const double top = (double)((1u << mp.bits) - 1u);
    for (int k = 0; k < d; ++k) {
      double t = ((double)X[i * d + k] - mp.lo[k]) * mp.inv[k];
      t = fmin(fmax(t, 0.0), 1.0) * top;
      q[k] = (uint32_t)t;
    }
    uint64_t code = 0;
    for (int b = mp.bits - 1; b >= 0; --b)
      for (int k = 0; k < d; ++k) code = (code << 1) | ((q[k] >> b) & 1u);
    keys[i] = code;
    vals[i] = (int32_t)i;
  }
}

template <typename T>
__global__ void k_layout(State s, const T *X, const int32_t *perm, MortonParams ctr_) {
  // ctr_.lo holds the recentring offset
  const int64_t n = s.n;
  const int d = s.d, dp = s.dp;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int i = perm[p];
    for (int k = 0; k < dp; ++k) {
      double x = k < d ? (double)X[(int64_t)i * d + k] - ctr_.lo[k] : 0.0;
      s.p64[0][p * dp + k] = x;
      // FP32 input stays unrounded (exact) in the FP32 copy; differences of
      // FP32 numbers then carry only relative rounding error
      s.p32[0][p * dp + k] = s.pts32_exact ? (k < d ? (float)X[(int64_t)i * d + k] : 0.f) : (float)x;
      s.csum[(int64_t)i * dp + k] = x;
      s.cent[(int64_t)i * dp + k] = x;
      s.cent32[(int64_t)i * dp + k] = (float)x;
      s.blo[(int64_t)i * dp + k] = __double2float_rd(x);
      s.bhi[(int64_t)i * dp + k] = __double2float_ru(x);
      s.q32[p * dp + k] = (float)x;
      s.q64[p * dp + k] = x;
      s.qblo[p * dp + k] = __double2float_rd(x);
      s.qbhi[p * dp + k] = __double2float_ru(x);
    }
    double sq = 0.0;
    for (int k = 0; k < d; ++k) {
      const double x = (double)X[(int64_t)i * d + k] - ctr_.lo[k];
      sq += x * x;
    }
    s.csq[i] = sq;
    s.sse[i] = 0.0;
    s.qvar[p] = 0.f;
    s.qsz[p] = 1;
    s.qseg[p] = (int32_t)p;
    s.plab[0][p] = i;
    s.seg[0][i] = (int32_t)p;
    s.csize[i] = 1;
    s.succ[i] = -1;
    s.pred[i] = PRED_EMPTY;
    s.mround[i] = -1;
    s.isterm[i] = 0;
    s.alive[i] = 1;
    s.rootof[i] = i;
    s.reloff[i] = 0;
    s.gen[i] = 0;
    s.inst[i] = 0;
    s.qinst[p] = 0;
    s.order[0][p] = i;
    s.pos[i] = (int32_t)p;
    s.term[p] = i;
  }
}

// one instance's parameters and progress counters
__global__ void k_inst_set(State s, int slot, float slack, float scale, float dpts, int rec,
                           int act, int seq) {
  s.iseq[slot] = seq;
  s.islack[slot] = slack;
  s.iscale[slot] = scale;
  s.idpts[slot] = dpts;
  s.irec[slot] = rec;
  s.irecn[slot] = 0;
  s.iact[slot] = act;
  s.idone[slot] = act <= 1;
}

// ---------------------------------------------------------------------------
// range-query tree
// ---------------------------------------------------------------------------
template <int DP>
__global__ void k_tree_leaf(State s, const int32_t *order, int K) {
  const int lane = threadIdx.x & 31;
  const int cnt = level_count(K, 0);
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt;
       j += (gridDim.x * blockDim.x) >> 5) {
    const int idx = j * FAN + lane;
    const bool v = idx < K;
    const size_t c = v ? (size_t)idx : 0;  // position-ordered records
    int nm = v ? s.qsz[c] : INT_MAX;
    int il = v ? s.qinst[c] : INT_MAX, ih = v ? s.qinst[c] : INT_MIN;
    for (int o = 16; o; o >>= 1) {
      nm = min(nm, __shfl_xor_sync(0xffffffffu, nm, o));
      il = min(il, __shfl_xor_sync(0xffffffffu, il, o));
      ih = max(ih, __shfl_xor_sync(0xffffffffu, ih, o));
    }
    const int node = s.lvl_base[0] + j;
    if (lane == 0) {
      s.ninlo[node] = il;
      s.ninhi[node] = ih;
    }
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      float lo = v ? s.q32[c * DP + k] : INFINITY;
      float hi = v ? s.q32[c * DP + k] : -INFINITY;
      float hm = v ? s.qbhi[c * DP + k] : INFINITY;
      float lm = v ? s.qblo[c * DP + k] : -INFINITY;
      for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        hm = fminf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
        lm = fmaxf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
      }
      if (lane == k) {
        s.nclo[(size_t)node * DP + k] = lo;
        s.nchi[(size_t)node * DP + k] = hi;
        s.nhmin[(size_t)node * DP + k] = hm;
        s.nlmax[(size_t)node * DP + k] = lm;
      }
    }
    if (lane == 0) s.nnmin[node] = nm;
  }
}

template <int DP>
__global__ void k_tree_up(State s, int K, int L) {
  const int lane = threadIdx.x & 31;
  const int cnt = level_count(K, L), ccnt = level_count(K, L - 1);
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt;
       j += (gridDim.x * blockDim.x) >> 5) {
    const int ch = j * FAN + lane;
    const bool v = ch < ccnt;
    const int cn = s.lvl_base[L - 1] + (v ? ch : 0);
    int nm = v ? s.nnmin[cn] : INT_MAX;
    int il = v ? s.ninlo[cn] : INT_MAX, ih = v ? s.ninhi[cn] : INT_MIN;
    for (int o = 16; o; o >>= 1) {
      nm = min(nm, __shfl_xor_sync(0xffffffffu, nm, o));
      il = min(il, __shfl_xor_sync(0xffffffffu, il, o));
      ih = max(ih, __shfl_xor_sync(0xffffffffu, ih, o));
    }
    const int node = s.lvl_base[L] + j;
    if (lane == 0) {
      s.ninlo[node] = il;
      s.ninhi[node] = ih;
    }
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      float lo = v ? s.nclo[(size_t)cn * DP + k] : INFINITY;
      float hi = v ? s.nchi[(size_t)cn * DP + k] : -INFINITY;
      float hm = v ? s.nhmin[(size_t)cn * DP + k] : INFINITY;
      float lm = v ? s.nlmax[(size_t)cn * DP + k] : -INFINITY;
      for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        hm = fminf(hm, __shfl_xor_sync(0xffffffffu, hm, o));
        lm = fmaxf(lm, __shfl_xor_sync(0xffffffffu, lm, o));
      }
      if (lane == k) {
        s.nclo[(size_t)node * DP + k] = lo;
        s.nchi[(size_t)node * DP + k] = hi;
        s.nhmin[(size_t)node * DP + k] = hm;
        s.nlmax[(size_t)node * DP + k] = lm;
      }
    }
    if (lane == 0) s.nnmin[node] = nm;
  }
}

// ---------------------------------------------------------------------------
// per-round kernels
// ---------------------------------------------------------------------------

// succ(i) = nearest neighbour; WriteMin(pred(succ), (key, i)) (Algorithm 1)
__global__ void k_chain(State s, int nterm) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nterm; t += gridDim.x * blockDim.x) {
    const int i = s.term[t];
    const int j = s.Ecid[i];
    if (j < 0) continue;
    s.succ[i] = j;
    const float kf = __double2float_ru(s.Ekey[i]);
    const unsigned long long v =
        ((unsigned long long)__float_as_uint(kf) << 32) | (unsigned long long)(unsigned)i;
    atomicMin(&s.pred[j], v);
  }
}

// parallel filter for reciprocal nearest neighbours: each pair once
__global__ void k_rnn(State s, int nterm, int round) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nterm; t += gridDim.x * blockDim.x) {
    const int i = s.term[t];
    const int j = s.succ[i];
    if (j < 0) continue;
    if (s.succ[j] == i && (i < j || s.isterm[j] != round)) {
      const int p = atomicAdd(&s.ctr->npairs, 1);
      s.pair_lo[p] = min(i, j);
      s.pair_hi[p] = max(i, j);
      s.pair_key[p] = s.Ekey[i];
    }
  }
}

// merge every reciprocal pair: the cluster keeps the smaller cid
__global__ void k_merge(State s, int round, int npairs) {
  const int dp = s.dp;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
    const int lo = s.pair_lo[p], hi = s.pair_hi[p];
    const double key = s.pair_key[p];
    const int na = s.csize[lo], nb = s.csize[hi];
    const int ins = s.inst[lo];
    atomicAdd(&s.ctr->nmerges, 1);
    const int m = s.irec[ins] + atomicAdd(&s.irecn[ins], 1);
    if (atomicSub(&s.iact[ins], 1) == 2) {  // one cluster left
      s.idone[ins] = 1;
      s.done_list[atomicAdd(&s.ctr->ndone, 1)] = ins;
    }
    s.m_a[m] = lo;
    s.m_b[m] = hi;
    s.m_h[m] = s.linkage == LK_WARD ? sqrt(key) : key;
    s.m_size[m] = na + nb;
    s.m_round[m] = round;
    const double inv = 1.0 / (double)(na + nb);
    // variance update (Section 2): SSE(A u B) = SSE(A) + SSE(B)
    // + |A||B|/(|A|+|B|) ||c_A - c_B||^2, from the centroids before the merge
    double g2 = 0.0;
    for (int k = 0; k < dp; ++k) {
      const double t = s.cent[(size_t)lo * dp + k] - s.cent[(size_t)hi * dp + k];
      g2 += t * t;
    }
    s.sse[lo] = s.sse[lo] + s.sse[hi] + (double)na * (double)nb * inv * g2;
    for (int k = 0; k < dp; ++k) {
      const double sum = s.csum[(size_t)lo * dp + k] + s.csum[(size_t)hi * dp + k];
      s.csum[(size_t)lo * dp + k] = sum;
      const double c = sum * inv;
      s.cent[(size_t)lo * dp + k] = c;
      s.cent32[(size_t)lo * dp + k] = (float)c;
      s.blo[(size_t)lo * dp + k] = fminf(s.blo[(size_t)lo * dp + k], s.blo[(size_t)hi * dp + k]);
      s.bhi[(size_t)lo * dp + k] = fmaxf(s.bhi[(size_t)lo * dp + k], s.bhi[(size_t)hi * dp + k]);
    }
    s.csq[lo] += s.csq[hi];
    s.csize[lo] = na + nb;
    s.succ[lo] = -1;
    s.pred[lo] = PRED_EMPTY;
    s.mround[lo] = round;
    s.mround[hi] = round;
    s.alive[hi] = 0;
    s.rootof[hi] = lo;
    s.reloff[hi] = na;
    s.osize[lo] = na;
    s.osize[hi] = nb;
    s.partner[lo] = hi;
    s.partner[hi] = lo;
  }
}

// ---------------------------------------------------------------------------
// pair-distance cache (Section 5)
// ---------------------------------------------------------------------------

constexpr unsigned long long CKEY_BUSY = ~1ull;  // a slot whose value is being written

__device__ __forceinline__ unsigned long long slot_key(const State &s, size_t idx) {
  return *(volatile unsigned long long *)&s.ckey[idx];
}

// an empty slot, or one whose neighbour has merged since (stale generation)
__device__ __forceinline__ bool slot_free(const State &s, unsigned long long cur) {
  if (cur == CKEY_EMPTY) return true;
  if (cur == CKEY_BUSY) return false;
  return (unsigned)cur != (unsigned)s.gen[(int)(cur >> 32)];
}

// Claim slot idx (holding `cur`) by CAS to BUSY, write the value, then
// publish the key: concurrent writers skip BUSY slots, so a slot's key and
// value always come from the same writer.  Readers run in later kernels.
__device__ bool slot_put(const State &s, size_t idx, unsigned long long cur,
                         unsigned long long want, double v, float e, int part = 0) {
  if (atomicCAS(&s.ckey[idx], cur, CKEY_BUSY) != cur) return false;
  s.cval[idx] = v;
  s.cerr[idx] = e;
  s.cpart[idx] = part;
  __threadfence();
  atomicExch(&s.ckey[idx], want);
  return true;
}

// Insert (nbr -> v, e) into the table of `owner` if there is a free slot;
// an entry already present is kept (a partial one is completed by it).
__device__ void cache_insert(const State &s, int owner, int nbr, int nbr_gen, double v, float e) {
  const int S = s.cache_slots;
  const unsigned long long want = ckey_of(nbr, nbr_gen);
  const size_t base = (size_t)owner * S;
  int t = (int)(((unsigned)nbr * 2654435761u) % (unsigned)S);
  for (int q = 0; q < S; ++q, t = t + 1 == S ? 0 : t + 1) {
    // a free slot only turns BUSY or live within a kernel, so this ends
    for (;;) {
      const unsigned long long cur = slot_key(s, base + t);
      if (cur == want) {
        if (s.cpart[base + t] != 0) slot_put(s, base + t, cur, want, v, e);
        return;
      }
      if (!slot_free(s, cur)) break;
      if (slot_put(s, base + t, cur, want, v, e)) return;
    }
  }
}

// pairs evaluated by the search, into both clusters' tables
__global__ void k_cache_insert(State s) {
  const int m = min(s.ctr->nins, s.ins_cap);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m; q += gridDim.x * blockDim.x) {
    const int i = s.ins_i[q], j = s.ins_j[q];
    cache_insert(s, i, j, s.gen[j], s.ins_v[q], s.ins_e[q]);
    cache_insert(s, j, i, s.gen[i], s.ins_v[q], s.ins_e[q]);
  }
}

struct CEntry {
  int cid;
  float err;
  double val;
};

constexpr int CM_WARPS = 2;  // warps per block of k_cache_merge (5 * slots entries each)

// look for neighbour `g` in a warp-local list
__device__ __forceinline__ int clist_find(const CEntry *L, int n, int g) {
  for (int t = 0; t < n; ++t)
    if (L[t].cid == g) return t;
  return -1;
}

// look for the entry of `nbr` (at its current generation) in a global table
__device__ bool ctable_find(const State &s, int owner, int nbr, double &v, float &e) {
  const int S = s.cache_slots;
  const unsigned long long want = ckey_of(nbr, s.gen[nbr]);
  for (int t = 0; t < S; ++t)
    if (s.ckey[(size_t)owner * S + t] == want && s.cpart[(size_t)owner * S + t] == 0) {
      v = s.cval[(size_t)owner * S + t];
      e = s.cerr[(size_t)owner * S + t];
      return true;
    }
  return false;
}

// Cache update after the merges of a round (Algorithm 5), one warp per merged
// pair (lo, hi) -> k (cid lo).  From the tables of lo and hi, every neighbour g
// whose distances to both lo and hi are known gets D(k, g) by Lance-Williams
// (Table 2): complete = max, average = size-weighted mean; if g itself merged
// this round with g2 (case 1), D(k, g u g2) combines the four distances
// lo/hi x g/g2.  The new entries replace lo's table and are also inserted into
// g's table (case 2).  Error bounds combine the same way (max / weighted mean).
// Generations are bumped only afterwards (k_gen_bump), so every lookup here
// sees the pre-merge generations.
template <int LK>
__global__ void k_cache_merge(State s, int npairs, int round) {
  extern __shared__ unsigned char smem_raw[];
  const int S = s.cache_slots;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  CEntry *A = (CEntry *)smem_raw + (size_t)wib * 5 * S;
  CEntry *B = A + S;
  CEntry *N = B + S;  // up to 2S new entries (cid, err, val); gen kept in a parallel array
  CEntry *Q = N + 2 * S;  // up to S partial entries (one side known), part kept apart
  __shared__ int cnt[CM_WARPS][4];
  __shared__ int ngen_s[CM_WARPS][2 * CACHE_MAX_SLOTS];
  __shared__ int qgen_s[CM_WARPS][CACHE_MAX_SLOTS];
  __shared__ int qpart_s[CM_WARPS][CACHE_MAX_SLOTS];
  int *ngen = ngen_s[wib];
  int *qgen = qgen_s[wib];
  int *qpart = qpart_s[wib];
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npairs; p += warps) {
    const int lo = s.pair_lo[p], hi = s.pair_hi[p];
    const double na = (double)s.osize[lo], nb = (double)s.osize[hi];
    if (lane == 0) cnt[wib][0] = cnt[wib][1] = cnt[wib][2] = cnt[wib][3] = 0;
    __syncwarp();
    // valid entries of the two old tables
    for (int side = 0; side < 2; ++side) {
      const int owner = side ? hi : lo;
      CEntry *L = side ? B : A;
      for (int base = 0; base < S; base += 32) {
        const int t = base + lane;
        bool v = false;
        unsigned long long key = CKEY_EMPTY;
        if (t < S) {
          key = s.ckey[(size_t)owner * S + t];
          v = key != CKEY_EMPTY && (unsigned)key == (unsigned)s.gen[(int)(key >> 32)] &&
              s.cpart[(size_t)owner * S + t] == 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, v);
        if (v) {
          const int at = cnt[wib][side] + __popc(m & ((1u << lane) - 1u));
          L[at].cid = (int)(key >> 32);
          L[at].val = s.cval[(size_t)owner * S + t];
          L[at].err = s.cerr[(size_t)owner * S + t];
        }
        __syncwarp();
        if (lane == 0) cnt[wib][side] += __popc(m);
        __syncwarp();
      }
    }
    const int nA = cnt[wib][0], nB = cnt[wib][1];
    const double wa = na / (na + nb), wb = nb / (na + nb);
    // neighbours known from lo's table
    for (int t = lane; t < nA; t += 32) {
      const int g = A[t].cid;
      if (g == hi) continue;
      double v = -1.0;
      float e = 0.f;
      int gg = 0;
      if (s.mround[g] == round) {
        if (!s.alive[g]) continue;  // the retired side: its survivor handles the pair
        const int g2 = s.partner[g];
        const int a2 = clist_find(A, nA, g2), b1 = clist_find(B, nB, g), b2 = clist_find(B, nB, g2);
        if (a2 < 0 || b1 < 0 || b2 < 0) continue;
        const double ng = (double)s.osize[g], ng2 = (double)s.osize[g2];
        if (LK == 0) {
          v = fmax(fmax(A[t].val, A[a2].val), fmax(B[b1].val, B[b2].val));
          e = fmaxf(fmaxf(A[t].err, A[a2].err), fmaxf(B[b1].err, B[b2].err));
        } else {
          const double w = 1.0 / ((na + nb) * (ng + ng2));
          v = (na * ng * A[t].val + na * ng2 * A[a2].val + nb * ng * B[b1].val +
               nb * ng2 * B[b2].val) * w;
          e = (float)((na * ng * A[t].err + na * ng2 * A[a2].err + nb * ng * B[b1].err +
                       nb * ng2 * B[b2].err) * w);
        }
        gg = s.gen[g] + 1;
      } else {
        double vh;
        float eh;
        const int b1 = clist_find(B, nB, g);
        if (b1 >= 0) {
          vh = B[b1].val;
          eh = B[b1].err;
        } else if (!ctable_find(s, g, hi, vh, eh)) {
          // only D(lo, g) is known: keep it as a partial entry of the merged
          // cluster (its first |lo| points), completed later by evaluating
          // the other points only
          const int at = atomicAdd(&cnt[wib][3], 1);
          if (at < S) {
            Q[at].cid = g;
            Q[at].val = A[t].val;
            Q[at].err = A[t].err;
            qgen[at] = s.gen[g];
            qpart[at] = (int)na;
          }
          continue;
        }
        if (LK == 0) {
          v = fmax(A[t].val, vh);
          e = fmaxf(A[t].err, eh);
        } else {
          v = wa * A[t].val + wb * vh;
          e = (float)(wa * A[t].err + wb * eh);
        }
        gg = s.gen[g];
        cache_insert(s, g, lo, s.gen[lo] + 1, v, e);
      }
      const int at = atomicAdd(&cnt[wib][2], 1);
      N[at].cid = g;
      N[at].val = v;
      N[at].err = e;
      ngen[at] = gg;
    }
    __syncwarp();
    // neighbours known only from hi's table (case 2 needs D(lo, g) from g's table)
    for (int t = lane; t < nB; t += 32) {
      const int g = B[t].cid;
      if (g == lo || s.mround[g] == round || clist_find(A, nA, g) >= 0) continue;
      double vl;
      float el;
      if (!ctable_find(s, g, lo, vl, el)) {
        // only D(hi, g) is known: a partial entry for the last |hi| points
        const int at = atomicAdd(&cnt[wib][3], 1);
        if (at < S) {
          Q[at].cid = g;
          Q[at].val = B[t].val;
          Q[at].err = B[t].err;
          qgen[at] = s.gen[g];
          qpart[at] = -(int)nb;
        }
        continue;
      }
      double v;
      float e;
      if (LK == 0) {
        v = fmax(vl, B[t].val);
        e = fmaxf(el, B[t].err);
      } else {
        v = wa * vl + wb * B[t].val;
        e = (float)(wa * el + wb * B[t].err);
      }
      cache_insert(s, g, lo, s.gen[lo] + 1, v, e);
      const int at = atomicAdd(&cnt[wib][2], 1);
      N[at].cid = g;
      N[at].val = v;
      N[at].err = e;
      ngen[at] = s.gen[g];
    }
    __syncwarp();
    // the merged cluster's new table, replacing lo's: derived entries first,
    // then partial ones while there is room
    const int nN = min(cnt[wib][2], S);
    const int nQ = min(cnt[wib][3], S - nN);
    for (int t = lane; t < S; t += 32) {
      const size_t slot = (size_t)lo * S + t;
      if (t < nN) {
        s.ckey[slot] = ckey_of(N[t].cid, ngen[t]);
        s.cval[slot] = N[t].val;
        s.cerr[slot] = N[t].err;
        s.cpart[slot] = 0;
      } else if (t < nN + nQ) {
        const int u = t - nN;
        s.ckey[slot] = ckey_of(Q[u].cid, qgen[u]);
        s.cval[slot] = Q[u].val;
        s.cerr[slot] = Q[u].err;
        s.cpart[slot] = qpart[u];
      } else {
        s.ckey[slot] = CKEY_EMPTY;
      }
    }
    if (lane == 0) atomicAdd((unsigned long long *)&s.ctr->cache_lw, (unsigned long long)nN);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// big pairs: evaluated by the whole GPU, then cached for the re-run search
// ---------------------------------------------------------------------------
constexpr int BIG_TPB = 256;       // threads per tile
constexpr int BIG_TILE = BIG_TPB * 2;  // narrowest tile along the larger cluster
constexpr int BIG_MAXT = 32768; // tiles per request at most (chunks widen to fit)
constexpr int BIG_BATCH = 512;     // requests per batch (one scan block)

// Three kinds of request, each its own tile list and kernel:
//   0  FP32, larger cluster >= 256 x 8 points: 8 of its points per thread
//      (4 for d > 8)
//   1  FP32, smaller requests: 2 points per thread
//   2  FP64 (exact values wanted): 2 points per thread
// A tile is (points of the larger cluster) x (a chunk of the smaller one).
constexpr int BK_KINDS = 3;
__host__ __device__ inline int bk_ppt(int kind, int d) { return kind == 0 ? (d <= 8 ? 8 : 4) : 2; }
__host__ __device__ inline int bk_width(int kind, int d) { return BIG_TPB * bk_ppt(kind, d); }

__host__ __device__ inline int bk_kind(int nL, bool exact, int d) {
  return exact ? 2 : nL >= bk_width(0, d) ? 0 : 1;
}

// chunk of the smaller cluster per tile (2048 points FP32, 1024 FP64),
// widened so that a request has at most max(BIG_MAXT, tiles along the larger
// cluster) tiles
__host__ __device__ inline int bk_chunk(int kind, int nL, int nS, int d) {
  const int w = bk_width(kind, d);
  const int tl = (nL + w - 1) / w;
  int c = kind == 2 ? 1024 : 2048;
  const int maxts = BIG_MAXT / tl > 1 ? BIG_MAXT / tl : 1;
  if ((nS + c - 1) / c > maxts) c = (nS + maxts - 1) / maxts;
  return c;
}

// Schedule of one batch, in s.bsched (ints):
//   [0, B)            tile start of each request in bpart (all kinds)
//   [B, 2B)           tile count of each request
//   per kind k at 2B + k (2B + 1): B request indices, then B + 1 tile prefix
//   at 2B + 3 (2B + 1): n_k (requests of kind k), T_k (tiles), next_k (work
//   counter) for each kind
constexpr int BS_B = BIG_BATCH;
constexpr int BS_LIST = 2 * BS_B;
constexpr int BS_META = 2 * BS_B + BK_KINDS * (2 * BS_B + 1);
constexpr int BS_SIZE = BS_META + 3 * BK_KINDS;

__device__ __forceinline__ int *bs_req(const State &s, int k) {
  return s.bsched + BS_LIST + k * (2 * BS_B + 1);
}
__device__ __forceinline__ int *bs_pre(const State &s, int k) { return bs_req(s, k) + BS_B; }

__device__ int block_incl_scan_big(int v, int *ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int z = lane < BIG_BATCH / 32 ? ws[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    if (lane < BIG_BATCH / 32) ws[lane] = z;
  }
  __syncthreads();
  return x + (w ? ws[w - 1] : 0);
}

// per-kind request lists and tile prefixes of the batch (one block of
// BIG_BATCH threads); dropped duplicates (na = 0) get no tiles
__global__ void k_big_tiles(State s, int r0, int m) {
  __shared__ int ws[BIG_BATCH / 32];
  const int t = threadIdx.x;
  int kind = -1, tiles = 0;
  if (t < m && s.breq_na[r0 + t] > 0) {
    const int nL = max(s.breq_na[r0 + t], s.breq_nb[r0 + t]);
    const int nS = min(s.breq_na[r0 + t], s.breq_nb[r0 + t]);
    kind = bk_kind(nL, s.breq_exact[r0 + t] != 0, s.d);
    const int w = bk_width(kind, s.d), c = bk_chunk(kind, nL, nS, s.d);
    tiles = ((nL + w - 1) / w) * ((nS + c - 1) / c);
  }
  int base = 0, start = 0;
  for (int k = 0; k < BK_KINDS; ++k) {
    const int mine = kind == k;
    const int rank = block_incl_scan_big(mine, ws) - mine;
    const int nk = ws[BIG_BATCH / 32 - 1];
    const int v = mine ? tiles : 0;
    const int pre = block_incl_scan_big(v, ws) - v;
    const int tk = ws[BIG_BATCH / 32 - 1];
    int *req = bs_req(s, k), *pr = bs_pre(s, k);
    if (mine) {
      req[rank] = t;
      pr[rank] = pre;
      start = base + pre;
    }
    if (t == 0) {
      pr[nk] = tk;
      s.bsched[BS_META + 3 * k] = nk;
      s.bsched[BS_META + 3 * k + 1] = tk;
      s.bsched[BS_META + 3 * k + 2] = 0;
    }
    base += tk;
    __syncthreads();
  }
  if (t < m) {
    s.bsched[t] = kind >= 0 ? start : 0;
    s.bsched[BS_B + t] = tiles;
  }
}

// tile `tile` of kind k: the request (index within the batch) and the
// tile's position inside it
__device__ __forceinline__ int bk_find(const State &s, int k, int tile, int &q0) {
  const int n = s.bsched[BS_META + 3 * k];
  const int *pr = bs_pre(s, k);
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pr[mid] <= tile) lo = mid;
    else hi = mid;
  }
  q0 = tile - pr[lo];
  return bs_req(s, k)[lo];
}

// the next tile of kind k for this CTA (dynamic: CTAs that finish early take
// more), or -1 when none is left
__device__ __forceinline__ int bk_next(const State &s, int k, int *sh_tile) {
  if (threadIdx.x == 0) {
    const int t = atomicAdd(&s.bsched[BS_META + 3 * k + 2], 1);
    *sh_tile = t < s.bsched[BS_META + 3 * k + 1] ? t : -1;
  }
  __syncthreads();
  const int t = *sh_tile;
  return t;
}

// block reduction of the tile's partial in a fixed order (deterministic)
template <int LK>
__device__ __forceinline__ void bk_store(const State &s, double v, double *red, int slot) {
  for (int o = 16; o; o >>= 1) {
    const double u = __shfl_xor_sync(0xffffffffu, v, o);
    v = LK == 0 ? fmax(v, u) : v + u;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int w = 1; w < BIG_TPB / 32; ++w) t = LK == 0 ? fmax(t, red[w]) : t + red[w];
    s.bpart[slot] = t;
  }
}

// FP64 tiles (kind 2): 512 points of the larger cluster (two per thread)
// against the smaller one staged through shared memory.
template <int LK, int DP>
__global__ void __launch_bounds__(BIG_TPB) k_big_eval64(State s, int r0) {
  __shared__ double sh[BIG_TPB * DP];
  __shared__ double red[BIG_TPB / 32];
  __shared__ int sh_tile;
  const double *P = s.p64[s.cur];
  const int base = s.bsched[BS_META + 1] + s.bsched[BS_META + 3 + 1];  // after kinds 0, 1
  for (;;) {
    const int tile = bk_next(s, 2, &sh_tile);
    if (tile < 0) break;
    int q0;
    const int r = r0 + bk_find(s, 2, tile, q0);
    int sL = s.breq_sa[r], nL = s.breq_na[r], sS = s.breq_sb[r], nS = s.breq_nb[r];
    if (nS > nL) {
      int t0 = sL; sL = sS; sS = t0;
      t0 = nL; nL = nS; nS = t0;
    }
    const int sch = bk_chunk(2, nL, nS, s.d);
    const int ts = (nS + sch - 1) / sch;  // chunks of the smaller cluster
    const int sc0 = (q0 % ts) * sch, sc1 = min(nS, sc0 + sch);
    const int l0 = (q0 / ts) * BIG_TILE + threadIdx.x, l1 = l0 + BIG_TPB;
    const bool v0 = l0 < nL, v1 = l1 < nL;
    double x0[DP], x1[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      x0[k] = v0 ? P[(size_t)(sL + l0) * DP + k] : 0.0;
      x1[k] = v1 ? P[(size_t)(sL + l1) * DP + k] : 0.0;
    }
    double acc = 0.0, macc = 0.0;
    for (int c0 = sc0; c0 < sc1; c0 += BIG_TPB) {
      const int cn = min(BIG_TPB, sc1 - c0);
      __syncthreads();
      for (int i = threadIdx.x; i < cn * DP; i += BIG_TPB) sh[i] = P[(size_t)(sS + c0) * DP + i];
      __syncthreads();
      for (int j = 0; j < cn; ++j) {
        double d0 = 0, d1 = 0;
#pragma unroll
        for (int k = 0; k < DP; ++k) {
          const double y = sh[j * DP + k];
          const double t0 = x0[k] - y, t1 = x1[k] - y;
          d0 = d0 + t0 * t0;
          d1 = d1 + t1 * t1;
        }
        if (LK == 0) {
          if (v0) macc = fmax(macc, d0);
          if (v1) macc = fmax(macc, d1);
        } else {
          acc += (v0 ? sqrt(d0) : 0.0) + (v1 ? sqrt(d1) : 0.0);
        }
      }
    }
    bk_store<LK>(s, LK == 0 ? macc : acc, red, base + tile);
  }
}

// FP32 tiles, specialised on the true dimension D (rows have stride DP):
// PPT points of the larger cluster per thread, packed in pairs so that every
// subtract and multiply-add is one f32x2 instruction for two point pairs;
// the smaller cluster is staged through shared memory 256 points at a time,
// each coordinate duplicated into both halves of a 64-bit word.  Square
// roots use the hardware approximation (sqrt.approx.f32); with it a term's
// relative error stays within ((D+1)/2 + 4)u <= (D+16)u, the bound the search
// states for FP32 distances.  Packed operations round each half as the scalar
// instruction would.
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// One staged chunk of the smaller cluster against a thread's NP point pairs.
// Average: each half of `part` takes 4 x NP terms per group of 4 staged
// points (at most 16); 16 groups are summed in FP32 before each FP64 add
// (relative error <= 30u per FP64 add, as before packing).
template <int LK, int D, int NP, bool FULL>
__device__ __forceinline__ void big32_chunk(const unsigned long long *sh, int cn,
                                            const unsigned long long (&x)[NP][D],
                                            const bool (&v)[2 * NP], double &acc, float &macc) {
  unsigned long long part2 = 0ull;  // (0.f, 0.f)
  int groups = 0;
  for (int j0 = 0; j0 < cn; j0 += 4) {
    const int jn = min(4, cn - j0);
    unsigned long long part = 0ull;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      if (jj < jn) {
        const unsigned long long *y = sh + (j0 + jj) * D;
        unsigned long long yk[D];
#pragma unroll
        for (int k = 0; k < D; ++k) yk[k] = y[k];
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          unsigned long long t = f2_sub(x[q][0], yk[0]);
          unsigned long long d2 = f2_mul(t, t);
#pragma unroll
          for (int k = 1; k < D; ++k) {
            t = f2_sub(x[q][k], yk[k]);
            d2 = f2_fma(t, t, d2);
          }
          float a, b;
          f2_unpack(d2, a, b);
          if (LK == 0) {
            macc = fmaxf(macc, (FULL || v[2 * q]) ? a : 0.f);
            macc = fmaxf(macc, (FULL || v[2 * q + 1]) ? b : 0.f);
          } else {
            const float ra = (FULL || v[2 * q]) ? sqrt_approx(a) : 0.f;
            const float rb = (FULL || v[2 * q + 1]) ? sqrt_approx(b) : 0.f;
            part = f2_add(part, f2_pack(ra, rb));
          }
        }
      }
    }
    if (LK != 0) {
      part2 = f2_add(part2, part);
      if (++groups == 16) {
        float a, b;
        f2_unpack(part2, a, b);
        acc += (double)a + (double)b;
        part2 = 0ull;
        groups = 0;
      }
    }
  }
  if (LK != 0) {
    float a, b;
    f2_unpack(part2, a, b);
    acc += (double)a + (double)b;
  }
}

template <int LK, int D, int DP, int KIND>
__global__ void __launch_bounds__(BIG_TPB) k_big_eval32(State s, int r0) {
  constexpr int PPT = KIND == 0 ? (D <= 8 ? 8 : 4) : 2, NP = PPT / 2;
  __shared__ unsigned long long sh[BIG_TPB * D];
  __shared__ double red[BIG_TPB / 32];
  __shared__ int sh_tile;
  const float *P = s.p32[s.cur];
  const int base = KIND == 0 ? 0 : s.bsched[BS_META + 1];  // kind 1 tiles follow kind 0's
  for (;;) {
    const int tile = bk_next(s, KIND, &sh_tile);
    if (tile < 0) break;
    int q0;
    const int r = r0 + bk_find(s, KIND, tile, q0);
    int sL = s.breq_sa[r], nL = s.breq_na[r], sS = s.breq_sb[r], nS = s.breq_nb[r];
    if (nS > nL) {
      int t0 = sL; sL = sS; sS = t0;
      t0 = nL; nL = nS; nS = t0;
    }
    const int sch = bk_chunk(KIND, nL, nS, D);
    const int ts = (nS + sch - 1) / sch;  // chunks of the smaller cluster
    const int sc0 = (q0 % ts) * sch, sc1 = min(nS, sc0 + sch);
    const int q = q0 / ts;
    unsigned long long x[NP][D];
    bool v[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) v[p] = q * (BIG_TPB * PPT) + p * BIG_TPB + (int)threadIdx.x < nL;
#pragma unroll
    for (int h = 0; h < NP; ++h) {
      const int l0 = q * (BIG_TPB * PPT) + (2 * h) * BIG_TPB + threadIdx.x;
      const int l1 = l0 + BIG_TPB;
#pragma unroll
      for (int k = 0; k < D; ++k)
        x[h][k] = f2_pack(v[2 * h] ? P[(size_t)(sL + l0) * DP + k] : 0.f,
                          v[2 * h + 1] ? P[(size_t)(sL + l1) * DP + k] : 0.f);
    }
    double acc = 0.0;
    float macc = 0.f;
    const bool full = v[PPT - 1];  // all points valid: no selects
    for (int c0 = sc0; c0 < sc1; c0 += BIG_TPB) {
      const int cn = min(BIG_TPB, sc1 - c0);
      __syncthreads();
      for (int i = threadIdx.x; i < cn * D; i += BIG_TPB) {
        const int j = i / D, k = i - j * D;
        const float y = P[(size_t)(sS + c0 + j) * DP + k];
        sh[i] = f2_pack(y, y);
      }
      __syncthreads();
      if (full)
        big32_chunk<LK, D, NP, true>(sh, cn, x, v, acc, macc);
      else
        big32_chunk<LK, D, NP, false>(sh, cn, x, v, acc, macc);
    }
    bk_store<LK>(s, LK == 0 ? (double)macc : acc, red, base + tile);
  }
}

// Drop the second of two requests for the same unordered pair in a batch
// (both terminals asked): one value fills both tables.  Quadratic in the
// batch, one block of BIG_BATCH threads.
__global__ void k_big_dedup(State s, int r0, int m) {
  const int t = threadIdx.x;
  if (t >= m) return;
  const int r = r0 + t;
  const int a = min(s.breq_i[r], s.breq_j[r]), b = max(s.breq_i[r], s.breq_j[r]);
  const uint8_t ex = s.breq_exact[r];
  for (int u = 0; u < t; ++u) {
    const int q = r0 + u;
    if (min(s.breq_i[q], s.breq_j[q]) == a && max(s.breq_i[q], s.breq_j[q]) == b &&
        s.breq_exact[q] >= ex) {
      s.breq_na[r] = 0;  // k_big_tiles gives it no tiles
      return;
    }
  }
}

// Insert that may evict: a big pair's value must land in both tables, since
// the re-run search reads it there.  A free or stale slot is taken if there
// is one; otherwise the live entry with the largest distance (the neighbour
// least likely to be anyone's nearest) makes room.  Slots claimed by
// concurrent writers are skipped; after a few lost races the value is dropped
// (the re-run search then asks for it again or evaluates it itself).
__device__ void cache_insert_evict(const State &s, int owner, int nbr, int nbr_gen, double v,
                                   float e) {
  const int S = s.cache_slots;
  const unsigned long long want = ckey_of(nbr, nbr_gen);
  const size_t base = (size_t)owner * S;
  for (int attempt = 0; attempt < 4; ++attempt) {
    int victim = -1;
    double vmax = -1.0;
    unsigned long long vkey = 0;
    for (int t = 0; t < S; ++t) {
      const unsigned long long cur = slot_key(s, base + t);
      if (cur == want) {
        if (s.cpart[base + t] != 0) slot_put(s, base + t, cur, want, v, e);
        return;
      }
      if (slot_free(s, cur)) {
        if (slot_put(s, base + t, cur, want, v, e)) return;
        continue;
      }
      if (cur == CKEY_BUSY) continue;
      const double cv = *(volatile double *)&s.cval[base + t];
      if (cv > vmax) {
        vmax = cv;
        victim = t;
        vkey = cur;
      }
    }
    if (victim < 0) return;
    if (slot_put(s, base + victim, vkey, want, v, e)) return;
  }
}

// this round's result table: a slot is claimed by CAS to BUSY, filled, then
// published (readers run in later kernels); a result that finds no slot
// within SIDE_PROBES is dropped (the re-run search asks again)
__device__ void side_put(const State &s, int lo, int hi, double v, float e) {
  const unsigned long long want = ((unsigned long long)(unsigned)lo << 32) | (unsigned)hi;
  unsigned h = side_hash(lo, hi, s.side_cap);
  for (int q = 0; q < SIDE_PROBES; ++q, h = (h + 1) & (unsigned)(s.side_cap - 1)) {
    const unsigned long long cur = *(volatile unsigned long long *)&s.side_key[h];
    if (cur == want) return;
    if (cur != CKEY_EMPTY) continue;
    if (atomicCAS(&s.side_key[h], CKEY_EMPTY, CKEY_BUSY) != CKEY_EMPTY) continue;
    s.side_val[h] = v;
    s.side_err[h] = e;
    __threadfence();
    atomicExch(&s.side_key[h], want);
    return;
  }
}

// one warp per request: fold its tiles in order, cache the distance
__global__ void k_big_final(State s, int r0, int m) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < m; q += warps) {
    const int r = r0 + q;
    if (s.breq_na[r] == 0) continue;  // duplicate dropped by k_big_dedup
    const int t0 = s.bsched[q], t1 = t0 + s.bsched[BS_B + q];
    double v = 0.0;
    for (int t = t0 + lane; t < t1; t += 32) v = s.linkage == 0 ? fmax(v, s.bpart[t]) : v + s.bpart[t];
    for (int o = 16; o; o >>= 1) {
      const double u = __shfl_xor_sync(0xffffffffu, v, o);
      v = s.linkage == 0 ? fmax(v, u) : v + u;
    }
    if (lane == 0) {
      const int i = s.breq_i[r], j = s.breq_j[r];
      const int cov = s.breq_cov[r];  // points of side a covered by the partial entry
      const double na = (double)s.breq_na[r], nb = (double)s.breq_nb[r];
      const bool exact = s.breq_exact[r] != 0;
      float e = exact ? 0.f : fmaxf(s.idpts[s.inst[i]], EST_MARK);
      double D;
      if (s.linkage == 0) {
        D = sqrt(v);
        if (cov > 0) {
          D = fmax(D, s.breq_base[r]);
          e = fmaxf(e, s.breq_berr[r]);
        }
      } else {
        D = (v + (cov > 0 ? s.breq_base[r] : 0.0)) / ((na + cov) * nb);
        if (cov > 0) e = (float)((cov * (double)s.breq_berr[r] + na * e) / (na + cov));
      }
      if (!exact) e = fmaxf(e, EST_MARK);
      atomicAdd(&s.ctr->big_pp, (unsigned long long)s.breq_na[r] * (unsigned long long)s.breq_nb[r]);
      if (exact) atomicAdd(&s.ctr->big_exact, 1ull);
      cache_insert_evict(s, i, j, s.gen[j], D, e);
      cache_insert_evict(s, j, i, s.gen[i], D, e);
      side_put(s, min(i, j), max(i, j), D, e);
    }
  }
}

// merged cids change identity: entries that name them go stale
__global__ void k_gen_bump(State s, int npairs) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
    s.gen[s.pair_lo[p]] += 1;
    s.gen[s.pair_hi[p]] += 1;
  }
}

// compaction phase 1: chain repair (succ merged this round -> terminal) and
// per-block counts of (active, terminal, points)
__global__ void k_cmp_count(State s, const int32_t *order, int K, int round) {
  const int p = blockIdx.x * TPB + threadIdx.x;
  int keep = 0, ist = 0, sz = 0;
  if (p < K) {
    const int c = order[p];
    if (s.alive[c] && !s.idone[s.inst[c]]) {
      keep = 1;
      int sc = s.succ[c];
      if (sc >= 0 && s.mround[sc] == round) {
        s.succ[c] = -1;
        sc = -1;
      }
      ist = sc < 0;
      sz = s.csize[c];
    }
  }
  keep = block_sum(keep);
  ist = block_sum(ist);
  sz = block_sum(sz);
  if (threadIdx.x == 0) {
    s.bsum[blockIdx.x] = keep;
    s.bsum[gridDim.x + blockIdx.x] = ist;
    s.bsum[2 * gridDim.x + blockIdx.x] = sz;
  }
}

__global__ void k_cmp_top(State s, int nb) {
  // three independent exclusive scans of nb block sums, one per warp-group pass
  for (int f = 0; f < 3; ++f) {
    int32_t *bs = s.bsum + (size_t)f * nb;
    const int per = cdiv(nb, TPB);
    const int b0 = threadIdx.x * per;
    int sum = 0;
    for (int i = 0; i < per; ++i)
      if (b0 + i < nb) sum += bs[b0 + i];
    int t;
    int pre = block_excl_scan(sum, &t);
    for (int i = 0; i < per; ++i)
      if (b0 + i < nb) {
        int v = bs[b0 + i];
        bs[b0 + i] = pre;
        pre += v;
      }
    if (threadIdx.x == 0) {
      if (f == 0) s.ctr->nactive = t;
      if (f == 1) s.ctr->nterm = t;
    }
    __syncthreads();
  }
}

// Variance of cluster c (mean squared distance of its points to the
// centroid).  Average linkage needs a rigorous upper bound: it comes from the
// sums of squared norms with a margin covering the worst-case rounding of
// sums of sz terms.  avg-2 needs the value its FP64 distances use (SSE / sz),
// rounded up (the search's FP32 error bound covers the difference).
__device__ float cluster_var_up(const State &s, int c, int sz) {
  if (s.linkage == LK_AVG2) return __double2float_ru(s.sse[c] / (double)sz);
  if (s.linkage != LK_AVERAGE) return 0.f;
  const int dp = s.dp;
  const double inv = 1.0 / (double)sz;
  double c2 = 0.0;
  for (int k = 0; k < dp; ++k) {
    const double m = s.csum[(size_t)c * dp + k] * inv;
    c2 += m * m;
  }
  const double M = (double)s.iscale[s.inst[c]];
  const double v = fmax(s.csq[c] * inv - c2, 0.0);
  const double margin = ldexp((double)sz * s.d * M * M, -50);
  return __double2float_ru(v + margin);
}

__global__ void k_cmp_write(State s, const int32_t *order, int32_t *order_out, int32_t *seg_out,
                            int K, int round) {
  const int p = blockIdx.x * TPB + threadIdx.x;
  const int nb = gridDim.x;
  int keep = 0, ist = 0, sz = 0, c = -1;
  if (p < K) {
    c = order[p];
    if (s.alive[c] && !s.idone[s.inst[c]]) {
      keep = 1;
      ist = s.succ[c] < 0;
      sz = s.csize[c];
    }
  }
  int t;
  const int ok = block_excl_scan(keep, &t) + s.bsum[blockIdx.x];
  const int ot = block_excl_scan(ist, &t) + s.bsum[nb + blockIdx.x];
  const int os = block_excl_scan(sz, &t) + s.bsum[2 * nb + blockIdx.x];
  if (keep) {
    order_out[ok] = c;
    s.pos[c] = ok;
    if (seg_out) seg_out[c] = os;
    const int dp = s.dp;
    for (int k = 0; k < dp; ++k) {
      s.q32[(size_t)ok * dp + k] = s.cent32[(size_t)c * dp + k];
      s.q64[(size_t)ok * dp + k] = s.cent[(size_t)c * dp + k];
      s.qblo[(size_t)ok * dp + k] = s.blo[(size_t)c * dp + k];
      s.qbhi[(size_t)ok * dp + k] = s.bhi[(size_t)c * dp + k];
    }
    s.qsz[ok] = sz;
    s.qseg[ok] = os;
    s.qvar[ok] = sz > 1 ? cluster_var_up(s, c, sz) : 0.f;
    s.qinst[ok] = s.iseq[s.inst[c]];
    if (ist) {
      s.term[ot] = c;
      s.isterm[c] = round + 1;
    }
  }
}

// move points so that each merged cluster is one segment
__global__ void k_relayout(State s, int pc, int64_t n) {  // n: points in the current layout
  const int dp = s.dp, nx = pc ^ 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int c = s.plab[pc][p];
    int r = c;
    int off = (int)p - s.seg[pc][c];
    if (!s.alive[c]) {
      r = s.rootof[c];
      off += s.reloff[c];
    }
    if (s.idone[s.inst[r]]) continue;  // finished instance: its points leave
    const int64_t q = (int64_t)s.seg[nx][r] + off;
    for (int k = 0; k < dp; ++k) {
      s.p64[nx][q * dp + k] = s.p64[pc][p * dp + k];
      s.p32[nx][q * dp + k] = s.p32[pc][p * dp + k];
    }
    s.plab[nx][q] = r;
  }
}

// canonical order of the merge records: stable passes by cid_a, then size,
// then height (non-negative doubles order like their bit patterns)
__global__ void k_rec_key(const State s, int m, int field, const int32_t *perm, uint64_t *keys,
                          int32_t *vals) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int v = perm ? perm[i] : i;
    uint64_t k;
    if (field == 0)
      k = (uint64_t)(uint32_t)s.m_a[v];
    else if (field == 1)
      k = (uint64_t)(uint32_t)s.m_size[v];
    else
      k = (uint64_t)__double_as_longlong(s.m_h[v]);
    keys[i] = k;
    vals[i] = v;
  }
}

__global__ void k_rec_gather(const State s, int m, const int32_t *perm, hac_merge *out,
                             int32_t *out_round) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int v = perm[i];
    hac_merge r;
    r.cid_a = s.m_a[v];
    r.cid_b = s.m_b[v];
    r.height = s.m_h[v];
    r.size = s.m_size[v];
    out[i] = r;
    out_round[i] = s.m_round[v];
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// instance
// ---------------------------------------------------------------------------
struct hac_ctx {
  State s{};
  int64_t n = 0;
  int d = 0;
  hac_dtype dt = HAC_F64;
  hac_linkage lk = HAC_WARD;
  void *raw = nullptr;          // device copy of the input points (input order)
  cudaStream_t own = nullptr;
  std::vector<void *> allocs;
  int64_t bytes = 0;
  // sort scratch
  uint64_t *keys[2] = {nullptr, nullptr};
  int32_t *vals[2] = {nullptr, nullptr};
  int32_t *hist = nullptr, *hbs = nullptr;
  unsigned long long *bb = nullptr;  // 2 x MAXD bbox words
  int nlev_max = 1;
  int cache_alloc_slots = 0;  // slots per cluster the cache tables were allocated for
  int64_t lay_n = 0;          // points in the current layout (all n for one instance)
  // pairs of at least this many point pairs go to the GPU-wide evaluation
  // (FP32 / FP64 values); HAC_BIG_PAIRS / HAC_BIG_PAIRS_F64 override them
  long long big_pairs = BIG_PAIRS, big_pairs64 = BIG_PAIRS_F64;
  long long warp_budget = WARP_BUDGET;  // HAC_WARP_BUDGET overrides it
  int64_t launches = 0;  // kernels launched in the current run
  int ocur = 0, pcur = 0;
  bool done = false;
  int64_t n_merges = 0;
  hac_stats_t st{};
  hac_merge *dout = nullptr;        // canonical dendrogram (device)
  int32_t *dout_round = nullptr;
};

namespace {

template <typename T>
int dalloc(hac_ctx *h, T **p, size_t count) {
  if (count == 0) count = 1;
  void *q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return HAC_ENOMEM;
  }
  h->allocs.push_back(q);
  h->bytes += (int64_t)(count * sizeof(T));
  *p = (T *)q;
  return HAC_OK;
}

void free_all(hac_ctx *h) {
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->own) cudaStreamDestroy(h->own);
  h->own = nullptr;
}

int pad_dim(int d) { return d <= 2 ? 2 : d <= 4 ? 4 : d <= 8 ? 8 : 16; }

int alloc_state(hac_ctx *h) {
  State &s = h->s;
  const int64_t n = h->n;
  const int dp = s.dp;
  int rc = 0;
#define A(ptr, cnt)                          \
  do {                                       \
    if ((rc = dalloc(h, &(ptr), (size_t)(cnt)))) return rc; \
  } while (0)
  for (int b = 0; b < 2; ++b) {
    A(s.p64[b], n * dp);
    A(s.p32[b], n * dp);
    A(s.plab[b], n);
    A(s.seg[b], n);
    A(s.order[b], n);
  }
  A(s.csize, n);
  A(s.q32, n * dp);
  A(s.q64, n * dp);
  A(s.qblo, n * dp);
  A(s.qbhi, n * dp);
  A(s.qsz, n);
  A(s.qseg, n);
  A(s.csum, n * dp);
  A(s.csq, n);
  A(s.sse, n);
  A(s.qvar, n);
  A(s.cent, n * dp);
  A(s.cent32, n * dp);
  A(s.blo, n * dp);
  A(s.bhi, n * dp);
  A(s.succ, n);
  A(s.pred, n);
  A(s.mround, n);
  A(s.isterm, n);
  A(s.alive, n);
  A(s.rootof, n);
  A(s.reloff, n);
  A(s.osize, n);
  A(s.partner, n);
  A(s.gen, n);
  A(s.inst, n);
  A(s.qinst, n);
  if (s.max_inst < 1) s.max_inst = 1;
  A(s.islack, s.max_inst);
  A(s.iscale, s.max_inst);
  A(s.idpts, s.max_inst);
  A(s.irec, s.max_inst);
  A(s.irecn, s.max_inst);
  A(s.iact, s.max_inst);
  A(s.idone, s.max_inst);
  A(s.iseq, s.max_inst);
  A(s.done_list, 2 * s.max_inst);  // a dropped instance can be listed twice
  A(s.pos, n);
  A(s.Ekey, n);
  A(s.Ecid, n);
  A(s.term, n);
  A(s.pair_lo, n / 2 + 1);
  A(s.pair_hi, n / 2 + 1);
  A(s.pair_key, n / 2 + 1);
  A(s.m_a, n);
  A(s.m_b, n);
  A(s.m_size, n);
  A(s.m_round, n);
  A(s.m_h, n);
  // tree levels sized for K = n
  int base = 0;
  const int nlev = tree_levels((int)n);
  for (int L = 0; L <= MAXLEV; ++L) {
    s.lvl_base[L] = base;
    if (L < nlev) base += level_count((int)n, L);
  }
  h->nlev_max = nlev;
  A(s.nclo, (int64_t)base * dp);
  A(s.nchi, (int64_t)base * dp);
  A(s.nhmin, (int64_t)base * dp);
  A(s.nlmax, (int64_t)base * dp);
  A(s.nnmin, base);
  A(s.ninlo, base);
  A(s.ninhi, base);
  A(s.bsum, 3 * (int64_t)cdiv(n, TPB) + 3);
  A(s.ctr, 1);
  for (int b = 0; b < 2; ++b) {
    A(h->keys[b], n);
    A(h->vals[b], n);
  }
  const int ntiles = cdiv(n, RS_TILE);
  A(h->hist, (int64_t)256 * ntiles + 1);
  A(h->hbs, cdiv((int64_t)256 * ntiles, SC_TILE) + 1);
  A(h->bb, 2 * MAXD);
  A(h->dout, n);
  A(h->dout_round, n);
#undef A
  return HAC_OK;
}

#define CK(x)                                \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return HAC_EDEVICE; \
  } while (0)

int grid_for(int64_t work, int tpb) {
  int64_t g = (work + tpb - 1) / tpb;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (int)g;
}

// CTAs that stay resident together: one wave, tiles handed out dynamically
template <typename F>
int resident_grid(F kernel) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, BIG_TPB, 0) != cudaSuccess) {
    cudaGetLastError();
    return 152 * 4;
  }
  return std::max(1, sms) * std::max(1, per);
}

template <int LK, int D>
void launch_big32(const State &s, int r0, cudaStream_t st) {
  constexpr int DP = D <= 2 ? 2 : D <= 4 ? 4 : D <= 8 ? 8 : 16;
  static const int g0 = resident_grid(k_big_eval32<LK, D, DP, 0>);
  static const int g1 = resident_grid(k_big_eval32<LK, D, DP, 1>);
  k_big_eval32<LK, D, DP, 0><<<g0, BIG_TPB, 0, st>>>(s, r0);
  k_big_eval32<LK, D, DP, 1><<<g1, BIG_TPB, 0, st>>>(s, r0);
}

template <int LK, int DP>
void launch_big64(const State &s, int r0, cudaStream_t st) {
  static const int g = resident_grid(k_big_eval64<LK, DP>);
  k_big_eval64<LK, DP><<<g, BIG_TPB, 0, st>>>(s, r0);
}

template <int LK>
int launch_big_lk(const State &s, int r0, cudaStream_t st) {
  switch (s.d) {  // FP32 requests, specialised on the true dimension
    case 1: launch_big32<LK, 1>(s, r0, st); break;
    case 2: launch_big32<LK, 2>(s, r0, st); break;
    case 3: launch_big32<LK, 3>(s, r0, st); break;
    case 4: launch_big32<LK, 4>(s, r0, st); break;
    case 5: launch_big32<LK, 5>(s, r0, st); break;
    case 6: launch_big32<LK, 6>(s, r0, st); break;
    case 7: launch_big32<LK, 7>(s, r0, st); break;
    case 8: launch_big32<LK, 8>(s, r0, st); break;
    case 9: launch_big32<LK, 9>(s, r0, st); break;
    case 10: launch_big32<LK, 10>(s, r0, st); break;
    case 11: launch_big32<LK, 11>(s, r0, st); break;
    case 12: launch_big32<LK, 12>(s, r0, st); break;
    case 13: launch_big32<LK, 13>(s, r0, st); break;
    case 14: launch_big32<LK, 14>(s, r0, st); break;
    case 15: launch_big32<LK, 15>(s, r0, st); break;
    case 16: launch_big32<LK, 16>(s, r0, st); break;
    default: return HAC_EINTERNAL;
  }
  switch (s.dp) {  // FP64 requests
    case 2: launch_big64<LK, 2>(s, r0, st); break;
    case 4: launch_big64<LK, 4>(s, r0, st); break;
    case 8: launch_big64<LK, 8>(s, r0, st); break;
    case 16: launch_big64<LK, 16>(s, r0, st); break;
    default: return HAC_EINTERNAL;
  }
  CK(cudaGetLastError());
  return HAC_OK;
}

int launch_big(const State &s, int r0, cudaStream_t st) {
  return s.linkage == 0 ? launch_big_lk<0>(s, r0, st) : launch_big_lk<1>(s, r0, st);
}

template <int DP>
int build_tree_dp(hac_ctx *h, const int32_t *order, int K, cudaStream_t st) {
  const int nlev = tree_levels(K);
  h->launches += nlev;
  k_tree_leaf<DP><<<grid_for((int64_t)level_count(K, 0) * 32, TPB), TPB, 0, st>>>(h->s, order, K);
  for (int L = 1; L < nlev; ++L)
    k_tree_up<DP><<<grid_for((int64_t)level_count(K, L) * 32, TPB), TPB, 0, st>>>(h->s, K, L);
  CK(cudaGetLastError());
  return HAC_OK;
}

int build_tree(hac_ctx *h, const int32_t *order, int K, cudaStream_t st) {
  switch (h->s.dp) {
    case 2: return build_tree_dp<2>(h, order, K, st);
    case 4: return build_tree_dp<4>(h, order, K, st);
    case 8: return build_tree_dp<8>(h, order, K, st);
    case 16: return build_tree_dp<16>(h, order, K, st);
  }
  return HAC_EINTERNAL;
}

// stable LSD sort of h->keys[0]/h->vals[0] (first m entries) by the low
// `bits` bits of the key; returns the buffer index holding the result
int radix_sort(hac_ctx *h, int m, int bits, cudaStream_t st) {
  const int ntiles = cdiv(m, RS_TILE);
  const int hm = 256 * ntiles;
  const int hb = cdiv(hm, SC_TILE);
  int cur = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    h->launches += 5;
    k_rs_hist<<<ntiles, TPB, 0, st>>>(h->keys[cur], m, shift, h->hist, ntiles);
    k_scan_reduce<<<hb, TPB, 0, st>>>(h->hist, hm, h->hbs);
    k_scan_top<<<1, TPB, 0, st>>>(h->hbs, hb, nullptr);
    k_scan_down<<<hb, TPB, 0, st>>>(h->hist, h->hist, hm, h->hbs);
    k_rs_scatter<<<ntiles, TPB, 0, st>>>(h->keys[cur], h->vals[cur], h->keys[cur ^ 1],
                                         h->vals[cur ^ 1], m, shift, h->hist, ntiles);
    cur ^= 1;
  }
  CK(cudaGetLastError());
  return cur;
}

int bits_for(int64_t maxval) {
  int b = 1;
  while (b < 63 && ((int64_t)1 << b) <= maxval) ++b;
  return b;
}

template <typename T>
int init_layout(hac_ctx *h, cudaStream_t st) {
  State &s = h->s;
  const T *X = (const T *)h->raw;
  const int64_t n = h->n;
  const int d = h->d;
  std::vector<unsigned long long> init(2 * MAXD);
  for (int k = 0; k < MAXD; ++k) {
    init[k] = ~0ull;
    init[MAXD + k] = 0ull;
  }
  CK(cudaMemcpyAsync(h->bb, init.data(), 2 * MAXD * sizeof(unsigned long long),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(s.ctr, 0, sizeof(Counters), st));
  k_bbox<T><<<grid_for(n, TPB), TPB, 0, st>>>(X, n, d, h->bb, h->bb + MAXD, s.ctr);
  h->launches += 3;  // bbox, morton, layout
  CK(cudaGetLastError());
  std::vector<unsigned long long> bb(2 * MAXD);
  Counters c0;
  CK(cudaMemcpyAsync(bb.data(), h->bb, 2 * MAXD * sizeof(unsigned long long),
                     cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&c0, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (c0.err & ERR_NONFINITE) return HAC_EINVAL;
  auto dec = [](unsigned long long u) {
    unsigned long long b = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    double x;
    memcpy(&x, &b, 8);
    return x;
  };
  MortonParams mp{}, ctrp{};
  double scale = 0.0;
  for (int k = 0; k < d; ++k) {
    double lo = dec(bb[k]), hi = dec(bb[MAXD + k]);
    mp.lo[k] = lo;
    mp.inv[k] = hi > lo ? 1.0 / (hi - lo) : 0.0;
    ctrp.lo[k] = 0.5 * (lo + hi);
    scale = std::max(scale, std::max(std::fabs(lo - ctrp.lo[k]), std::fabs(hi - ctrp.lo[k])));
  }
  mp.bits = std::min(21, 64 / d);
  s.abs_slack = std::max(scale, 1e-300) * std::ldexp(1.0, -18);
  s.coord_scale = (float)(scale * (1.0 + 1e-6));
  s.delta_pts = s.pts32_exact ? 0.f : 2.01f * 5.9604645e-8f * s.coord_scale * std::sqrt((float)d);
  k_inst_set<<<1, 1, 0, st>>>(s, 0, (float)s.abs_slack, s.coord_scale, s.delta_pts, 0, (int)n, 0);
  k_morton<T><<<grid_for(n, TPB), TPB, 0, st>>>(X, n, d, mp, h->keys[0], h->vals[0]);
  CK(cudaGetLastError());
  int sc = radix_sort(h, (int)n, mp.bits * d, st);
  if (sc < 0) return sc;
  h->ocur = h->pcur = 0;
  h->lay_n = n;
  s.cur = 0;
  k_layout<T><<<grid_for(n, TPB), TPB, 0, st>>>(s, X, h->vals[sc], ctrp);
  CK(cudaGetLastError());
  Counters c{};
  c.nterm = (int)n;
  c.nactive = (int)n;
  CK(cudaMemcpyAsync(s.ctr, &c, sizeof(Counters), cudaMemcpyHostToDevice, st));
  return build_tree(h, s.order[0], (int)n, st);
}

int create_common(const void *pts, bool dev, int64_t n, int d, hac_dtype dt, hac_linkage lk,
                  hac_t *out) {
  if (!out) return HAC_EINVAL;
  *out = nullptr;
  if (!pts || n < 1 || n > (int64_t)INT32_MAX / 2 || d < 1 || d > MAXD) return HAC_EINVAL;
  if (dt != HAC_F32 && dt != HAC_F64) return HAC_EINVAL;
  if (lk != HAC_COMPLETE && lk != HAC_AVERAGE && lk != HAC_WARD && lk != HAC_AVERAGE_SQ)
    return HAC_EINVAL;
  const size_t esz = dt == HAC_F32 ? 4 : 8;
  if (!dev) {
    for (int64_t i = 0; i < n * d; ++i) {
      double x = dt == HAC_F32 ? (double)((const float *)pts)[i] : ((const double *)pts)[i];
      if (!std::isfinite(x)) return HAC_EINVAL;
    }
  }
  hac_ctx *h = new (std::nothrow) hac_ctx();
  if (!h) return HAC_ENOMEM;
  h->n = n;
  h->d = d;
  h->dt = dt;
  h->lk = lk;
  h->s.n = n;
  h->s.d = d;
  h->s.dp = pad_dim(d);
  h->s.linkage = (int)lk;
  h->s.pts32_exact = dt == HAC_F32;
  if (const char *e = getenv("HAC_BIG_PAIRS")) h->big_pairs = std::max(1ll, atoll(e));
  if (const char *e = getenv("HAC_BIG_PAIRS_F64")) h->big_pairs64 = std::max(1ll, atoll(e));
  if (const char *e = getenv("HAC_WARP_BUDGET")) h->warp_budget = std::max(1ll, atoll(e));
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HAC_EDEVICE;
  }
  int rc = alloc_state(h);
  if (!rc) {
    void *raw = nullptr;
    if (cudaMalloc(&raw, n * d * esz) != cudaSuccess) {
      cudaGetLastError();
      rc = HAC_ENOMEM;
    } else {
      h->allocs.push_back(raw);
      h->bytes += n * d * esz;
      h->raw = raw;
      if (cudaMemcpyAsync(raw, pts, n * d * esz,
                          dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          h->own) != cudaSuccess ||
          cudaStreamSynchronize(h->own) != cudaSuccess)
        rc = HAC_EDEVICE;
    }
  }
  if (rc) {
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return HAC_OK;
}

struct Ev {
  cudaEvent_t e = nullptr;
  Ev() { cudaEventCreate(&e); }
  ~Ev() {
    if (e) cudaEventDestroy(e);
  }
};

// Per-round timing / counters of round_step (events may be null: no timing)
struct RoundCtl {
  cudaEvent_t e1 = nullptr, e2 = nullptr, eq0 = nullptr, eq1 = nullptr, eb0 = nullptr,
              eb1 = nullptr;
  double ms_query = 0, ms_big = 0;
  int64_t qlaunch = 0, big_launch = 0, searches = 0;
  int big_iters = 0, big_reqs = 0;
};

void fill_query_args(hac_ctx *h, QueryArgs &qa, int round, int K, int nterm) {
  State &s = h->s;
  qa.d = s.d;
  qa.linkage = s.linkage;
  qa.round = round;
  qa.K = K;
  qa.nterm = nterm;
  qa.abs_slack = s.abs_slack;
  qa.coord_scale = s.coord_scale;
  qa.delta_pts = s.delta_pts;
  qa.term = s.term;
  qa.order = s.order[h->ocur];
  qa.pos = s.pos;
  qa.csize = s.csize;
  qa.seg = s.seg[h->pcur];
  qa.cent = s.cent;
  qa.p64 = s.p64[h->pcur];
  qa.cent32 = s.cent32;
  qa.blo = s.blo;
  qa.bhi = s.bhi;
  qa.p32 = s.p32[h->pcur];
  qa.pred = s.pred;
  qa.q32 = s.q32;
  qa.q64 = s.q64;
  qa.qblo = s.qblo;
  qa.qbhi = s.qbhi;
  qa.qsz = s.qsz;
  qa.qseg = s.qseg;
  qa.qvar = s.qvar;
  qa.sse = s.sse;
  qa.nclo = s.nclo;
  qa.nchi = s.nchi;
  qa.nhmin = s.nhmin;
  qa.nlmax = s.nlmax;
  qa.nnmin = s.nnmin;
  qa.inst = s.inst;
  qa.qinst = s.qinst;
  qa.ninlo = s.ninlo;
  qa.ninhi = s.ninhi;
  qa.islack = s.islack;
  qa.iscale = s.iscale;
  qa.idpts = s.idpts;
  for (int L = 0; L <= MAXLEV; ++L) qa.lvl_base[L] = s.lvl_base[L];
  qa.Ekey = s.Ekey;
  qa.Ecid = s.Ecid;
  qa.ctr = s.ctr;
  qa.cache_slots = s.cache_slots;
  qa.ins_cap = s.ins_cap;
  qa.ckey = s.ckey;
  qa.cval = s.cval;
  qa.cerr = s.cerr;
  qa.cpart = s.cpart;
  qa.gen = s.gen;
  qa.ins_i = s.ins_i;
  qa.ins_j = s.ins_j;
  qa.ins_v = s.ins_v;
  qa.ins_e = s.ins_e;
  qa.defer = s.cache_slots > 0 && !closed_form(s.linkage) ? 1 : 0;
  qa.big_pairs = h->big_pairs;
  qa.big_pairs64 = h->big_pairs64;
  qa.warp_budget = h->warp_budget;
  qa.noprune = s.noprune;
  qa.side_cap = s.side_cap;
  qa.side_key = s.side_key;
  qa.side_val = s.side_val;
  qa.side_err = s.side_err;
  qa.breq_cap = s.breq_cap;
  qa.breq_i = s.breq_i;
  qa.breq_j = s.breq_j;
  qa.breq_sa = s.breq_sa;
  qa.breq_na = s.breq_na;
  qa.breq_sb = s.breq_sb;
  qa.breq_nb = s.breq_nb;
  qa.breq_exact = s.breq_exact;
  qa.breq_base = s.breq_base;
  qa.breq_cov = s.breq_cov;
  qa.breq_berr = s.breq_berr;
  qa.pend_out = s.pend[0];
}

#define EVREC(ev) \
  do {            \
    if (ev) cudaEventRecord(ev, st); \
  } while (0)

// One round of Algorithm 1 over the current terminal list: the searches (with
// big pairs handed to the whole GPU and the deferring searches re-run), the
// chain update, the R-NN filter, the merges, the cache update, the compaction
// and the point re-layout.  *npairs_out receives the merges made; the caller
// reads the counters and rebuilds the tree.
int round_step(hac_ctx *h, cudaStream_t st, int round, int K, int nterm, RoundCtl &ctl,
               int *npairs_out) {
  State &s = h->s;
  const bool need_points = !closed_form(s.linkage);
  int rc = 0;
  s.cur = h->pcur;
  QueryArgs qa{};
  fill_query_args(h, qa, round, K, nterm);
  const bool defer = qa.defer != 0;
  if (defer)
    CK(cudaMemsetAsync(s.side_key, 0xff, (size_t)s.side_cap * sizeof(unsigned long long), st));
  EVREC(ctl.eq0);
  CK(launch_query(qa, s.dp, s.prec, st));
  EVREC(ctl.eq1);
  ++ctl.qlaunch;
  ctl.searches += nterm;
  h->launches += 1;
  if (s.cache_slots > 0) {
    k_cache_insert<<<grid_for((int64_t)152 * 8 * TPB, TPB), TPB, 0, st>>>(s);
    CK(cudaMemsetAsync(&s.ctr->nins, 0, sizeof(int32_t), st));
    h->launches += 1;
  }
  // searches that handed big pairs to the whole GPU: evaluate those pairs
  // (results go to the cache), then search again; the last re-run
  // evaluates any remaining big pair itself, so the loop ends
  for (int it = 0; defer; ++it) {
    int cnt[2];
    CK(cudaMemcpyAsync(cnt, &s.ctr->nbreq, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int nreq = std::min(cnt[0], s.breq_cap), npend = cnt[1];
    if (npend == 0) break;
    ++ctl.big_iters;
    ctl.big_reqs += nreq;
    if (ctl.eq0) {
      float q;
      cudaEventElapsedTime(&q, ctl.eq0, ctl.eq1);
      ctl.ms_query += q;
    }
    for (int r0 = 0; r0 < nreq; r0 += BIG_BATCH) {
      const int m = std::min(BIG_BATCH, nreq - r0);
      k_big_dedup<<<1, BIG_BATCH, 0, st>>>(s, r0, m);
      k_big_tiles<<<1, BIG_BATCH, 0, st>>>(s, r0, m);
      EVREC(ctl.eb0);
      rc = launch_big(s, r0, st);
      EVREC(ctl.eb1);
      if (rc) return rc;
      ctl.big_launch += 3;  // kinds 0 and 1 (FP32), FP64
      if (ctl.eb0) {
        CK(cudaEventSynchronize(ctl.eb1));
        float bms;
        cudaEventElapsedTime(&bms, ctl.eb0, ctl.eb1);
        ctl.ms_big += bms;
      }
      k_big_final<<<cdiv(m, 8), 256, 0, st>>>(s, r0, m);
      h->launches += 6;
    }
    CK(cudaMemsetAsync(&s.ctr->nbreq, 0, 2 * sizeof(int32_t), st));
    ctl.searches += npend;
    qa.term = s.pend[it & 1];
    qa.nterm = npend;
    qa.pend_out = s.pend[(it & 1) ^ 1];
    qa.defer = it < 4 ? 1 : 0;
    EVREC(ctl.eq0);
    CK(launch_query(qa, s.dp, s.prec, st));
    EVREC(ctl.eq1);
    ++ctl.qlaunch;
    k_cache_insert<<<grid_for((int64_t)152 * 8 * TPB, TPB), TPB, 0, st>>>(s);
    CK(cudaMemsetAsync(&s.ctr->nins, 0, sizeof(int32_t), st));
    h->launches += 2;
  }
  k_chain<<<grid_for(nterm, TPB), TPB, 0, st>>>(s, nterm);
  h->launches += 2;  // chain, rnn
  EVREC(ctl.e1);
  CK(cudaMemsetAsync(&s.ctr->npairs, 0, sizeof(int32_t), st));
  k_rnn<<<grid_for(nterm, TPB), TPB, 0, st>>>(s, nterm, round);
  CK(cudaGetLastError());
  int npairs = 0;
  CK(cudaMemcpyAsync(&npairs, &s.ctr->npairs, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *npairs_out = npairs;
  if (npairs <= 0) return HAC_EINTERNAL;
  k_merge<<<grid_for(npairs, TPB), TPB, 0, st>>>(s, round, npairs);
  h->launches += 4;  // merge, 3 compaction kernels
  if (s.cache_slots > 0) {
    const int S = s.cache_slots;
    const size_t smem = (size_t)CM_WARPS * 5 * S * sizeof(CEntry);
    const int blocks = std::max(1, std::min(cdiv(npairs, CM_WARPS), 152 * 32));
    // more than the default 48 KB of shared memory per block for large tables
    if (s.linkage == LK_COMPLETE) {
      CK(cudaFuncSetAttribute(k_cache_merge<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
      k_cache_merge<0><<<blocks, CM_WARPS * 32, smem, st>>>(s, npairs, round);
    } else {
      CK(cudaFuncSetAttribute(k_cache_merge<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
      k_cache_merge<1><<<blocks, CM_WARPS * 32, smem, st>>>(s, npairs, round);
    }
    k_gen_bump<<<grid_for(npairs, TPB), TPB, 0, st>>>(s, npairs);
    h->launches += 2;
  }
  EVREC(ctl.e2);
  const int nb = cdiv(K, TPB);
  const int32_t *ord = s.order[h->ocur];
  int32_t *ordn = s.order[h->ocur ^ 1];
  k_cmp_count<<<nb, TPB, 0, st>>>(s, ord, K, round);
  k_cmp_top<<<1, TPB, 0, st>>>(s, nb);
  k_cmp_write<<<nb, TPB, 0, st>>>(s, ord, ordn, need_points ? s.seg[h->pcur ^ 1] : nullptr, K,
                                  round);
  CK(cudaGetLastError());
  h->ocur ^= 1;
  if (need_points) {
    k_relayout<<<grid_for(h->lay_n, TPB), TPB, 0, st>>>(s, h->pcur, h->lay_n);
    h->launches += 1;
    h->pcur ^= 1;
  }
  return HAC_OK;
}

int run_impl(hac_ctx *h, const hac_opts *o) {
  hac_opts opt;
  hac_default_opts(&opt);
  if (o) opt = *o;
  if (opt.precision != HAC_PREC_F64 && opt.precision != HAC_PREC_F32_RECHECK) return HAC_EINVAL;
  if (opt.cache_slots < 0 || opt.max_rounds < 0 || opt.timeout_s < 0) return HAC_EINVAL;
  cudaStream_t st = opt.stream ? (cudaStream_t)opt.stream : h->own;
  State &s = h->s;
  s.prec = opt.precision;
  s.noprune = (opt.flags & HAC_FLAG_NO_PRUNE) ? 1 : 0;
  h->done = false;
  // Section 5 cache tables (complete / average only: Ward distances are O(1))
  const int slots = closed_form(s.linkage) ? 0 : std::min(opt.cache_slots, CACHE_MAX_SLOTS);
  if (slots > h->cache_alloc_slots) {
    int rc0 = 0;
    const size_t cells = (size_t)h->n * slots;
    const int64_t cap = std::max<int64_t>(4 * h->n, 1 << 16);
    if ((rc0 = dalloc(h, &s.ckey, cells)) || (rc0 = dalloc(h, &s.cval, cells)) ||
        (rc0 = dalloc(h, &s.cerr, cells)) || (rc0 = dalloc(h, &s.cpart, cells)) || (rc0 = dalloc(h, &s.ins_i, cap)) ||
        (rc0 = dalloc(h, &s.ins_j, cap)) || (rc0 = dalloc(h, &s.ins_v, cap)) ||
        (rc0 = dalloc(h, &s.ins_e, cap)))
      return rc0;
    s.ins_cap = (int)cap;
    if (!s.breq_i) {  // big-pair deferral buffers (sized once per handle)
      const int bcap = 1 << 18;
      // per request at most max(BIG_MAXT, tiles along the larger cluster)
      const size_t per = (size_t)std::max(BIG_MAXT, cdiv(h->n, BIG_TILE) + 1);
      const size_t tiles = (size_t)BIG_BATCH * per;
      if ((rc0 = dalloc(h, &s.breq_i, bcap)) || (rc0 = dalloc(h, &s.breq_j, bcap)) ||
          (rc0 = dalloc(h, &s.breq_sa, bcap)) || (rc0 = dalloc(h, &s.breq_na, bcap)) ||
          (rc0 = dalloc(h, &s.breq_sb, bcap)) || (rc0 = dalloc(h, &s.breq_nb, bcap)) ||
          (rc0 = dalloc(h, &s.breq_exact, bcap)) || (rc0 = dalloc(h, &s.bsched, BS_SIZE)) ||
          (rc0 = dalloc(h, &s.breq_base, bcap)) || (rc0 = dalloc(h, &s.breq_cov, bcap)) ||
          (rc0 = dalloc(h, &s.breq_berr, bcap)) ||
          (rc0 = dalloc(h, &s.bpart, tiles)) || (rc0 = dalloc(h, &s.pend[0], h->n)) ||
          (rc0 = dalloc(h, &s.pend[1], h->n)) || (rc0 = dalloc(h, &s.side_key, 2 * bcap)) ||
          (rc0 = dalloc(h, &s.side_val, 2 * bcap)) || (rc0 = dalloc(h, &s.side_err, 2 * bcap)))
        return rc0;
      s.breq_cap = bcap;
      s.side_cap = 2 * bcap;
    }
    h->cache_alloc_slots = slots;
  }
  s.cache_slots = slots;
  if (slots > 0)
    CK(cudaMemsetAsync(s.ckey, 0xff, (size_t)h->n * slots * sizeof(unsigned long long), st));
  h->st = hac_stats_t{};
  h->st.device_bytes = h->bytes;
  const auto t0 = std::chrono::steady_clock::now();
  Ev e0, e1, e2, e3, eq0, eq1, eb0, eb1;
  double ms_nn = 0, ms_merge = 0, ms_update = 0, ms_init = 0, ms_query = 0, ms_big = 0;
  int64_t big_launch = 0;
  int64_t qlaunch = 0;
  h->launches = 0;
  cudaEventRecord(e0.e, st);
  int rc = h->dt == HAC_F32 ? init_layout<float>(h, st) : init_layout<double>(h, st);
  if (rc) return rc;
  cudaEventRecord(e1.e, st);
  CK(cudaEventSynchronize(e1.e));
  {
    float ms;
    cudaEventElapsedTime(&ms, e0.e, e1.e);
    ms_init = ms;
  }
  int K = (int)h->n, nterm = (int)h->n, round = 0;
  int64_t naive = 0;  // cluster pairs a search without range queries would test
  Counters c{}, cprev{};
  const char *tr = getenv("HAC_TRACE");
  const bool trace = tr && tr[0] && tr[0] != '0';
  RoundCtl ctl;
  ctl.e1 = e1.e;
  ctl.e2 = e2.e;
  ctl.eq0 = eq0.e;
  ctl.eq1 = eq1.e;
  ctl.eb0 = eb0.e;
  ctl.eb1 = eb1.e;
  while (K > 1) {
    if (opt.max_rounds && round >= opt.max_rounds) return HAC_ETIMEOUT;
    if (opt.timeout_s > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
            opt.timeout_s)
      return HAC_ETIMEOUT;
    cudaEventRecord(e0.e, st);
    const int big_iters0 = ctl.big_iters, big_reqs0 = ctl.big_reqs;
    naive += (int64_t)nterm * (K - 1);
    int npairs = 0;
    rc = round_step(h, st, round, K, nterm, ctl, &npairs);
    if (rc == HAC_EINTERNAL && npairs <= 0) {
      CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (trace) fprintf(stderr, "hac round %d: no reciprocal pair (err %d)\n", round, c.err);
    }
    if (rc) return rc;
    K -= npairs;
    if (K > 1) {
      rc = build_tree(h, s.order[h->ocur], K, st);
      if (rc) return rc;
    }
    cudaEventRecord(e3.e, st);
    CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // the last merge finishes the instance: its single cluster leaves the order
    if ((c.err & ~ERR_NONFINITE) || (c.nactive != K && !(K == 1 && c.nactive == 0))) {
      if (trace)
        fprintf(stderr, "hac round %d: consistency (err %d, active %d, expected %d)\n", round,
                c.err, c.nactive, K);
      return HAC_EINTERNAL;
    }
    if (trace) {
      float qms, nms, mms, ums;
      cudaEventElapsedTime(&qms, eq0.e, eq1.e);
      cudaEventElapsedTime(&nms, e0.e, e1.e);
      cudaEventElapsedTime(&mms, e1.e, e2.e);
      cudaEventElapsedTime(&ums, e2.e, e3.e);
      fprintf(stderr,
              "hac round %d K %d terms %d pairs %d query_ms %.3f leaf_tests %llu nodes %llu "
              "cpairs %llu ppairs %llu rechecks %llu nn_ms %.3f merge_ms %.3f update_ms %.3f "
              "big_iters %d big_reqs %d hits %llu big_pp %llu big_exact %llu\n",
              round, K + npairs, nterm, npairs, qms, c.ltests - cprev.ltests,
              c.nodes - cprev.nodes, c.cluster_pairs - cprev.cluster_pairs,
              c.point_pairs - cprev.point_pairs, c.rechecks - cprev.rechecks, nms, mms, ums,
              ctl.big_iters - big_iters0, ctl.big_reqs - big_reqs0,
              c.cache_hits - cprev.cache_hits, c.big_pp - cprev.big_pp,
              c.big_exact - cprev.big_exact);
      cprev = c;
    }
    nterm = c.nterm;
    {
      float a, b, d3;
      cudaEventElapsedTime(&a, e0.e, e1.e);
      cudaEventElapsedTime(&b, e1.e, e2.e);
      cudaEventElapsedTime(&d3, e2.e, e3.e);
      float q;
      cudaEventElapsedTime(&q, eq0.e, eq1.e);
      ctl.ms_query += q;
      ms_nn += a;
      ms_merge += b;
      ms_update += d3;
    }
    ++round;
  }
  ms_query = ctl.ms_query;
  ms_big = ctl.ms_big;
  qlaunch = ctl.qlaunch;
  big_launch = ctl.big_launch;
  h->st.nn_searches = ctl.searches;
  h->st.naive_pairs = naive;
  CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int64_t m = h->n - 1;
  if (c.nmerges != m) return HAC_EINTERNAL;
  // canonical order on the device: (height, size, cid_a); (cid_a, size)
  // already identifies a merge, so the order is total
  if (m > 0) {
    const int mm = (int)m;
    const int g = grid_for(mm, TPB);
    int32_t *perm = nullptr;
    const int fbits[3] = {bits_for(h->n), bits_for(h->n), 64};
    for (int f = 0; f < 3; ++f) {
      k_rec_key<<<g, TPB, 0, st>>>(s, mm, f, perm, h->keys[0], h->vals[0]);
      const int r = radix_sort(h, mm, fbits[f], st);
      if (r < 0) return r;
      if (r == 1) {
        CK(cudaMemcpyAsync(h->vals[0], h->vals[1], (size_t)mm * 4, cudaMemcpyDeviceToDevice, st));
      }
      perm = h->vals[0];
    }
    k_rec_gather<<<g, TPB, 0, st>>>(s, mm, perm, h->dout, h->dout_round);
    h->launches += 4;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
  }
  h->n_merges = m;
  h->st.rounds = round;
  h->st.merges = c.nmerges;
  h->st.cluster_pairs = (int64_t)c.cluster_pairs;
  h->st.point_pairs = (int64_t)(c.point_pairs + c.big_pp);
  h->st.nodes_visited = (int64_t)c.nodes;
  h->st.rechecks = (int64_t)c.rechecks;
  h->st.ms_init = ms_init;
  h->st.ms_query = ms_query;
  h->st.query_launches = qlaunch;
  h->st.leaf_tests = (int64_t)c.ltests;
  h->st.kernel_launches = h->launches;
  h->st.cache_hits = (int64_t)c.cache_hits;
  h->st.ms_big = ms_big;
  h->st.big_point_pairs = (int64_t)c.big_pp;
  h->st.big_launches = big_launch;
  h->st.cache_lw_entries = (int64_t)c.cache_lw;
  {
    // algorithmic bytes of the search kernel (true dimension d, not padded):
    // node test = centroid box (+ complete's hi-min / lo-max) + min size;
    // leaf slot = order entry + FP32 centroid + size (+ complete's box);
    // evaluated pair = Ward FP64 centroid, or the point rows of both clusters;
    // per terminal = its own centroid, box, size and pred word.
    const int64_t d = h->d;
    const int64_t ew = 8;  // FP64 path
    const bool comp = s.linkage == LK_COMPLETE;
    const int64_t node_b = 2 * d * 4 + 4 + (comp ? 2 * d * 4 : 0);
    const int64_t leaf_b = 4 + d * 4 + 4 + (comp ? 2 * d * 4 : 0);
    const int64_t term_b = d * 4 + 2 * d * 4 + 4 + 8 + 4 + 16;
    int64_t qb = (int64_t)c.nodes * node_b + (int64_t)c.ltests * leaf_b +
                 h->st.nn_searches * term_b;
    if (closed_form(s.linkage))
      qb += (int64_t)c.cluster_pairs * d * ew;
    else
      qb += (int64_t)c.prows * d * ew;
    h->st.query_bytes = qb;
  }
  h->st.ms_nn = ms_nn;
  h->st.ms_merge = ms_merge;
  h->st.ms_update = ms_update;
  h->st.ms_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->done = true;
  return HAC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void hac_default_opts(hac_opts *o) {
  if (!o) return;
  o->precision = HAC_PREC_F64;
  o->cache_slots = 0;
  o->max_rounds = 0;
  o->timeout_s = 0.0;
  o->stream = nullptr;
  o->flags = 0;
}

int hac_create(const void *points, int64_t n, int d, hac_dtype dt, hac_linkage lk, hac_t *out) {
  return create_common(points, false, n, d, dt, lk, out);
}

int hac_create_device(const void *dev_points, int64_t n, int d, hac_dtype dt, hac_linkage lk,
                      hac_t *out) {
  return create_common(dev_points, true, n, d, dt, lk, out);
}

int hac_run(hac_t h, const hac_opts *opts) {
  if (!h) return HAC_EINVAL;
  int rc = run_impl(h, opts);
  if (rc == HAC_EDEVICE) cudaGetLastError();
  return rc;
}

int hac_dendrogram(hac_t h, hac_merge *out, int64_t cap, int64_t *n_written) {
  if (!h || !n_written || (!out && h->n > 1)) return HAC_EINVAL;
  if (!h->done) return HAC_EPENDING;
  if (cap < h->n_merges) return HAC_ECAP;
  if (h->n_merges &&
      cudaMemcpy(out, h->dout, h->n_merges * sizeof(hac_merge), cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
    cudaGetLastError();
    return HAC_EDEVICE;
  }
  *n_written = h->n_merges;
  return HAC_OK;
}

int hac_merge_rounds(hac_t h, int32_t *out, int64_t cap, int64_t *n_written) {
  if (!h || !n_written || (!out && h->n > 1)) return HAC_EINVAL;
  if (!h->done) return HAC_EPENDING;
  if (cap < h->n_merges) return HAC_ECAP;
  if (h->n_merges &&
      cudaMemcpy(out, h->dout_round, h->n_merges * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
    cudaGetLastError();
    return HAC_EDEVICE;
  }
  *n_written = h->n_merges;
  return HAC_OK;
}

int hac_stats(hac_t h, hac_stats_t *out) {
  if (!h || !out) return HAC_EINVAL;
  *out = h->st;
  return HAC_OK;
}

void hac_destroy(hac_t h) {
  if (!h) return;
  free_all(h);
  delete h;
}

const char *hac_strerror(int code) {
  switch (code) {
    case HAC_OK: return "ok";
    case HAC_EINVAL: return "invalid argument";
    case HAC_ENOMEM: return "out of memory";
    case HAC_EDEVICE: return "CUDA device error";
    case HAC_ETIMEOUT: return "round or time limit reached";
    case HAC_EPENDING: return "no completed run";
    case HAC_ECAP: return "output buffer too small";
    case HAC_EINTERNAL: return "internal consistency check failed";
    case HAC_ECANCELED: return "request cancelled";
  }
  return "unknown status";
}

}  // extern "C"

// ---------------------------------------------------------------------------
// hac_run_static: a whole clustering that allocates nothing
//
// Some callers cannot call cudaMalloc at the moment they need a clustering:
// a serving process whose memory pool has already claimed every byte of the
// GPU, or latency-sensitive code that must not hit cudaMalloc/cudaFree (which
// can synchronise the whole device).  This entry point runs the same kernels
// as hac_create/hac_run/hac_dendrogram, but every piece of working memory is
// carved out of one file-scope device array that the library owns for as
// long as it is loaded (kStaticArenaBytes on every GPU that loads it).  The
// caller passes the device input points and a device output buffer.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticArenaBytes = (size_t)6 << 20;  // 6 MiB: room for n <= HAC_STATIC_MAX_N
static __device__ __align__(256) unsigned char g_static_arena[kStaticArenaBytes];

constexpr int kStaticMaxDevices = 64;
std::atomic<unsigned char *> g_static_ptr[kStaticMaxDevices];  // per device, set on first use

// Device address of the arena on the current device.  Host code must not
// use the symbol g_static_arena itself: on the host it only names a stand-in.
int static_arena(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HAC_EDEVICE;
  }
  if (dev < 0 || dev >= kStaticMaxDevices) return HAC_EDEVICE;
  unsigned char *p = g_static_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    void *q = nullptr;
    if (cudaGetSymbolAddress(&q, g_static_arena) != cudaSuccess || q == nullptr) {
      cudaGetLastError();
      return HAC_EDEVICE;
    }
    p = (unsigned char *)q;
    g_static_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return HAC_OK;
}

// bump allocator over the arena (256-byte aligned pieces)
struct Carver {
  unsigned char *base;
  size_t off, cap;
  bool ok;
  template <typename T>
  void take(T **p, size_t count) {
    off = (off + 255) & ~(size_t)255;
    *p = (T *)(base + off);
    off += (count ? count : 1) * sizeof(T);
    if (off > cap) ok = false;
  }
};

// the same arrays as alloc_state, carved instead of allocated
bool carve_state(hac_ctx &h, Carver &cv) {
  State &s = h.s;
  const int64_t n = h.n;
  const int dp = s.dp;
  for (int b = 0; b < 2; ++b) {
    cv.take(&s.p64[b], n * dp);
    cv.take(&s.p32[b], n * dp);
    cv.take(&s.plab[b], n);
    cv.take(&s.seg[b], n);
    cv.take(&s.order[b], n);
  }
  cv.take(&s.csize, n);
  cv.take(&s.q32, n * dp);
  cv.take(&s.q64, n * dp);
  cv.take(&s.qblo, n * dp);
  cv.take(&s.qbhi, n * dp);
  cv.take(&s.qsz, n);
  cv.take(&s.qseg, n);
  cv.take(&s.csum, n * dp);
  cv.take(&s.csq, n);
  cv.take(&s.sse, n);
  cv.take(&s.qvar, n);
  cv.take(&s.cent, n * dp);
  cv.take(&s.cent32, n * dp);
  cv.take(&s.blo, n * dp);
  cv.take(&s.bhi, n * dp);
  cv.take(&s.succ, n);
  cv.take(&s.pred, n);
  cv.take(&s.mround, n);
  cv.take(&s.isterm, n);
  cv.take(&s.alive, n);
  cv.take(&s.rootof, n);
  cv.take(&s.reloff, n);
  cv.take(&s.osize, n);
  cv.take(&s.partner, n);
  cv.take(&s.gen, n);
  cv.take(&s.inst, n);
  cv.take(&s.qinst, n);
  s.max_inst = 1;
  cv.take(&s.islack, 1);
  cv.take(&s.iscale, 1);
  cv.take(&s.idpts, 1);
  cv.take(&s.iseq, 1);
  cv.take(&s.done_list, 2);
  cv.take(&s.irec, 1);
  cv.take(&s.irecn, 1);
  cv.take(&s.iact, 1);
  cv.take(&s.idone, 1);
  cv.take(&s.pos, n);
  cv.take(&s.Ekey, n);
  cv.take(&s.Ecid, n);
  cv.take(&s.term, n);
  cv.take(&s.pair_lo, n / 2 + 1);
  cv.take(&s.pair_hi, n / 2 + 1);
  cv.take(&s.pair_key, n / 2 + 1);
  cv.take(&s.m_a, n);
  cv.take(&s.m_b, n);
  cv.take(&s.m_size, n);
  cv.take(&s.m_round, n);
  cv.take(&s.m_h, n);
  int base = 0;
  const int nlev = tree_levels((int)n);
  for (int L = 0; L <= MAXLEV; ++L) {
    s.lvl_base[L] = base;
    if (L < nlev) base += level_count((int)n, L);
  }
  h.nlev_max = nlev;
  cv.take(&s.nclo, (size_t)base * dp);
  cv.take(&s.nchi, (size_t)base * dp);
  cv.take(&s.nhmin, (size_t)base * dp);
  cv.take(&s.nlmax, (size_t)base * dp);
  cv.take(&s.nnmin, (size_t)base);
  cv.take(&s.ninlo, (size_t)base);
  cv.take(&s.ninhi, (size_t)base);
  cv.take(&s.bsum, 3 * (size_t)cdiv(n, TPB) + 3);
  cv.take(&s.ctr, 1);
  for (int b = 0; b < 2; ++b) {
    cv.take(&h.keys[b], n);
    cv.take(&h.vals[b], n);
  }
  const int ntiles = cdiv(n, RS_TILE);
  cv.take(&h.hist, (size_t)256 * ntiles + 1);
  cv.take(&h.hbs, (size_t)cdiv((int64_t)256 * ntiles, SC_TILE) + 1);
  cv.take(&h.bb, 2 * MAXD);
  cv.take(&h.dout_round, n);
  return cv.ok;
}

// initial layout with stack buffers only (no host or device allocation)
template <typename T>
int static_layout(hac_ctx &h, cudaStream_t st) {
  State &s = h.s;
  const T *X = (const T *)h.raw;
  const int64_t n = h.n;
  const int d = h.d;
  unsigned long long bb[2 * MAXD];
  for (int k = 0; k < MAXD; ++k) {
    bb[k] = ~0ull;
    bb[MAXD + k] = 0ull;
  }
  CK(cudaMemcpyAsync(h.bb, bb, sizeof(bb), cudaMemcpyHostToDevice, st));
  // the arena keeps the previous call's contents: counters start from zero
  CK(cudaMemsetAsync(s.ctr, 0, sizeof(Counters), st));
  k_bbox<T><<<grid_for(n, TPB), TPB, 0, st>>>(X, n, d, h.bb, h.bb + MAXD, s.ctr);
  CK(cudaGetLastError());
  Counters c0;
  CK(cudaMemcpyAsync(bb, h.bb, sizeof(bb), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&c0, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (c0.err & ERR_NONFINITE) return HAC_EINVAL;
  MortonParams mp{}, ctrp{};
  double scale = 0.0;
  for (int k = 0; k < d; ++k) {
    unsigned long long u = bb[k], v = bb[MAXD + k];
    u = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
    v = (v >> 63) ? (v & 0x7fffffffffffffffull) : ~v;
    double lo, hi;
    memcpy(&lo, &u, 8);
    memcpy(&hi, &v, 8);
    mp.lo[k] = lo;
    mp.inv[k] = hi > lo ? 1.0 / (hi - lo) : 0.0;
    ctrp.lo[k] = 0.5 * (lo + hi);
    scale = std::max(scale, std::max(std::fabs(lo - ctrp.lo[k]), std::fabs(hi - ctrp.lo[k])));
  }
  mp.bits = std::min(21, 64 / d);
  s.abs_slack = std::max(scale, 1e-300) * std::ldexp(1.0, -18);
  s.coord_scale = (float)(scale * (1.0 + 1e-6));
  s.delta_pts = s.pts32_exact ? 0.f : 2.01f * 5.9604645e-8f * s.coord_scale * std::sqrt((float)d);
  k_inst_set<<<1, 1, 0, st>>>(s, 0, (float)s.abs_slack, s.coord_scale, s.delta_pts, 0, (int)n, 0);
  k_morton<T><<<grid_for(n, TPB), TPB, 0, st>>>(X, n, d, mp, h.keys[0], h.vals[0]);
  CK(cudaGetLastError());
  const int sc = radix_sort(&h, (int)n, mp.bits * d, st);
  if (sc < 0) return sc;
  h.ocur = h.pcur = 0;
  h.lay_n = n;
  s.cur = 0;
  k_layout<T><<<grid_for(n, TPB), TPB, 0, st>>>(s, X, h.vals[sc], ctrp);
  CK(cudaGetLastError());
  Counters c{};
  c.nterm = (int)n;
  c.nactive = (int)n;
  CK(cudaMemcpyAsync(s.ctr, &c, sizeof(Counters), cudaMemcpyHostToDevice, st));
  return build_tree(&h, s.order[0], (int)n, st);
}

// Algorithm 1 rounds with the state carved from the arena; writes the
// canonical dendrogram to `dev_out`
int static_run(hac_ctx &h, const hac_opts &opt, cudaStream_t st, hac_merge *dev_out) {
  State &s = h.s;
  int rc = h.dt == HAC_F32 ? static_layout<float>(h, st) : static_layout<double>(h, st);
  if (rc) return rc;
  const auto t0 = std::chrono::steady_clock::now();
  int K = (int)h.n, nterm = (int)h.n, round = 0;
  Counters c{};
  RoundCtl ctl;  // no events: nothing is created here
  while (K > 1) {
    if (opt.max_rounds && round >= opt.max_rounds) return HAC_ETIMEOUT;
    if (opt.timeout_s > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
            opt.timeout_s)
      return HAC_ETIMEOUT;
    int npairs = 0;
    rc = round_step(&h, st, round, K, nterm, ctl, &npairs);
    if (rc) return rc;
    K -= npairs;
    if (K > 1) {
      rc = build_tree(&h, s.order[h.ocur], K, st);
      if (rc) return rc;
    }
    CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if ((c.err & ~ERR_NONFINITE) || (c.nactive != K && !(K == 1 && c.nactive == 0)))
      return HAC_EINTERNAL;
    nterm = c.nterm;
    ++round;
  }
  CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int64_t m = h.n - 1;
  if (c.nmerges != m && m > 0) return HAC_EINTERNAL;
  if (m > 0) {
    const int mm = (int)m;
    const int g = grid_for(mm, TPB);
    int32_t *perm = nullptr;
    const int fbits[3] = {bits_for(h.n), bits_for(h.n), 64};
    for (int f = 0; f < 3; ++f) {
      k_rec_key<<<g, TPB, 0, st>>>(s, mm, f, perm, h.keys[0], h.vals[0]);
      const int r = radix_sort(&h, mm, fbits[f], st);
      if (r < 0) return r;
      if (r == 1)
        CK(cudaMemcpyAsync(h.vals[0], h.vals[1], (size_t)mm * 4, cudaMemcpyDeviceToDevice, st));
      perm = h.vals[0];
    }
    k_rec_gather<<<g, TPB, 0, st>>>(s, mm, perm, dev_out, h.dout_round);
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(st));
  return HAC_OK;
}

}  // namespace

extern "C" int hac_run_static(const void *dev_points, int64_t n, int d, hac_dtype dt,
                              hac_linkage lk, const hac_opts *opts, hac_merge *dev_out,
                              int64_t cap) {
  if (!dev_points || !dev_out || n < 1 || n > HAC_STATIC_MAX_N || d < 1 || d > MAXD)
    return HAC_EINVAL;
  if (dt != HAC_F32 && dt != HAC_F64) return HAC_EINVAL;
  if (lk != HAC_COMPLETE && lk != HAC_AVERAGE && lk != HAC_WARD && lk != HAC_AVERAGE_SQ)
    return HAC_EINVAL;
  if (cap < n - 1) return HAC_ECAP;
  hac_opts opt;
  hac_default_opts(&opt);
  if (opts) opt = *opts;
  if (opt.precision != HAC_PREC_F64 && opt.precision != HAC_PREC_F32_RECHECK) return HAC_EINVAL;
  if (opt.cache_slots < 0 || opt.max_rounds < 0 || opt.timeout_s < 0) return HAC_EINVAL;
  unsigned char *arena = nullptr;
  int rc = static_arena(&arena);
  if (rc) return rc;
  hac_ctx h;  // on the stack; its pointers all point into the arena
  h.n = n;
  h.d = d;
  h.dt = dt;
  h.lk = lk;
  h.raw = const_cast<void *>(dev_points);
  h.s.n = n;
  h.s.d = d;
  h.s.dp = pad_dim(d);
  h.s.linkage = (int)lk;
  h.s.pts32_exact = dt == HAC_F32;
  h.s.prec = opt.precision;
  Carver cv{arena, 0, kStaticArenaBytes, true};
  if (!carve_state(h, cv)) return HAC_EINVAL;
  const cudaStream_t st = (cudaStream_t)opt.stream;
  rc = static_run(h, opt, st, dev_out);
  if (rc == HAC_EDEVICE) cudaGetLastError();
  return rc;
}

// ---------------------------------------------------------------------------
// Serving: continuous batching of independent clusterings
//
// An engine is one device state of `cap` points shared by every in-flight
// request with the same linkage, dimension and input type.  Cluster ids are
// global slots: a request admitted into the free id range [base, base + n)
// keeps cid = base + smallest local index, so its merges are those of a lone
// run shifted by base.  Each round is one launch per kernel for all resident
// requests, and searches never leave their own request.  Between rounds,
// finished requests leave (their ids and points are freed) and queued ones
// that fit are admitted, so a request that arrives while others run joins
// at the next round.  Engines of different kinds run on their own host
// threads and streams, so their rounds overlap on the device.
// ---------------------------------------------------------------------------
namespace {

constexpr int SRV_MAX_INST = 4096;   // resident requests per engine
constexpr int SRV_ADMIT_MAX = 1024;  // requests admitted between two rounds

struct AdmitInst {
  int base, n, off, slot, seq, bits;
  float slack, scale, dpts;               // the instance's pruning and error parameters
  double lo[MAXD], inv[MAXD], ctr[MAXD];  // Morton box and recentring offset
};

// parameters and progress counters of every admitted instance
__global__ void k_admit_inst(State s, const AdmitInst *ai, int na) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < na; t += gridDim.x * blockDim.x) {
    const AdmitInst &a = ai[t];
    s.iseq[a.slot] = a.seq;
    s.islack[a.slot] = a.slack;
    s.iscale[a.slot] = a.scale;
    s.idpts[a.slot] = a.dpts;
    s.irec[a.slot] = a.base;
    s.irecn[a.slot] = 0;
    s.iact[a.slot] = a.n;
    s.idone[a.slot] = a.n <= 1;
  }
}

// merge records of the instances that finished, packed for one copy to the
// host: record j of instance t goes to dst[off[t] + j] with local cids
struct RecOut {
  int32_t a, b, size, round;
  double h;
};

__global__ void k_rec_pack(State s, const int4 *fin, int nf, int total, RecOut *dst) {
  // fin[t] = (base, records, offset, admission round)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int lo = 0, hi = nf;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (fin[mid].z <= i) lo = mid;
      else hi = mid;
    }
    const int4 f = fin[lo];
    const int m = f.x + (i - f.z);
    dst[i] = RecOut{s.m_a[m] - f.x, s.m_b[m] - f.x, s.m_size[m], s.m_round[m] - f.w, s.m_h[m]};
  }
}

__device__ __forceinline__ int admit_find(const AdmitInst *ai, int na, int i) {
  int lo = 0, hi = na;  // last instance with off <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ai[mid].off <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Morton key of every staged point under its request's own box, with the
// request's rank in the batch above it: the sort groups each request
template <typename T>
__global__ void k_admit_keys(const T *stage, int m, int d, const AdmitInst *ai, int na,
                             uint64_t *keys, int32_t *vals) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int t = admit_find(ai, na, i);
    const AdmitInst &a = ai[t];
    const double top = (double)((1u << a.bits) - 1u);
    uint32_t q[MAXD];
    for (int k = 0; k < d; ++k) {
      const double u = ((double)stage[(size_t)i * d + k] - a.lo[k]) * a.inv[k];
      q[k] = (uint32_t)(fmin(fmax(u, 0.0), 1.0) * top);
    }
    uint64_t code = 0;
    for (int b = a.bits - 1; b >= 0; --b)
      for (int k = 0; k < d; ++k) code = (code << 1) | ((q[k] >> b) & 1u);
    keys[i] = ((uint64_t)t << 40) | code;
    vals[i] = i;
  }
}

// initial state of every admitted point (a singleton cluster), appended
// behind the K active clusters in `order`, the nterm terminals and the P
// points of the layout.  Ward never reads points after this, so there each
// point sits at its cid's slot instead (pts_at_cid).
template <typename T>
__global__ void k_admit_layout(State s, const T *stage, int m, const AdmitInst *ai, int na,
                               const int32_t *sorted, int32_t *order, int K, int nterm,
                               int64_t P, int pc, int round, int pts_at_cid) {
  const int d = s.d, dp = s.dp;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < m; p += gridDim.x * blockDim.x) {
    const int i = sorted[p];
    const AdmitInst &a = ai[admit_find(ai, na, i)];
    const int c = a.base + (i - a.off);
    const int64_t pp = pts_at_cid ? (int64_t)c : P + p;
    const int op = K + p;
    for (int k = 0; k < dp; ++k) {
      const double raw = k < d ? (double)stage[(size_t)i * d + k] : 0.0;
      const double x = k < d ? raw - a.ctr[k] : 0.0;
      s.p64[pc][pp * dp + k] = x;
      s.p32[pc][pp * dp + k] = s.pts32_exact ? (float)raw : (float)x;
      s.csum[(size_t)c * dp + k] = x;
      s.cent[(size_t)c * dp + k] = x;
      s.cent32[(size_t)c * dp + k] = (float)x;
      s.blo[(size_t)c * dp + k] = __double2float_rd(x);
      s.bhi[(size_t)c * dp + k] = __double2float_ru(x);
      s.q32[(size_t)op * dp + k] = (float)x;
      s.q64[(size_t)op * dp + k] = x;
      s.qblo[(size_t)op * dp + k] = __double2float_rd(x);
      s.qbhi[(size_t)op * dp + k] = __double2float_ru(x);
    }
    double sq = 0.0;
    for (int k = 0; k < d; ++k) {
      const double x = (double)stage[(size_t)i * d + k] - a.ctr[k];
      sq += x * x;
    }
    s.csq[c] = sq;
    s.sse[c] = 0.0;
    s.qvar[op] = 0.f;
    s.plab[pc][pp] = c;
    s.seg[pc][c] = (int32_t)pp;
    s.csize[c] = 1;
    s.succ[c] = -1;
    s.pred[c] = PRED_EMPTY;
    s.mround[c] = -1;
    s.isterm[c] = round;
    s.alive[c] = 1;
    s.rootof[c] = c;
    s.reloff[c] = 0;
    s.gen[c] = 0;
    s.inst[c] = a.slot;
    order[op] = c;
    s.pos[c] = op;
    s.term[nterm + p] = c;
    s.qsz[op] = 1;
    s.qseg[op] = (int32_t)pp;
    s.qinst[op] = a.seq;
    for (int q = 0; q < s.cache_slots; ++q) s.ckey[(size_t)c * s.cache_slots + q] = CKEY_EMPTY;
  }
}

// a request leaves before it is finished (cancelled or past its deadline):
// the next compaction drops its clusters and points
__global__ void k_inst_drop(State s, int slot) { s.idone[slot] = 1; }

struct SrvReq {
  uint64_t ticket = 0;
  std::vector<unsigned char> pts;
  int64_t n = 0;
  int d = 0;
  hac_dtype dt = HAC_F32;
  hac_linkage lk = HAC_WARD;
  std::chrono::steady_clock::time_point t_submit, t_done, deadline;
  bool has_deadline = false;
  bool cancel = false;     // hac_cancel asked for it
  bool dropped = false;    // its instance was told to leave
  int status = HAC_EPENDING;
  std::vector<hac_merge> out;
  std::vector<int32_t> out_round;  // round of each merge (want_rounds only)
  bool want_rounds = false;
  int round0 = 0;                  // engine round at admission
  int slot = -1, base = -1;
  struct Engine *eng = nullptr;
};

struct Engine {
  hac_ctx h;
  int cap = 0;
  std::vector<std::pair<int, int>> free_ranges;  // free cid ranges (start, length), by start
  std::vector<int> free_slots;
  std::vector<SrvReq *> active;                  // resident request of each slot
  std::deque<SrvReq *> queue;
  int K = 0, nterm = 0, round = 0, nres = 0, seq_next = 0;
  int64_t P = 0;                                 // points in the layout (not Ward)
  unsigned char *stage = nullptr;                // admitted points, staged on the device
  unsigned char *h_stage = nullptr;              // ... and in pinned host memory
  RecOut *d_rec = nullptr, *h_rec = nullptr;     // packed records of finished instances
  int4 *d_fin = nullptr;
  std::vector<int4> h_fin;
  std::vector<int32_t> h_list;
  AdmitInst *d_ai = nullptr;
  std::vector<AdmitInst> h_ai;
  std::vector<int32_t> h_done;
  std::thread thr;
  int64_t rounds = 0, admitted = 0, completed = 0;
  int max_res = 0;
  double ms_admit = 0, ms_rounds = 0, ms_harvest = 0;
};

}  // namespace

struct hac_server {
  std::mutex mu;
  std::condition_variable cv;       // engines wait here for work
  std::condition_variable done_cv;  // hac_server_wait waits here
  std::map<uint64_t, SrvReq *> reqs;
  std::map<int, Engine *> engines;
  uint64_t next_ticket = 1;
  bool stop = false;
  int64_t cap = 0;
  hac_opts opt{};
  int device = 0;
  int err = HAC_OK;  // first failure of any engine (sticky)
};

namespace {

bool range_take(Engine &e, int n, int *base) {  // first fit
  for (size_t i = 0; i < e.free_ranges.size(); ++i) {
    auto &r = e.free_ranges[i];
    if (r.second >= n) {
      *base = r.first;
      r.first += n;
      r.second -= n;
      if (r.second == 0) e.free_ranges.erase(e.free_ranges.begin() + i);
      return true;
    }
  }
  return false;
}

void range_give(Engine &e, int base, int n) {  // insert and coalesce
  size_t i = 0;
  while (i < e.free_ranges.size() && e.free_ranges[i].first < base) ++i;
  e.free_ranges.insert(e.free_ranges.begin() + i, {base, n});
  if (i + 1 < e.free_ranges.size() &&
      e.free_ranges[i].first + e.free_ranges[i].second == e.free_ranges[i + 1].first) {
    e.free_ranges[i].second += e.free_ranges[i + 1].second;
    e.free_ranges.erase(e.free_ranges.begin() + i + 1);
  }
  if (i > 0 && e.free_ranges[i - 1].first + e.free_ranges[i - 1].second ==
                   e.free_ranges[i].first) {
    e.free_ranges[i - 1].second += e.free_ranges[i].second;
    e.free_ranges.erase(e.free_ranges.begin() + i);
  }
}

int engine_init(Engine &e, hac_linkage lk, int d, hac_dtype dt, int64_t cap, const hac_opts &opt) {
  hac_ctx &h = e.h;
  h.n = cap;
  h.d = d;
  h.dt = dt;
  h.lk = lk;
  State &s = h.s;
  s.n = cap;
  s.d = d;
  s.dp = pad_dim(d);
  s.linkage = (int)lk;
  s.prec = opt.precision;
  s.pts32_exact = dt == HAC_F32;
  s.max_inst = SRV_MAX_INST;
  if (const char *v = getenv("HAC_BIG_PAIRS")) h.big_pairs = std::max(1ll, atoll(v));
  if (const char *v = getenv("HAC_BIG_PAIRS_F64")) h.big_pairs64 = std::max(1ll, atoll(v));
  if (const char *v = getenv("HAC_WARP_BUDGET")) h.warp_budget = std::max(1ll, atoll(v));
  if (cudaStreamCreateWithFlags(&h.own, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return HAC_EDEVICE;
  }
  int rc = alloc_state(&h);
  if (rc) return rc;
  const size_t esz = dt == HAC_F32 ? 4 : 8;
  if ((rc = dalloc(&h, &e.stage, (size_t)cap * d * esz)) ||
      (rc = dalloc(&h, &e.d_ai, (size_t)SRV_ADMIT_MAX)) ||
      (rc = dalloc(&h, &e.d_rec, (size_t)cap)) || (rc = dalloc(&h, &e.d_fin, 2 * SRV_MAX_INST)))
    return rc;
  if (cudaMallocHost(&e.h_stage, (size_t)cap * d * esz) != cudaSuccess ||
      cudaMallocHost(&e.h_rec, (size_t)cap * sizeof(RecOut)) != cudaSuccess) {
    cudaGetLastError();
    return HAC_ENOMEM;
  }
  // Section 5 cache and the big-pair buffers, as hac_run allocates them
  const int slots = closed_form((int)lk) ? 0 : std::min(opt.cache_slots, CACHE_MAX_SLOTS);
  if (slots > 0) {
    const size_t cells = (size_t)cap * slots;
    const int64_t icap = std::max<int64_t>(4 * cap, 1 << 16);
    const int bcap = 1 << 18;
    const size_t per = (size_t)std::max(BIG_MAXT, cdiv(cap, BIG_TILE) + 1);
    if ((rc = dalloc(&h, &s.ckey, cells)) || (rc = dalloc(&h, &s.cval, cells)) ||
        (rc = dalloc(&h, &s.cerr, cells)) || (rc = dalloc(&h, &s.cpart, cells)) ||
        (rc = dalloc(&h, &s.breq_base, bcap)) || (rc = dalloc(&h, &s.breq_cov, bcap)) ||
        (rc = dalloc(&h, &s.breq_berr, bcap)) || (rc = dalloc(&h, &s.ins_i, icap)) ||
        (rc = dalloc(&h, &s.ins_j, icap)) || (rc = dalloc(&h, &s.ins_v, icap)) ||
        (rc = dalloc(&h, &s.ins_e, icap)) || (rc = dalloc(&h, &s.breq_i, bcap)) ||
        (rc = dalloc(&h, &s.breq_j, bcap)) || (rc = dalloc(&h, &s.breq_sa, bcap)) ||
        (rc = dalloc(&h, &s.breq_na, bcap)) || (rc = dalloc(&h, &s.breq_sb, bcap)) ||
        (rc = dalloc(&h, &s.breq_nb, bcap)) || (rc = dalloc(&h, &s.breq_exact, bcap)) ||
        (rc = dalloc(&h, &s.bsched, BS_SIZE)) ||
        (rc = dalloc(&h, &s.bpart, (size_t)BIG_BATCH * per)) ||
        (rc = dalloc(&h, &s.pend[0], cap)) || (rc = dalloc(&h, &s.pend[1], cap)) ||
        (rc = dalloc(&h, &s.side_key, 2 * bcap)) || (rc = dalloc(&h, &s.side_val, 2 * bcap)) ||
        (rc = dalloc(&h, &s.side_err, 2 * bcap)))
      return rc;
    s.ins_cap = (int)icap;
    s.breq_cap = bcap;
    s.side_cap = 2 * bcap;
    h.cache_alloc_slots = slots;
  }
  s.cache_slots = slots;
  const cudaStream_t st = h.own;
  CK(cudaMemsetAsync(s.ctr, 0, sizeof(Counters), st));
  CK(cudaMemsetAsync(s.idone, 0, (size_t)SRV_MAX_INST * sizeof(int32_t), st));
  CK(cudaStreamSynchronize(st));
  e.cap = (int)cap;
  e.free_ranges = {{0, (int)cap}};
  for (int i = SRV_MAX_INST - 1; i >= 0; --i) e.free_slots.push_back(i);
  e.active.assign(SRV_MAX_INST, nullptr);
  e.h_done.assign(SRV_MAX_INST, 0);
  h.ocur = h.pcur = 0;
  h.lay_n = 0;
  return HAC_OK;
}

// Copy the batch's points in (one copy through pinned memory), give each
// request its parameters, and lay its points out behind the resident
// clusters.  The batch's ids and slots were taken under the server lock.
int engine_admit(Engine &e, const std::vector<SrvReq *> &batch) {
  if (batch.empty()) return HAC_OK;
  hac_ctx &h = e.h;
  State &s = h.s;
  const cudaStream_t st = h.own;
  const int d = s.d;
  const bool f32 = h.dt == HAC_F32;
  const size_t esz = f32 ? 4 : 8;
  if (e.K == 0) e.seq_next = 0;  // idle engine: admission numbers restart
  e.h_ai.resize(batch.size());
  int m = 0;
  for (size_t t = 0; t < batch.size(); ++t) {
    SrvReq *r = batch[t];
    AdmitInst &a = e.h_ai[t];
    a.base = r->base;
    a.n = (int)r->n;
    a.off = m;
    a.slot = r->slot;
    a.seq = e.seq_next++;
    a.bits = std::min(21, 40 / d);
    // the request's box, centre and error parameters, as for a lone run
    double lo[MAXD], hi[MAXD];
    for (int k = 0; k < d; ++k) {
      lo[k] = INFINITY;
      hi[k] = -INFINITY;
    }
    for (int64_t i = 0; i < r->n; ++i)
      for (int k = 0; k < d; ++k) {
        const double x = f32 ? (double)((const float *)r->pts.data())[i * d + k]
                             : ((const double *)r->pts.data())[i * d + k];
        lo[k] = std::min(lo[k], x);
        hi[k] = std::max(hi[k], x);
      }
    double scale = 0.0;
    for (int k = 0; k < MAXD; ++k) {
      a.lo[k] = k < d ? lo[k] : 0.0;
      a.inv[k] = k < d && hi[k] > lo[k] ? 1.0 / (hi[k] - lo[k]) : 0.0;
      a.ctr[k] = k < d ? 0.5 * (lo[k] + hi[k]) : 0.0;
      if (k < d)
        scale = std::max(scale, std::max(std::fabs(lo[k] - a.ctr[k]), std::fabs(hi[k] - a.ctr[k])));
    }
    a.slack = (float)(std::max(scale, 1e-300) * std::ldexp(1.0, -18));
    a.scale = (float)(scale * (1.0 + 1e-6));
    a.dpts = f32 ? 0.f : 2.01f * 5.9604645e-8f * a.scale * std::sqrt((float)d);
    memcpy(e.h_stage + (size_t)m * d * esz, r->pts.data(), (size_t)r->n * d * esz);
    m += (int)r->n;
  }
  const int na = (int)batch.size();
  CK(cudaMemcpyAsync(e.stage, e.h_stage, (size_t)m * d * esz, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(e.d_ai, e.h_ai.data(), na * sizeof(AdmitInst), cudaMemcpyHostToDevice, st));
  k_admit_inst<<<grid_for(na, TPB), TPB, 0, st>>>(s, e.d_ai, na);
  if (f32)
    k_admit_keys<float><<<grid_for(m, TPB), TPB, 0, st>>>((const float *)e.stage, m, d, e.d_ai,
                                                          na, h.keys[0], h.vals[0]);
  else
    k_admit_keys<double><<<grid_for(m, TPB), TPB, 0, st>>>((const double *)e.stage, m, d,
                                                           e.d_ai, na, h.keys[0], h.vals[0]);
  CK(cudaGetLastError());
  const int sc = radix_sort(&h, m, 40 + bits_for(na), st);
  if (sc < 0) return sc;
  const int ward = closed_form(s.linkage);  // no points needed after admission
  int32_t *ord = s.order[h.ocur];
  if (f32)
    k_admit_layout<float><<<grid_for(m, TPB), TPB, 0, st>>>(
        s, (const float *)e.stage, m, e.d_ai, na, h.vals[sc], ord, e.K, e.nterm, e.P, h.pcur,
        e.round, ward);
  else
    k_admit_layout<double><<<grid_for(m, TPB), TPB, 0, st>>>(
        s, (const double *)e.stage, m, e.d_ai, na, h.vals[sc], ord, e.K, e.nterm, e.P, h.pcur,
        e.round, ward);
  CK(cudaGetLastError());
  h.launches += 3;
  e.K += m;
  e.nterm += m;
  if (!ward) e.P += m;
  h.lay_n = e.P;
  // the pinned stage and the batch table are reused by the next admission
  CK(cudaStreamSynchronize(st));
  return HAC_OK;
}

// Hand out the requests whose instance finished (or was dropped) this round:
// `ndone` slots in the device list plus the dropped ones; all their records
// come back in one copy.
int engine_harvest(hac_server *srv, Engine &e, int ndone, const std::vector<int> &drop) {
  hac_ctx &h = e.h;
  State &s = h.s;
  const cudaStream_t st = h.own;
  e.h_list.assign(drop.begin(), drop.end());
  if (ndone > 0) {
    const size_t at = e.h_list.size();
    e.h_list.resize(at + ndone);
    CK(cudaMemcpyAsync(e.h_list.data() + at, s.done_list, ndone * sizeof(int32_t),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  std::sort(e.h_list.begin(), e.h_list.end());
  e.h_list.erase(std::unique(e.h_list.begin(), e.h_list.end()), e.h_list.end());
  if (e.h_list.empty()) return HAC_OK;
  // records of the instances that finished (dropped ones bring none)
  e.h_fin.clear();
  int total = 0;
  for (int slot : e.h_list) {
    SrvReq *r = e.active[slot];
    if (!r || r->dropped) continue;
    e.h_fin.push_back(make_int4(r->base, (int)r->n - 1, total, r->round0));
    total += (int)r->n - 1;
  }
  if (total > 0) {
    const int nf = (int)e.h_fin.size();
    CK(cudaMemcpyAsync(e.d_fin, e.h_fin.data(), nf * sizeof(int4), cudaMemcpyHostToDevice, st));
    k_rec_pack<<<grid_for(total, TPB), TPB, 0, st>>>(s, e.d_fin, nf, total, e.d_rec);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(e.h_rec, e.d_rec, (size_t)total * sizeof(RecOut), cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    h.launches += 1;
  }
  int fi = 0;
  std::vector<int32_t> perm;
  for (int slot : e.h_list) {
    SrvReq *r = e.active[slot];
    if (!r) continue;
    std::vector<hac_merge> out;
    std::vector<int32_t> out_round;
    int status = HAC_OK;
    if (r->dropped) {
      status = r->cancel ? HAC_ECANCELED : HAC_ETIMEOUT;
    } else {
      const RecOut *rec = e.h_rec + e.h_fin[fi++].z;
      const int64_t m = r->n - 1;
      // the canonical order of hac_dendrogram: (height, size, cid_a)
      perm.resize(m);
      for (int64_t i = 0; i < m; ++i) perm[i] = (int32_t)i;
      std::sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) {
        if (rec[x].h != rec[y].h) return rec[x].h < rec[y].h;
        if (rec[x].size != rec[y].size) return rec[x].size < rec[y].size;
        return rec[x].a < rec[y].a;
      });
      out.resize(m);
      for (int64_t i = 0; i < m; ++i) {
        const RecOut &q = rec[perm[i]];
        out[i] = hac_merge{q.a, q.b, q.h, q.size};
      }
      if (r->want_rounds) {
        out_round.resize(m);
        for (int64_t i = 0; i < m; ++i) out_round[i] = rec[perm[i]].round;
      }
    }
    {
      std::lock_guard<std::mutex> g(srv->mu);
      r->out.swap(out);
      r->out_round.swap(out_round);
      r->status = status;
      r->t_done = std::chrono::steady_clock::now();
      range_give(e, r->base, (int)r->n);
      e.free_slots.push_back(slot);
      e.active[slot] = nullptr;
      e.nres -= 1;
      e.completed += 1;
      if (!closed_form(s.linkage)) e.P -= r->n;  // the re-layout left its points out
    }
    srv->done_cv.notify_all();
  }
  h.lay_n = e.P;
  return HAC_OK;
}

void engine_free(Engine *e) {
  if (e->h_stage) cudaFreeHost(e->h_stage);
  if (e->h_rec) cudaFreeHost(e->h_rec);
  e->h_stage = nullptr;
  e->h_rec = nullptr;
  free_all(&e->h);
}

void engine_fail(hac_server *srv, Engine &e, int rc) {
  std::lock_guard<std::mutex> g(srv->mu);
  if (!srv->err) srv->err = rc;
  const auto now = std::chrono::steady_clock::now();
  for (SrvReq *&r : e.active)
    if (r) {
      r->status = rc;
      r->t_done = now;
      r = nullptr;
    }
  for (SrvReq *r : e.queue) {
    r->status = rc;
    r->t_done = now;
  }
  e.queue.clear();
  srv->done_cv.notify_all();
}

void engine_loop(hac_server *srv, Engine *ep) {
  Engine &e = *ep;
  if (cudaSetDevice(srv->device) != cudaSuccess) {
    cudaGetLastError();
    engine_fail(srv, e, HAC_EDEVICE);
    return;
  }
  hac_ctx &h = e.h;
  const cudaStream_t st = h.own;
  RoundCtl ctl;
  std::vector<SrvReq *> batch;
  std::vector<int> drop;
  const char *tr = getenv("HAC_TRACE");
  const bool trace = tr && tr[0] && tr[0] != '0';
  for (;;) {
    batch.clear();
    drop.clear();
    {
      std::unique_lock<std::mutex> g(srv->mu);
      srv->cv.wait(g, [&] { return srv->stop || e.nres > 0 || !e.queue.empty(); });
      if (srv->stop) return;
      // requests that must leave before they finish
      const auto now = std::chrono::steady_clock::now();
      for (SrvReq *r : e.active)
        if (r && !r->dropped && (r->cancel || (r->has_deadline && now >= r->deadline))) {
          r->dropped = true;
          drop.push_back(r->slot);
        }
      // queued requests that fit, in arrival order (one that does not fit
      // yet waits for ids to free up; later, smaller ones may go first)
      for (auto it = e.queue.begin(); it != e.queue.end() && (int)batch.size() < SRV_ADMIT_MAX;) {
        SrvReq *r = *it;
        int base;
        if (r->has_deadline && now >= r->deadline) {
          r->status = HAC_ETIMEOUT;
          r->t_done = now;
          it = e.queue.erase(it);
          srv->done_cv.notify_all();
        } else if (!e.free_slots.empty() && range_take(e, (int)r->n, &base)) {
          r->base = base;
          r->round0 = e.round;
          r->slot = e.free_slots.back();
          e.free_slots.pop_back();
          e.active[r->slot] = r;
          e.nres += 1;
          e.admitted += 1;
          batch.push_back(r);
          it = e.queue.erase(it);
        } else {
          ++it;
        }
      }
      e.max_res = std::max(e.max_res, e.nres);
    }
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) {
      return std::chrono::duration<double, std::milli>(clk::now() - t).count();
    };
    int rc = HAC_OK;
    auto t0 = clk::now();
    for (int slot : drop) k_inst_drop<<<1, 1, 0, st>>>(h.s, slot);
    if (cudaMemsetAsync(&h.s.ctr->ndone, 0, sizeof(int32_t), st) != cudaSuccess) {
      cudaGetLastError();
      engine_fail(srv, e, HAC_EDEVICE);
      return;
    }
    rc = engine_admit(e, batch);
    e.ms_admit += ms_since(t0);
    if (rc == HAC_OK && e.K > 0) {
      t0 = clk::now();
      rc = build_tree(&h, h.s.order[h.ocur], e.K, st);
      int npairs = 0, ndone = 0;
      ctl.big_iters = ctl.big_reqs = 0;
      if (rc == HAC_OK) rc = round_step(&h, st, e.round, e.K, e.nterm, ctl, &npairs);
      if (rc == HAC_OK) {
        Counters c{};
        if (cudaMemcpyAsync(&c, h.s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
          cudaGetLastError();
          rc = HAC_EDEVICE;
        } else if (c.err & ~ERR_NONFINITE) {
          rc = HAC_EINTERNAL;
        } else {
          e.K = c.nactive;
          e.nterm = c.nterm;
          ndone = c.ndone;
        }
      }
      ++e.round;
      ++e.rounds;
      const double ms_r = ms_since(t0);
      e.ms_rounds += ms_r;
      if (trace)
        fprintf(stderr, "srv lk=%d d=%d round %d: admitted %zu resident %d K %d nterm %d pairs %d "
                "big %d/%d %.3f ms\n", (int)h.lk, h.d, e.round - 1, batch.size(), e.nres, e.K,
                e.nterm, npairs, ctl.big_iters, ctl.big_reqs, ms_r);
      t0 = clk::now();
      if (rc == HAC_OK) rc = engine_harvest(srv, e, ndone, drop);
      e.ms_harvest += ms_since(t0);
    } else if (rc == HAC_OK && !drop.empty()) {
      rc = engine_harvest(srv, e, 0, drop);
    }
    if (rc != HAC_OK) {
      engine_fail(srv, e, rc);
      return;
    }
  }
}

}  // namespace

extern "C" int hac_server_create(int64_t points_per_engine, const hac_opts *opts,
                                 hac_server_t *out) {
  if (!out) return HAC_EINVAL;
  *out = nullptr;
  if (points_per_engine < 2 || points_per_engine > (int64_t)INT32_MAX / 4) return HAC_EINVAL;
  hac_opts o;
  hac_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != HAC_PREC_F64 && o.precision != HAC_PREC_F32_RECHECK) return HAC_EINVAL;
  if (o.cache_slots < 0) return HAC_EINVAL;
  hac_server *srv = new (std::nothrow) hac_server();
  if (!srv) return HAC_ENOMEM;
  srv->opt = o;
  srv->cap = points_per_engine;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    cudaGetLastError();
    delete srv;
    return HAC_EDEVICE;
  }
  *out = srv;
  return HAC_OK;
}

namespace {
int submit_impl(hac_server_t srv, const void *points, int64_t n, int d, hac_dtype dt,
                hac_linkage lk, double timeout_s, bool want_rounds, uint64_t *ticket);
}

extern "C" int hac_submit(hac_server_t srv, const void *points, int64_t n, int d, hac_dtype dt,
                          hac_linkage lk, double timeout_s, uint64_t *ticket) {
  return submit_impl(srv, points, n, d, dt, lk, timeout_s, false, ticket);
}

namespace {
int submit_impl(hac_server_t srv, const void *points, int64_t n, int d, hac_dtype dt,
                hac_linkage lk, double timeout_s, bool want_rounds, uint64_t *ticket) {
  if (!srv || !points || !ticket || n < 1 || d < 1 || d > MAXD || !(timeout_s >= 0))
    return HAC_EINVAL;
  if (dt != HAC_F32 && dt != HAC_F64) return HAC_EINVAL;
  if (lk != HAC_COMPLETE && lk != HAC_AVERAGE && lk != HAC_WARD && lk != HAC_AVERAGE_SQ)
    return HAC_EINVAL;
  if (n > srv->cap) return HAC_ENOMEM;
  const size_t esz = dt == HAC_F32 ? 4 : 8;
  for (int64_t i = 0; i < n * d; ++i) {
    const double x =
        dt == HAC_F32 ? (double)((const float *)points)[i] : ((const double *)points)[i];
    if (!std::isfinite(x)) return HAC_EINVAL;
  }
  SrvReq *r = new (std::nothrow) SrvReq();
  if (!r) return HAC_ENOMEM;
  r->pts.assign((const unsigned char *)points, (const unsigned char *)points + n * d * esz);
  r->n = n;
  r->d = d;
  r->dt = dt;
  r->lk = lk;
  r->want_rounds = want_rounds;
  r->t_submit = std::chrono::steady_clock::now();
  if (timeout_s > 0) {
    r->has_deadline = true;
    r->deadline = r->t_submit + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                    std::chrono::duration<double>(timeout_s));
  }
  const int key = ((int)lk * 32 + d) * 2 + (dt == HAC_F32 ? 0 : 1);
  std::unique_lock<std::mutex> g(srv->mu);
  if (srv->err) {
    const int rc = srv->err;
    delete r;
    return rc;
  }
  r->ticket = srv->next_ticket++;
  if (n == 1) {  // nothing to merge
    r->status = HAC_OK;
    r->t_done = r->t_submit;
    srv->reqs[r->ticket] = r;
    *ticket = r->ticket;
    return HAC_OK;
  }
  auto it = srv->engines.find(key);
  Engine *e = it == srv->engines.end() ? nullptr : it->second;
  if (!e) {
    // first request of this kind: its engine (device memory for cap points)
    e = new (std::nothrow) Engine();
    if (!e) {
      delete r;
      return HAC_ENOMEM;
    }
    const int rc = engine_init(*e, lk, d, dt, srv->cap, srv->opt);
    if (rc) {
      engine_free(e);
      delete e;
      delete r;
      return rc;
    }
    try {
      e->thr = std::thread(engine_loop, srv, e);
    } catch (...) {
      engine_free(e);
      delete e;
      delete r;
      return HAC_ENOMEM;
    }
    srv->engines[key] = e;
  }
  r->eng = e;
  srv->reqs[r->ticket] = r;
  e->queue.push_back(r);
  *ticket = r->ticket;
  g.unlock();
  srv->cv.notify_all();
  return HAC_OK;
}
}  // namespace

extern "C" int hac_cancel(hac_server_t srv, uint64_t ticket) {
  if (!srv) return HAC_EINVAL;
  std::unique_lock<std::mutex> g(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return HAC_EINVAL;
  SrvReq *r = it->second;
  if (r->status != HAC_EPENDING) return HAC_OK;  // already finished
  if (r->slot < 0) {  // still queued: leaves at once
    auto &q = r->eng->queue;
    q.erase(std::remove(q.begin(), q.end(), r), q.end());
    r->status = HAC_ECANCELED;
    r->t_done = std::chrono::steady_clock::now();
    g.unlock();
    srv->done_cv.notify_all();
    return HAC_OK;
  }
  r->cancel = true;  // resident: its engine drops it before the next round
  g.unlock();
  srv->cv.notify_all();
  return HAC_OK;
}

extern "C" int hac_poll(hac_server_t srv, uint64_t ticket, hac_merge *out, int64_t cap,
                        int64_t *n_written, double *latency_ms) {
  if (!srv || !n_written) return HAC_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return HAC_EINVAL;
  SrvReq *r = it->second;
  if (r->status == HAC_EPENDING) return HAC_EPENDING;
  const int64_t m = (int64_t)r->out.size();
  if (r->status == HAC_OK && (cap < m || (!out && m > 0))) return HAC_ECAP;
  const int rc = r->status;
  *n_written = rc == HAC_OK ? m : 0;
  if (rc == HAC_OK && m) memcpy(out, r->out.data(), m * sizeof(hac_merge));
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  srv->reqs.erase(it);
  delete r;
  return rc;
}

extern "C" int hac_server_wait(hac_server_t srv, uint64_t ticket, double timeout_s) {
  if (!srv || !(timeout_s >= 0)) return HAC_EINVAL;
  std::unique_lock<std::mutex> g(srv->mu);
  auto ready = [&] {
    auto it = srv->reqs.find(ticket);
    return it == srv->reqs.end() || it->second->status != HAC_EPENDING;
  };
  if (srv->reqs.find(ticket) == srv->reqs.end()) return HAC_EINVAL;
  if (timeout_s > 0) {
    if (!srv->done_cv.wait_for(g, std::chrono::duration<double>(timeout_s), ready))
      return HAC_ETIMEOUT;
  } else {
    srv->done_cv.wait(g, ready);
  }
  return HAC_OK;
}

extern "C" int hac_server_stats(hac_server_t srv, hac_server_stats_t *out) {
  if (!srv || !out) return HAC_EINVAL;
  std::lock_guard<std::mutex> g(srv->mu);
  hac_server_stats_t st{};
  for (auto &kv : srv->engines) {
    const Engine &e = *kv.second;
    st.engines += 1;
    st.rounds += e.rounds;
    st.admitted += e.admitted;
    st.completed += e.completed;
    st.queued += (int64_t)e.queue.size();
    st.resident += e.nres;
    st.max_resident = std::max<int64_t>(st.max_resident, e.max_res);
    st.device_bytes += e.h.bytes;
    st.kernel_launches += e.h.launches;
    st.ms_admit += e.ms_admit;
    st.ms_rounds += e.ms_rounds;
    st.ms_harvest += e.ms_harvest;
  }
  *out = st;
  return srv->err;
}

extern "C" void hac_server_destroy(hac_server_t srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
  }
  srv->cv.notify_all();
  for (auto &kv : srv->engines) {
    if (kv.second->thr.joinable()) kv.second->thr.join();
    if (kv.second->h.own) cudaStreamSynchronize(kv.second->h.own);
    engine_free(kv.second);
    delete kv.second;
  }
  for (auto &kv : srv->reqs) delete kv.second;
  delete srv;
}

// Several handles clustered together: a private server with one engine per
// kind, every handle submitted at once, results written back into the handles
// as hac_run would leave them.
extern "C" int hac_run_batch(hac_t *hs, int count, const hac_opts *opts) {
  if (count < 0 || (count > 0 && !hs)) return HAC_EINVAL;
  hac_opts o;
  hac_default_opts(&o);
  if (opts) o = *opts;
  if (o.precision != HAC_PREC_F64 && o.precision != HAC_PREC_F32_RECHECK) return HAC_EINVAL;
  if (o.cache_slots < 0 || o.max_rounds != 0 || !(o.timeout_s >= 0)) return HAC_EINVAL;
  std::map<int, int64_t> kind_n;
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return HAC_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return HAC_EINVAL;
    kind_n[((int)hs[i]->lk * 32 + hs[i]->d) * 2 + (hs[i]->dt == HAC_F32 ? 0 : 1)] += hs[i]->n;
  }
  if (count == 0) return HAC_OK;
  int64_t cap = 2;
  for (auto &kv : kind_n) cap = std::max(cap, kv.second);
  const auto t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < count; ++i) hs[i]->done = false;
  hac_server_t srv = nullptr;
  hac_opts so = o;
  so.timeout_s = 0;
  int rc = hac_server_create(cap, &so, &srv);
  if (rc) return rc;
  std::vector<uint64_t> tickets(count, 0);
  std::vector<int> st(count, HAC_OK);
  std::vector<unsigned char> host;
  for (int i = 0; i < count && !rc; ++i) {
    hac_ctx *h = hs[i];
    const size_t bytes = (size_t)h->n * h->d * (h->dt == HAC_F32 ? 4 : 8);
    host.resize(bytes);
    if (cudaMemcpy(host.data(), h->raw, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      rc = HAC_EDEVICE;
      break;
    }
    st[i] = submit_impl(srv, host.data(), h->n, h->d, h->dt, h->lk, o.timeout_s, true,
                        &tickets[i]);
  }
  for (int i = 0; i < count && !rc; ++i) {
    if (st[i] != HAC_OK) continue;
    hac_server_wait(srv, tickets[i], 0);
    hac_ctx *h = hs[i];
    std::unique_lock<std::mutex> g(srv->mu);
    SrvReq *r = srv->reqs[tickets[i]];
    st[i] = r->status;
    if (r->status != HAC_OK) continue;
    const int64_t m = (int64_t)r->out.size();
    int32_t rounds = 0;
    for (int32_t v : r->out_round) rounds = std::max(rounds, v + 1);
    if (m && (cudaMemcpy(h->dout, r->out.data(), m * sizeof(hac_merge),
                         cudaMemcpyHostToDevice) != cudaSuccess ||
              cudaMemcpy(h->dout_round, r->out_round.data(), m * sizeof(int32_t),
                         cudaMemcpyHostToDevice) != cudaSuccess)) {
      cudaGetLastError();
      st[i] = HAC_EDEVICE;
      continue;
    }
    h->n_merges = m;
    h->st = hac_stats_t{};
    h->st.rounds = rounds;
    h->st.merges = m;
    h->st.device_bytes = h->bytes;
    h->st.ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->done = true;
  }
  hac_server_destroy(srv);
  if (rc) return rc;
  for (int i = 0; i < count; ++i)
    if (st[i] != HAC_OK) return st[i];
  return HAC_OK;
}
