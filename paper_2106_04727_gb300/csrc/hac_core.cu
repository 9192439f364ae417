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
//                               k_tg_*: rebuild the range-query tree
#include "hac_impl.cuh"

#include <algorithm>
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
__global__ void k_layout(State s, const T *X, const int32_t *perm, const uint64_t *skey,
                         MortonParams ctr_) {
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
    s.mkey[i] = skey[p];
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
// Level L cuts the m elements below it (positions for L = 0, level-(L-1)
// nodes above) into runs of at most 32 consecutive elements.  An element's
// key is 96 bits: its instance's admission number, then the Morton key of its
// (first) position at layout; keys never decrease along the order.  A run is
// the largest cell of that key hierarchy (the elements sharing a key prefix)
// holding at most 32 elements, so sibling boxes are those of disjoint Morton
// cells instead of fixed slices that straddle cell boundaries.  Element i's
// cell has prefix length l* = 1 + c, c being the 32nd largest common-prefix
// length between i and its 64 neighbours i - 32 .. i + 32 (a cell of more
// than 32 elements has at least 32 of them in that window); i starts a run
// iff it shares at most c leading bits with i - 1.  Cells nest, so the runs
// partition the elements.  More than 32 equal keys are also cut every 32
// positions.  A level whose runs would exceed its capacity (tree_caps), or
// whose keys are out of order, is cut into fixed runs of 32 instead.
constexpr int TG_H = 32;              // window half-width
constexpr int TG_W = TPB + 2 * TG_H;  // keys staged per block

// keys of elements [b0 - 32, b0 + TPB + 32) into shared memory (instance -1:
// no element); level 0 reads them through the order
__device__ void tg_stage(uint64_t *sk, int32_t *sq, const uint64_t *ekey, const int32_t *eorder,
                         const int32_t *einst, int m, int b0) {
  for (int t = threadIdx.x; t < TG_W; t += TPB) {
    const int i = b0 - TG_H + t;
    const bool v = i >= 0 && i < m;
    sk[t] = v ? ekey[eorder ? eorder[i] : i] : 0ull;
    sq[t] = v ? einst[i] : -1;
  }
  __syncthreads();
}

// common-prefix length of the 96-bit keys at staged slots u and w (-1: none)
__device__ __forceinline__ int tg_cpl(const uint64_t *sk, const int32_t *sq, int u, int w) {
  if (sq[w] < 0) return -1;
  if (sq[u] != sq[w]) return __clz(sq[u] ^ sq[w]);
  const uint64_t x = sk[u] ^ sk[w];
  return x ? 32 + __clzll((long long)x) : 96;
}

// does element i (staged at slot t + 32) start a run?
__device__ bool tg_start(const uint64_t *sk, const int32_t *sq, int i, int t) {
  if (i == 0) return true;
  const int u = t + TG_H;
  const int left1 = tg_cpl(sk, sq, u, u - 1);
  // the 32nd largest of the 64 neighbour lengths: both sides fall off
  // monotonically, so merge them from the nearest outwards
  int a = 1, b = 1, lv = left1, rv = tg_cpl(sk, sq, u, u + 1), c = -1;
  for (int k = 0; k < TG_H; ++k) {
    if (lv >= rv) {
      c = lv;
      ++a;
      lv = a <= TG_H ? tg_cpl(sk, sq, u, u - a) : -2;
    } else {
      c = rv;
      ++b;
      rv = b <= TG_H ? tg_cpl(sk, sq, u, u + b) : -2;
    }
  }
  if (c >= 96) return left1 < 96 || (i % FAN) == 0;  // more than 32 equal keys
  return left1 <= c;
}

// elements of level L and whether the build stopped below it (a lower level
// already has at most 32 nodes)
__device__ __forceinline__ bool tg_idle(const State &s, int L) {
  const int top = s.tinfo[TI_TOP];
  return top != 0 && top - 1 < L;
}

// per-block counts of run starts; flags the level if its keys are out of order
__global__ void k_tg_count(State s, int L, const uint64_t *ekey, const int32_t *eorder,
                           const int32_t *einst, int K) {
  __shared__ uint64_t sk[TG_W];
  __shared__ int32_t sq[TG_W];
  if (tg_idle(s, L)) return;
  const int m = L ? s.tinfo[L - 1] : K;
  if ((int)blockIdx.x >= cdiv(m, TPB)) return;
  const int b0 = blockIdx.x * TPB;
  tg_stage(sk, sq, ekey, eorder, einst, m, b0);
  const int i = b0 + threadIdx.x;
  int f = 0;
  if (i < m) {
    f = tg_start(sk, sq, i, threadIdx.x);
    const int u = threadIdx.x + TG_H;
    if (i > 0 && (sq[u - 1] > sq[u] || (sq[u - 1] == sq[u] && sk[u - 1] > sk[u])))
      atomicOr(&s.tinfo[TI_FIXED], 1 << L);
  }
  f = block_sum(f);
  if (threadIdx.x == 0) s.bsum[blockIdx.x] = f;
}

// one block: scan of the block counts; the level's node count, its end
// entry, and the choice between the Morton runs and fixed runs of 32
__global__ void k_tg_top(State s, int L, int K, int cap) {
  if (tg_idle(s, L)) return;
  const int m = L ? s.tinfo[L - 1] : K;
  const int nb = cdiv(m, TPB);
  const int per = cdiv(nb, TPB);
  const int b0 = threadIdx.x * per;
  int sum = 0;
  for (int i = 0; i < per; ++i)
    if (b0 + i < nb) sum += s.bsum[b0 + i];
  int tot;
  int pre = block_excl_scan(sum, &tot);
  for (int i = 0; i < per; ++i)
    if (b0 + i < nb) {
      const int v = s.bsum[b0 + i];
      s.bsum[b0 + i] = pre;
      pre += v;
    }
  if (threadIdx.x == 0) {
    const bool fixed = ((s.tinfo[TI_FIXED] >> L) & 1) || tot > cap;
    const int mL = fixed ? cdiv(m, FAN) : tot;
    s.tinfo[L] = mL;
    if (fixed) s.tinfo[TI_FIXED] |= 1 << L;
    s.nch[s.chb[L] + mL] = m;
    if (mL <= FAN) s.tinfo[TI_TOP] = L + 1;
  }
}

// first child of every node of level L, the node's key (its first child's),
// and for L = 0 the bucket of every position
__global__ void k_tg_write(State s, int L, const uint64_t *ekey, const int32_t *eorder,
                           const int32_t *einst, uint64_t *okey, int32_t *oinst, int K) {
  __shared__ uint64_t sk[TG_W];
  __shared__ int32_t sq[TG_W];
  if (tg_idle(s, L)) return;
  const int m = L ? s.tinfo[L - 1] : K;
  if ((int)blockIdx.x >= cdiv(m, TPB)) return;
  const bool fixed = (s.tinfo[TI_FIXED] >> L) & 1;
  const int b0 = blockIdx.x * TPB;
  tg_stage(sk, sq, ekey, eorder, einst, m, b0);
  const int i = b0 + threadIdx.x;
  const int f = i < m && (fixed ? (i % FAN) == 0 : tg_start(sk, sq, i, threadIdx.x));
  int tot;
  const int idx = block_excl_scan(f, &tot) + (fixed ? b0 / FAN : s.bsum[blockIdx.x]);
  if (f) {
    s.nch[s.chb[L] + idx] = i;
    okey[idx] = sk[threadIdx.x + TG_H];
    oinst[idx] = sq[threadIdx.x + TG_H];
  }
  if (L == 0 && i < m) s.pbkt[i] = idx + f - 1;
}

// Box, least cluster size and instance range of node j of level L, one lane
// per child (children: positions for L = 0, of which there are mb)
template <int DP>
__device__ void tg_node_box(const State &s, int L, int j, int mb, int lane) {
  const int *nch = s.nch + s.chb[L];
  const int c0 = nch[j];
  int nc = nch[j + 1] - c0;
  if (nc < 1 || nc > FAN) {
    if (lane == 0) atomicOr(&s.ctr->err, ERR_TREE);
    nc = max(1, min(nc, FAN));
  }
  const bool v = lane < nc && c0 + lane < mb;
  // a child: a position-ordered record (L = 0) or a node of level L - 1
  const size_t c = (size_t)(L ? s.lvl_base[L - 1] : 0) + (size_t)(v ? c0 + lane : c0);
  int nm = v ? (L ? s.nnmin[c] : s.qsz[c]) : INT_MAX;
  int il = v ? (L ? s.ninlo[c] : s.qinst[c]) : INT_MAX;
  int ih = v ? (L ? s.ninhi[c] : s.qinst[c]) : INT_MIN;
  for (int o = 16; o; o >>= 1) {
    nm = min(nm, __shfl_xor_sync(0xffffffffu, nm, o));
    il = min(il, __shfl_xor_sync(0xffffffffu, il, o));
    ih = max(ih, __shfl_xor_sync(0xffffffffu, ih, o));
  }
  const int node = s.lvl_base[L] + j;
  if (lane == 0) {
    s.ninlo[node] = il;
    s.ninhi[node] = ih;
    s.nnmin[node] = nm;
  }
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    float lo, hi, hm, lm;
    if (L) {
      lo = v ? s.nclo[c * DP + k] : INFINITY;
      hi = v ? s.nchi[c * DP + k] : -INFINITY;
      hm = v ? s.nhmin[c * DP + k] : INFINITY;
      lm = v ? s.nlmax[c * DP + k] : -INFINITY;
    } else {
      lo = v ? s.q32[c * DP + k] : INFINITY;
      hi = v ? s.q32[c * DP + k] : -INFINITY;
      hm = v ? s.qbhi[c * DP + k] : INFINITY;
      lm = v ? s.qblo[c * DP + k] : -INFINITY;
    }
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
}

// boxes, least cluster size and instance range of every node of level L
// (one warp per node)
template <int DP>
__global__ void k_tg_box(State s, int L, int K) {
  if (tg_idle(s, L)) return;
  const int cnt = s.tinfo[L];
  const int mb = L ? s.tinfo[L - 1] : K;  // children of this level
  for (int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < cnt;
       j += (gridDim.x * blockDim.x) >> 5)
    tg_node_box<DP>(s, L, j, mb, threadIdx.x & 31);
}

// The upper levels in one block.  Once a level has at most TG_TAIL elements
// (and for the whole tree when K <= TG_TAIL), one block of 1,024 threads
// builds it and every level above: the elements' keys are staged in shared
// memory, runs are cut by the same rule as above (tg_start over the whole
// staged level), the node keys of the next level stay in shared memory, and
// the boxes are reduced by the block's 32 warps.  This saves four launches
// per level in the many late rounds of small K.
constexpr int TG_TAIL = 2048;
constexpr int TG_TT = 1024;  // threads of the tail block
struct TgCaps {
  int cap[MAXLEV + 1];
};

// exclusive scan of one int per thread over TG_TT threads
__device__ int tail_scan(int v, int *total, int *ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  const int pre = w ? ws[w - 1] : 0;
  *total = ws[31];
  __syncthreads();
  return pre + x - v;
}

// levels L0 .. nl - 1 in one block (L0: the first level the host leaves to
// it; a lower level may already be the top, then nothing is left to do)
template <int DP>
__global__ void __launch_bounds__(TG_TT) k_tg_tail(State s, const int32_t *order,
                                                   const uint64_t *ekey, const int32_t *einst,
                                                   int L0, int nl, int K, TgCaps caps) {
  // the level staged whole, between halos of TG_H empty slots (instance -1),
  // so that tg_start reads it exactly as the grid-wide kernels read theirs
  __shared__ uint64_t sk_h[TG_TAIL + 2 * TG_H];
  __shared__ int32_t sq_h[TG_TAIL + 2 * TG_H];
  uint64_t *sk = sk_h + TG_H;
  int32_t *sq = sq_h + TG_H;
  __shared__ int ws[32];
  __shared__ int s_fixed;
  if (L0 > 0 && tg_idle(s, L0)) return;  // uniform
  int m = L0 ? s.tinfo[L0 - 1] : K;
  if (m > TG_TAIL) {  // cannot happen: the host hands over levels of at most TG_TAIL
    if (threadIdx.x == 0) atomicOr(&s.ctr->err, ERR_TREE);
    return;
  }
  for (int i = threadIdx.x; i < m; i += TG_TT) {
    sk[i] = L0 ? ekey[i] : s.mkey[order[i]];
    sq[i] = L0 ? einst[i] : s.qinst[i];
  }
  for (int L = L0; L < nl; ++L) {
    // empty slots from m on (the halo below 0 stays empty)
    for (int i = threadIdx.x; i < TG_TAIL + TG_H; i += TG_TT) {
      if (i < TG_H) sq_h[i] = -1;
      if (i >= m) sq[i] = -1;
    }
    if (threadIdx.x == 0) s_fixed = 0;
    __syncthreads();
    // run starts of this thread's elements (at most TG_TAIL / TG_TT of them)
    constexpr int PER = TG_TAIL / TG_TT;
    bool f[PER];
    uint64_t kk[PER];
    int32_t qq[PER];
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = threadIdx.x * PER + r;
      f[r] = false;
      if (i < m) {
        f[r] = tg_start(sk_h, sq_h, i, i);
        kk[r] = sk[i];
        qq[r] = sq[i];
        if (i > 0 && (sq[i - 1] > sq[i] || (sq[i - 1] == sq[i] && sk[i - 1] > sk[i])))
          s_fixed = 1;
      }
    }
    __syncthreads();
    int tot;
#pragma unroll
    for (int r = 0; r < PER; ++r) cnt += f[r];
    int pre = tail_scan(cnt, &tot, ws);
    const bool fixed = s_fixed || tot > caps.cap[L];
    if (fixed) {
      cnt = 0;
#pragma unroll
      for (int r = 0; r < PER; ++r) {
        const int i = threadIdx.x * PER + r;
        f[r] = i < m && (i % FAN) == 0;
        cnt += f[r];
      }
      pre = tail_scan(cnt, &tot, ws);
    }
    const int mL = tot;
    // first children, node keys (into shared memory for the next level), buckets
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = threadIdx.x * PER + r;
      if (i >= m) continue;
      if (f[r]) {
        s.nch[s.chb[L] + pre] = i;
        sk[pre] = kk[r];
        sq[pre] = qq[r];
      }
      if (L == 0) s.pbkt[i] = pre + (f[r] ? 0 : -1);
      pre += f[r];
    }
    if (threadIdx.x == 0) {
      s.tinfo[L] = mL;
      if (fixed) s.tinfo[TI_FIXED] |= 1 << L;
      s.nch[s.chb[L] + mL] = m;
      if (mL <= FAN) s.tinfo[TI_TOP] = L + 1;
    }
    __syncthreads();
    for (int j = threadIdx.x >> 5; j < mL; j += TG_TT / 32)
      tg_node_box<DP>(s, L, j, m, threadIdx.x & 31);
    __syncthreads();
    if (mL <= FAN) break;
    m = mL;
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
// pair-distance cache (Section 5): search results and merges
// ---------------------------------------------------------------------------

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

#ifndef HAC_CM_WARPS
#define HAC_CM_WARPS 2
#endif
constexpr int CM_WARPS = HAC_CM_WARPS;  // warps per block of k_cache_merge (5 * slots entries each)

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

namespace hacg {

int device_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (dev >= 0 && dev < kMaxDev) {
    const int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1) {
    cudaGetLastError();
    return 1;
  }
  if (dev >= 0 && dev < kMaxDev) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

void free_all(hac_ctx *h) {
  for (void *p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->own) cudaStreamDestroy(h->own);
  h->own = nullptr;
}

int pad_dim(int d) { return d <= 2 ? 2 : d <= 4 ? 4 : d <= 8 ? 8 : 16; }

// Offsets of every tree level in the node arrays (lvl_base) and in the
// first-child array (chb, one end entry per level), for up to n clusters.
void tree_layout(State &s, int n, int *nodes, int *chs) {
  int cap[MAXLEV + 1];
  const int nl = tree_caps(n, cap);
  int base = 0, cb = 0;
  for (int L = 0; L <= MAXLEV; ++L) {
    s.lvl_base[L] = base;
    s.chb[L] = cb;
    if (L < nl) {
      base += cap[L];
      cb += cap[L] + 1;
    }
  }
  *nodes = base;
  *chs = cb;
}

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
  A(s.blist, n);
  A(s.pair_lo, n / 2 + 1);
  A(s.pair_hi, n / 2 + 1);
  A(s.pair_key, n / 2 + 1);
  A(s.m_a, n);
  A(s.m_b, n);
  A(s.m_size, n);
  A(s.m_round, n);
  A(s.m_h, n);
  // tree levels sized for K = n
  int base = 0, chbase = 0;
  tree_layout(s, (int)n, &base, &chbase);
  A(s.nclo, (int64_t)base * dp);
  A(s.nchi, (int64_t)base * dp);
  A(s.nhmin, (int64_t)base * dp);
  A(s.nlmax, (int64_t)base * dp);
  A(s.nnmin, base);
  A(s.ninlo, base);
  A(s.ninhi, base);
  A(s.nch, chbase);
  A(s.pbkt, n);
  A(s.mkey, n);
  A(s.tinfo, TI_SIZE);
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

template <int DP>
int build_tree_dp(hac_ctx *h, const int32_t *order, int K, cudaStream_t st) {
  State &s = h->s;
  int cap[MAXLEV + 1];
  const int nl = tree_caps(K, cap);
  CK(cudaMemsetAsync(s.tinfo, 0, TI_SIZE * sizeof(int32_t), st));
  // levels whose elements may exceed TG_TAIL: four grid-wide launches each;
  // levels above the first one of at most 32 nodes return at once
  int L = 0;
  for (; L < nl && (L ? cap[L - 1] : K) > TG_TAIL; ++L) {
    const int nb = cdiv(L ? cap[L - 1] : K, TPB);  // blocks for the most elements possible
    const uint64_t *ek = L ? h->keys[(L - 1) & 1] : s.mkey;
    const int32_t *eo = L ? nullptr : order;
    const int32_t *ei = L ? h->vals[(L - 1) & 1] : s.qinst;
    k_tg_count<<<nb, TPB, 0, st>>>(s, L, ek, eo, ei, K);
    k_tg_top<<<1, TPB, 0, st>>>(s, L, K, cap[L]);
    k_tg_write<<<nb, TPB, 0, st>>>(s, L, ek, eo, ei, h->keys[L & 1], h->vals[L & 1], K);
    k_tg_box<DP><<<grid_for((int64_t)cap[L] * 32, TPB), TPB, 0, st>>>(s, L, K);
    h->launches += 4;
  }
  // the rest in one block
  if (L < nl) {
    TgCaps c{};
    for (int l = 0; l < nl; ++l) c.cap[l] = cap[l];
    k_tg_tail<DP><<<1, TG_TT, 0, st>>>(s, order, L ? h->keys[(L - 1) & 1] : nullptr,
                                       L ? h->vals[(L - 1) & 1] : nullptr, L, nl, K, c);
    h->launches += 1;
  }
  h->launches += 1;
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

// Initial layout (Algorithm 1 initialisation): bounding box, recentring,
// Morton keys, radix sort, permuted points and per-cluster state, the tree.
// Host buffers are stack arrays, so hac_run_static can use it unchanged.
template <typename T>
int init_layout(hac_ctx *h, cudaStream_t st) {
  State &s = h->s;
  const T *X = (const T *)h->raw;
  const int64_t n = h->n;
  const int d = h->d;
  unsigned long long bb[2 * MAXD];
  for (int k = 0; k < MAXD; ++k) {
    bb[k] = ~0ull;
    bb[MAXD + k] = 0ull;
  }
  CK(cudaMemcpyAsync(h->bb, bb, sizeof(bb), cudaMemcpyHostToDevice, st));
  // counters start from zero (the allocation-free arena keeps the last call's)
  CK(cudaMemsetAsync(s.ctr, 0, sizeof(Counters), st));
  k_bbox<T><<<grid_for(n, TPB), TPB, 0, st>>>(X, n, d, h->bb, h->bb + MAXD, s.ctr);
  h->launches += 3;  // bbox, morton, layout
  CK(cudaGetLastError());
  Counters c0;
  CK(cudaMemcpyAsync(bb, h->bb, sizeof(bb), cudaMemcpyDeviceToHost, st));
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
  double scale = 0.0, raw = 0.0;
  for (int k = 0; k < d; ++k) {
    double lo = dec(bb[k]), hi = dec(bb[MAXD + k]);
    mp.lo[k] = lo;
    mp.inv[k] = hi > lo ? 1.0 / (hi - lo) : 0.0;
    ctrp.lo[k] = 0.5 * (lo + hi);
    scale = std::max(scale, std::max(std::fabs(lo - ctrp.lo[k]), std::fabs(hi - ctrp.lo[k])));
    raw = std::max(raw, std::max(std::fabs(lo), std::fabs(hi)));
  }
  // the FP32 copy holds the input itself (FP32 input) or the recentred points
  s.p32_max = s.pts32_exact ? raw : scale * (1.0 + 1e-6);
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
  s.dense = 0;
  s.dk = 0;
  k_layout<T><<<grid_for(n, TPB), TPB, 0, st>>>(s, X, h->vals[sc], h->keys[sc], ctrp);
  CK(cudaGetLastError());
  Counters c{};
  c.nterm = (int)n;
  c.nactive = (int)n;
  CK(cudaMemcpyAsync(s.ctr, &c, sizeof(Counters), cudaMemcpyHostToDevice, st));
  return build_tree(h, s.order[0], (int)n, st);
}

// Canonical order of the merge records on the device, (height, size, cid_a)
// by three stable radix passes ((cid_a, size) already identifies a merge, so
// the order is total), gathered into `out` / `out_round`.
int sort_records(hac_ctx *h, cudaStream_t st, hac_merge *out, int32_t *out_round) {
  State &s = h->s;
  const int64_t m = h->n - 1;
  if (m <= 0) return HAC_OK;
  const int mm = (int)m;
  const int g = grid_for(mm, TPB);
  int32_t *perm = nullptr;
  const int fbits[3] = {bits_for(h->n), bits_for(h->n), 64};
  for (int f = 0; f < 3; ++f) {
    k_rec_key<<<g, TPB, 0, st>>>(s, mm, f, perm, h->keys[0], h->vals[0]);
    const int r = radix_sort(h, mm, fbits[f], st);
    if (r < 0) return r;
    if (r == 1)
      CK(cudaMemcpyAsync(h->vals[0], h->vals[1], (size_t)mm * 4, cudaMemcpyDeviceToDevice, st));
    perm = h->vals[0];
  }
  k_rec_gather<<<g, TPB, 0, st>>>(s, mm, perm, out, out_round);
  h->launches += 4;
  CK(cudaGetLastError());
  return HAC_OK;
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
  if (const char *e = getenv("HAC_BRUTE")) h->brute_env = atoi(e) ? 1 : 0;
  if (const char *e = getenv("HAC_DENSE_K")) h->dense_k = std::max(0ll, atoll(e));
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
  qa.nch = s.nch;
  qa.pbkt = s.pbkt;
  qa.tinfo = s.tinfo;
  for (int L = 0; L <= MAXLEV; ++L) {
    qa.lvl_base[L] = s.lvl_base[L];
    qa.chb[L] = s.chb[L];
  }
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

// Exhaustive tiled search instead of the tree: closed-form linkages in the
// FP32 mode, one instance, and d > 8 (where the tree prunes little);
// HAC_BRUTE=0 / 1 turns it off / on for any row stride of 8 or 16.
bool use_brute(const hac_ctx *h) {
  const State &s = h->s;
  if (!closed_form(s.linkage) || s.prec != HAC_PREC_F32_RECHECK || s.max_inst != 1) return false;
  if (h->brute_env >= 0) return h->brute_env == 1 && (s.dp == 8 || s.dp == 16);
  return s.dp == 16;
}

// Candidate lists from the exhaustive scan instead of the tree for average
// linkage in d > 8 (one instance); HAC_BRUTE=0 / 1 turns them off / on for any
// row stride of 8 or 16.
bool use_cand_avg(const hac_ctx *h) {
  const State &s = h->s;
  if (s.linkage != LK_AVERAGE || s.max_inst != 1 || s.noprune || s.dense) return false;
  if (h->brute_env >= 0) return h->brute_env == 1 && (s.dp == 8 || s.dp == 16);
  return s.dp == 16;
}

// Precision of the tree search.  Ward and avg-2 distances are O(d) closed
// forms of the cluster records, so an FP64 evaluation costs no more than the
// FP32 bound test and needs no re-score pass: their tree searches run in FP64
// in both modes (measured faster on every workload tried); the FP32 mode
// keeps its FP32 bulk for the exhaustive scans and for complete / average.
int query_prec(const State &s) {
  return closed_form(s.linkage) ? (int)HAC_PREC_F64 : s.prec;
}

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
  // average linkage on the dense matrix once the active clusters fit
  const int dense = dense_maybe_enter(h, st, K, ctl);
  if (dense < 0) return dense;
  QueryArgs qa{};
  fill_query_args(h, qa, round, K, nterm);
  const bool defer = !dense && qa.defer != 0;
  if (defer)
    CK(cudaMemsetAsync(s.side_key, 0xff, (size_t)s.side_cap * sizeof(unsigned long long), st));
  const bool brute = !dense && use_brute(h);
  if (brute) {
    CK(cudaMemsetAsync(&s.ctr->npend, 0, sizeof(int32_t), st));
    qa.pend_out = s.blist;
  }
  if (!dense && use_cand_avg(h)) {
    if (!s.lpos) {  // sized once per handle: BL_CAP positions per cluster
      if ((rc = dalloc(h, &s.lpos, (size_t)h->n * BL_CAP)) ||
          (rc = dalloc(h, &s.llb, (size_t)h->n * BL_CAP)) || (rc = dalloc(h, &s.lcnt, h->n)) ||
          (rc = dalloc(h, &s.lub, h->n)))
        return rc;
    }
    CK(launch_cand_avg(qa, s.lpos, s.llb, s.lcnt, s.lub, s.dp, st));
    h->launches += 1;
    qa.lcap = BL_CAP;
    qa.lpos = s.lpos;
    qa.lcnt = s.lcnt;
    qa.lub = s.lub;
  }
  EVREC(ctl.eq0);
  if (dense) {
    rc = dense_search(h, st, K, nterm, ctl);
    if (rc) return rc;
    ++ctl.dense_rounds;
  } else if (brute) {
    CK(launch_brute(qa, s.dp, st));
  } else {
    CK(launch_query(qa, s.dp, query_prec(s), st));
  }
  EVREC(ctl.eq1);
  if (!dense) {
    ++ctl.qlaunch;
    ctl.searches += nterm;
    h->launches += 1;
  }
  if (!dense && s.cache_slots > 0) {
    k_cache_insert<<<grid_for((int64_t)device_sms() * 8 * TPB, TPB), TPB, 0, st>>>(s);
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
    // the batches of one pass run back to back; their device time (with
    // the small scheduling and folding kernels) is read once per pass
    EVREC(ctl.eb0);
    for (int r0 = 0; r0 < nreq; r0 += BIG_BATCH) {
      const int m = std::min(BIG_BATCH, nreq - r0);
      rc = big_prepare(s, r0, m, st);
      if (rc) return rc;
      rc = launch_big(s, r0, st);
      if (rc) return rc;
      ctl.big_launch += 3;  // kinds 0 and 1 (FP32), FP64
      rc = big_finish(s, r0, m, st);
      if (rc) return rc;
      h->launches += 6;
    }
    EVREC(ctl.eb1);
    if (ctl.eb0) {
      CK(cudaEventSynchronize(ctl.eb1));
      float bms;
      cudaEventElapsedTime(&bms, ctl.eb0, ctl.eb1);
      ctl.ms_big += bms;
    }
    CK(cudaMemsetAsync(&s.ctr->nbreq, 0, 2 * sizeof(int32_t), st));
    ctl.searches += npend;
    qa.term = s.pend[it & 1];
    qa.nterm = npend;
    qa.pend_out = s.pend[(it & 1) ^ 1];
    qa.defer = it < 4 ? 1 : 0;
    EVREC(ctl.eq0);
    CK(launch_query(qa, s.dp, query_prec(s), st));
    EVREC(ctl.eq1);
    ++ctl.qlaunch;
    k_cache_insert<<<grid_for((int64_t)device_sms() * 8 * TPB, TPB), TPB, 0, st>>>(s);
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
  if (dense) {
    rc = dense_update(h, st, round, K, npairs);
    if (rc) return rc;
  } else if (s.cache_slots > 0) {
    const int S = s.cache_slots;
    const size_t smem = (size_t)CM_WARPS * 5 * S * sizeof(CEntry);
    const int blocks = std::max(1, std::min(cdiv(npairs, CM_WARPS), device_sms() * 32));
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

// Release one array taken by dalloc (count elements) before the handle is
// destroyed; a null pointer is left alone.
template <typename T>
static void dfree(hac_ctx *h, T *&p, size_t count) {
  if (!p) return;
  for (auto it = h->allocs.begin(); it != h->allocs.end(); ++it)
    if (*it == (void *)p) {
      h->allocs.erase(it);
      cudaFree(p);
      h->bytes -= (int64_t)(std::max<size_t>(count, 1) * sizeof(T));
      break;
    }
  p = nullptr;
}

// Phase timing and per-round trace of run_rounds (hac_run only).
struct RoundTimes {
  cudaEvent_t e0 = nullptr, e3 = nullptr;
  double ms_nn = 0, ms_merge = 0, ms_update = 0;
  bool trace = false;
};

// Algorithm 1's rounds from the initial layout until one cluster is left:
// round_step, tree rebuild, then the round's counters are read and checked.
// HAC_ETIMEOUT once a limit of `opt` is reached (checked between rounds).
// `tm` may be null (no timing; ctl's events must be null too).
int run_rounds(hac_ctx *h, const hac_opts &opt, cudaStream_t st, RoundCtl &ctl, RoundTimes *tm,
               std::chrono::steady_clock::time_point t0, int *rounds_out) {
  State &s = h->s;
  int K = (int)h->n, nterm = (int)h->n, round = 0, rc = 0;
  Counters c{}, cprev{};
  const bool trace = tm && tm->trace;
  *rounds_out = 0;
  while (K > 1) {
    if (opt.max_rounds && round >= opt.max_rounds) return HAC_ETIMEOUT;
    if (opt.timeout_s > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >
            opt.timeout_s)
      return HAC_ETIMEOUT;
    if (tm) cudaEventRecord(tm->e0, st);
    const int big_iters0 = ctl.big_iters, big_reqs0 = ctl.big_reqs;
    ctl.naive += (int64_t)nterm * (K - 1);
    int npairs = 0;
    rc = round_step(h, st, round, K, nterm, ctl, &npairs);
    if (rc == HAC_EINTERNAL && npairs <= 0 && trace) {
      CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      fprintf(stderr, "hac round %d: no reciprocal pair (err %d)\n", round, c.err);
    }
    if (rc) return rc;
    K -= npairs;
    if (K > 1 && !s.dense) {
      rc = build_tree(h, s.order[h->ocur], K, st);
      if (rc) return rc;
    }
    if (tm) cudaEventRecord(tm->e3, st);
    CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // the last merge finishes the instance: its single cluster leaves the order
    if ((c.err & ~ERR_NONFINITE) || (c.nactive != K && !(K == 1 && c.nactive == 0))) {
      if (trace)
        fprintf(stderr, "hac round %d: consistency (err %d, active %d, expected %d)\n", round,
                c.err, c.nactive, K);
      return HAC_EINTERNAL;
    }
    if (tm) {
      float a, b, d3, q;
      cudaEventElapsedTime(&a, tm->e0, ctl.e1);
      cudaEventElapsedTime(&b, ctl.e1, ctl.e2);
      cudaEventElapsedTime(&d3, ctl.e2, tm->e3);
      cudaEventElapsedTime(&q, ctl.eq0, ctl.eq1);
      ctl.ms_query += q;
      tm->ms_nn += a;
      tm->ms_merge += b;
      tm->ms_update += d3;
      if (trace) {
        fprintf(stderr,
                "hac round %d K %d terms %d pairs %d query_ms %.3f leaf_tests %llu nodes %llu "
                "cpairs %llu ppairs %llu rechecks %llu nn_ms %.3f merge_ms %.3f update_ms %.3f "
                "big_iters %d big_reqs %d hits %llu big_pp %llu big_exact %llu\n",
                round, K + npairs, nterm, npairs, q, c.ltests - cprev.ltests,
                c.nodes - cprev.nodes, c.cluster_pairs - cprev.cluster_pairs,
                c.point_pairs - cprev.point_pairs, c.rechecks - cprev.rechecks, a, b, d3,
                ctl.big_iters - big_iters0, ctl.big_reqs - big_reqs0,
                c.cache_hits - cprev.cache_hits, c.big_pp - cprev.big_pp,
                c.big_exact - cprev.big_exact);
        cprev = c;
      }
    }
    nterm = c.nterm;
    ++round;
    *rounds_out = round;
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
    // a larger table replaces the old one (a smaller request reuses it)
    const size_t old_cells = (size_t)h->n * h->cache_alloc_slots;
    dfree(h, s.ckey, old_cells);
    dfree(h, s.cval, old_cells);
    dfree(h, s.cerr, old_cells);
    dfree(h, s.cpart, old_cells);
    h->cache_alloc_slots = 0;
    const size_t cells = (size_t)h->n * slots;
    if ((rc0 = dalloc(h, &s.ckey, cells)) || (rc0 = dalloc(h, &s.cval, cells)) ||
        (rc0 = dalloc(h, &s.cerr, cells)) || (rc0 = dalloc(h, &s.cpart, cells)))
      return rc0;
    if (!s.ins_i) {  // queue of evaluated pairs to insert (sized once per handle)
      const int64_t cap = std::max<int64_t>(4 * h->n, 1 << 16);
      if ((rc0 = dalloc(h, &s.ins_i, cap)) || (rc0 = dalloc(h, &s.ins_j, cap)) ||
          (rc0 = dalloc(h, &s.ins_v, cap)) || (rc0 = dalloc(h, &s.ins_e, cap)))
        return rc0;
      s.ins_cap = (int)cap;
    }
    if (!s.breq_i) {  // big-pair deferral buffers (sized once per handle)
      const int bcap = 1 << 18;
      // per request at most max(BIG_MAXT, tiles along the larger cluster)
      const size_t per = (size_t)std::max(BIG_MAXT, cdiv(h->n, BIG_TILE) + 1);
      const size_t tiles = (size_t)BIG_BATCH * per;
      if ((rc0 = dalloc(h, &s.breq_i, bcap)) || (rc0 = dalloc(h, &s.breq_j, bcap)) ||
          (rc0 = dalloc(h, &s.breq_sa, bcap)) || (rc0 = dalloc(h, &s.breq_na, bcap)) ||
          (rc0 = dalloc(h, &s.breq_sb, bcap)) || (rc0 = dalloc(h, &s.breq_nb, bcap)) ||
          (rc0 = dalloc(h, &s.breq_exact, bcap)) || (rc0 = dalloc(h, &s.bsched, BS_SIZE)) ||
          (rc0 = dalloc(h, &s.bmax2, BIG_BATCH)) ||
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
  if (s.p32_max >= FP32_COORD_LIMIT) s.prec = HAC_PREC_F64;  // FP32 would overflow
  if (h->dense_k < 0 && s.linkage == LK_AVERAGE) h->dense_def = dense_default(s.d);
  cudaEventRecord(e1.e, st);
  CK(cudaEventSynchronize(e1.e));
  {
    float ms;
    cudaEventElapsedTime(&ms, e0.e, e1.e);
    ms_init = ms;
  }
  RoundCtl ctl;
  ctl.e1 = e1.e;
  ctl.e2 = e2.e;
  ctl.eq0 = eq0.e;
  ctl.eq1 = eq1.e;
  ctl.eb0 = eb0.e;
  ctl.eb1 = eb1.e;
  RoundTimes tm;
  tm.e0 = e0.e;
  tm.e3 = e3.e;
  const char *tr = getenv("HAC_TRACE");
  tm.trace = tr && tr[0] && tr[0] != '0';
  int round = 0;
  rc = run_rounds(h, opt, st, ctl, &tm, t0, &round);
  if (rc) return rc;
  ms_nn = tm.ms_nn;
  ms_merge = tm.ms_merge;
  ms_update = tm.ms_update;
  const int64_t naive = ctl.naive;
  Counters c{};
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
  rc = sort_records(h, st, h->dout, h->dout_round);
  if (rc) return rc;
  CK(cudaStreamSynchronize(st));
  h->n_merges = m;
  h->st.rounds = round;
  h->st.merges = c.nmerges;
  h->st.cluster_pairs = (int64_t)c.cluster_pairs;
  h->st.point_pairs = (int64_t)(c.point_pairs + c.big_pp - c.big_skip);
  h->st.nodes_visited = (int64_t)c.nodes;
  h->st.rechecks = (int64_t)c.rechecks;
  h->st.ms_init = ms_init;
  h->st.ms_query = ms_query;
  h->st.query_launches = qlaunch;
  h->st.leaf_tests = (int64_t)c.ltests;
  h->st.kernel_launches = h->launches;
  h->st.cache_hits = (int64_t)c.cache_hits;
  h->st.ms_big = ms_big;
  h->st.big_point_pairs = (int64_t)(c.big_pp - c.big_skip);
  h->st.big_launches = big_launch;
  h->st.cache_lw_entries = (int64_t)c.cache_lw;
  h->st.dense_k = s.dense ? s.dk : 0;
  h->st.dense_rounds = ctl.dense_rounds;
  h->st.dense_point_pairs = (int64_t)c.dense_pp;
  h->st.dense_rechecks = ctl.dense_rechecks;
  h->st.ms_dense = ctl.ms_dense;
  h->st.point_pairs += (int64_t)(c.dense_pp + c.dense_rq_pp);
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

}  // namespace hacg

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
  return abi_guard([&] { return create_common(points, false, n, d, dt, lk, out); });
}

int hac_create_device(const void *dev_points, int64_t n, int d, hac_dtype dt, hac_linkage lk,
                      hac_t *out) {
  return abi_guard([&] { return create_common(dev_points, true, n, d, dt, lk, out); });
}

int hac_run(hac_t h, const hac_opts *opts) {
  if (!h) return HAC_EINVAL;
  int rc = abi_guard([&] { return run_impl(h, opts); });
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

// Device address of the arena on the current device, looked up on every
// call (after the module is loaded this allocates nothing; a cached address
// could outlive a device reset that reloads the module elsewhere).  Host code
// must not use the symbol g_static_arena itself: on the host it only names a
// stand-in.
int static_arena(unsigned char **out) {
  void *q = nullptr;
  if (cudaGetSymbolAddress(&q, g_static_arena) != cudaSuccess || q == nullptr) {
    cudaGetLastError();
    return HAC_EDEVICE;
  }
  *out = (unsigned char *)q;
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
  cv.take(&s.blist, n);
  cv.take(&s.term, n);
  cv.take(&s.pair_lo, n / 2 + 1);
  cv.take(&s.pair_hi, n / 2 + 1);
  cv.take(&s.pair_key, n / 2 + 1);
  cv.take(&s.m_a, n);
  cv.take(&s.m_b, n);
  cv.take(&s.m_size, n);
  cv.take(&s.m_round, n);
  cv.take(&s.m_h, n);
  int base = 0, chbase = 0;
  tree_layout(s, (int)n, &base, &chbase);
  cv.take(&s.nclo, (size_t)base * dp);
  cv.take(&s.nchi, (size_t)base * dp);
  cv.take(&s.nhmin, (size_t)base * dp);
  cv.take(&s.nlmax, (size_t)base * dp);
  cv.take(&s.nnmin, (size_t)base);
  cv.take(&s.ninlo, (size_t)base);
  cv.take(&s.ninhi, (size_t)base);
  cv.take(&s.nch, (size_t)chbase);
  cv.take(&s.pbkt, n);
  cv.take(&s.mkey, n);
  cv.take(&s.tinfo, TI_SIZE);
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

// Algorithm 1 with the state carved from the arena: the same layout, rounds
// and canonical record sort as hac_run (no events, no host allocation);
// writes the dendrogram to `dev_out`
int static_run(hac_ctx &h, const hac_opts &opt, cudaStream_t st, hac_merge *dev_out) {
  State &s = h.s;
  const auto t0 = std::chrono::steady_clock::now();
  int rc = h.dt == HAC_F32 ? init_layout<float>(&h, st) : init_layout<double>(&h, st);
  if (rc) return rc;
  if (s.p32_max >= FP32_COORD_LIMIT) s.prec = HAC_PREC_F64;  // FP32 would overflow
  RoundCtl ctl;  // no events: nothing is created here
  int rounds = 0;
  rc = run_rounds(&h, opt, st, ctl, nullptr, t0, &rounds);
  if (rc) return rc;
  Counters c{};
  CK(cudaMemcpyAsync(&c, s.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (c.nmerges != h.n - 1) return HAC_EINTERNAL;
  rc = sort_records(&h, st, dev_out, h.dout_round);
  if (rc) return rc;
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
  h.s.noprune = (opt.flags & HAC_FLAG_NO_PRUNE) ? 1 : 0;
  h.dense_k = 0;  // the fixed array has no room for the dense matrix
  Carver cv{arena, 0, kStaticArenaBytes, true};
  if (!carve_state(h, cv)) return HAC_EINVAL;
  const cudaStream_t st = (cudaStream_t)opt.stream;
  rc = abi_guard([&] { return static_run(h, opt, st, dev_out); });
  if (rc == HAC_EDEVICE) cudaGetLastError();
  return rc;
}
