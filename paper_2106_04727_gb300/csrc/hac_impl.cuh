// Host and device internals shared by the library's translation units
// (core rounds, big-pair evaluation, serving); not part of the C ABI.
#pragma once

#include "hac.h"
#include "hac_internal.cuh"
#include "hac_dev.cuh"

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <new>
#include <vector>

namespace hacg {

constexpr int TPB = 256;

__host__ __device__ inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// pair-distance cache slots (Section 5): the write protocol
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
__device__ inline bool slot_put(const State &s, size_t idx, unsigned long long cur,
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
__device__ inline void cache_insert(const State &s, int owner, int nbr, int nbr_gen, double v, float e) {
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

// ---------------------------------------------------------------------------
// big pairs: sizes of the GPU-wide evaluation
// ---------------------------------------------------------------------------
constexpr int BIG_TPB = 256;       // threads per tile
constexpr int BIG_TILE = BIG_TPB * 2;  // narrowest tile along the larger cluster
constexpr int BIG_MAXT = 32768; // tiles per request at most (chunks widen to fit)
constexpr int BIG_BATCH = 1024;    // requests per batch (one scan block of 32 warps)

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

}  // namespace hacg

// ---------------------------------------------------------------------------
// instance
// ---------------------------------------------------------------------------
struct hac_ctx {
  hacg::State s{};
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
  int cache_alloc_slots = 0;  // slots per cluster the cache tables were allocated for
  int64_t lay_n = 0;          // points in the current layout (all n for one instance)
  // pairs of at least this many point pairs go to the GPU-wide evaluation
  // (FP32 / FP64 values); HAC_BIG_PAIRS / HAC_BIG_PAIRS_F64 override them
  long long big_pairs = hacg::BIG_PAIRS, big_pairs64 = hacg::BIG_PAIRS_F64;
  long long warp_budget = hacg::WARP_BUDGET;  // HAC_WARP_BUDGET overrides it
  int brute_env = -1;   // HAC_BRUTE: -1 unset, 0 never, 1 whenever allowed
  // average linkage switches to the dense matrix once at most this many
  // clusters are active (HAC_DENSE_K overrides it; 0 = never)
  int64_t dense_k = -1;  // -1: the default for the instance
  int64_t dense_def = 0;  // that default for the current run (dense_default)
  int64_t dense_cap = 0; // matrix dimension the buffers were allocated for
  int64_t launches = 0;  // kernels launched in the current run
  int ocur = 0, pcur = 0;
  bool done = false;
  int64_t n_merges = 0;
  hac_stats_t st{};
  hac_merge *dout = nullptr;        // canonical dendrogram (device)
  int32_t *dout_round = nullptr;
};

namespace hacg {

template <typename T>
int dalloc(hac_ctx *h, T **p, size_t count) {
  if (count == 0) count = 1;
  void *q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return HAC_ENOMEM;
  }
  try {
    h->allocs.push_back(q);
  } catch (...) {
    cudaFree(q);
    return HAC_ENOMEM;
  }
  h->bytes += (int64_t)(count * sizeof(T));
  *p = (T *)q;
  return HAC_OK;
}

// Runs f() and turns a C++ exception (a failed host allocation, a thread
// that could not start) into a status code, so that none crosses the C ABI.
template <typename F>
int abi_guard(F &&f) noexcept {
  try {
    return f();
  } catch (const std::bad_alloc &) {
    return HAC_ENOMEM;
  } catch (...) {
    return HAC_EINTERNAL;
  }
}

void free_all(hac_ctx *h);
int pad_dim(int d);
int alloc_state(hac_ctx *h);

#define CK(x)                                \
  do {                                       \
    cudaError_t e_ = (x);                    \
    if (e_ != cudaSuccess) return HAC_EDEVICE; \
  } while (0)

// SM count of the current device (looked up once per device)
int device_sms();

// grid of a grid-stride kernel: one thread per work item, at most 64 blocks
// per SM
inline int grid_for(int64_t work, int tpb) {
  int64_t g = (work + tpb - 1) / tpb;
  if (g < 1) g = 1;
  const int64_t cap = (int64_t)device_sms() * 64;
  if (g > cap) g = cap;
  return (int)g;
}

// tree over the first K clusters of `order`; stable LSD radix sort of the
// first m keys/values in h->keys[0]/vals[0] (returns the buffer holding the
// result); bits needed for values up to maxval
int build_tree(hac_ctx *h, const int32_t *order, int K, cudaStream_t st);
int radix_sort(hac_ctx *h, int m, int bits, cudaStream_t st);
int bits_for(int64_t maxval);

// Per-round timing / counters of round_step (events may be null: no timing)
struct RoundCtl {
  cudaEvent_t e1 = nullptr, e2 = nullptr, eq0 = nullptr, eq1 = nullptr, eb0 = nullptr,
              eb1 = nullptr;
  double ms_query = 0, ms_big = 0;
  int64_t qlaunch = 0, big_launch = 0, searches = 0;
  int64_t naive = 0;  // terminals x (active clusters - 1), summed over rounds
  int big_iters = 0, big_reqs = 0;
  double ms_dense = 0;         // device time of the dense sweep
  int64_t dense_launches = 0;  // launches of the dense phase's kernels
  int64_t dense_rounds = 0;    // rounds run on the dense matrix
  int64_t dense_rechecks = 0;  // matrix entries re-scored in FP64
};

int round_step(hac_ctx *h, cudaStream_t st, int round, int K, int nterm, RoundCtl &ctl,
               int *npairs_out);

// big-pair evaluation of requests [r0, r0 + m) (hac_big*.cu): drop duplicate
// requests and build the tile schedule; run the evaluation kernels; fold the
// tiles and fill the cache tables and this round's result table
int big_prepare(const State &s, int r0, int m, cudaStream_t st);
int launch_big(const State &s, int r0, cudaStream_t st);
int big_finish(const State &s, int r0, int m, cudaStream_t st);
int launch_big_complete(const State &s, int r0, cudaStream_t st);
int launch_big_average(const State &s, int r0, cudaStream_t st);

// dense phase (hac_dense.cu): whether this round should run on the matrix
// (entering it if needed: allocation, the all-pairs sweep); the
// nearest-neighbour search of the round's terminals on the matrix (with the
// FP64 re-score of near ties in the FP32 mode); the Lance-Williams update of
// the matrix after the round's merges (before the compaction)
int64_t dense_default(int d);
int dense_maybe_enter(hac_ctx *h, cudaStream_t st, int K, RoundCtl &ctl);
int dense_search(hac_ctx *h, cudaStream_t st, int K, int nterm, RoundCtl &ctl);
int dense_update(hac_ctx *h, cudaStream_t st, int round, int K, int npairs);

}  // namespace hacg
