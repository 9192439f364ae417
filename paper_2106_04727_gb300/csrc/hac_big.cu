// Big cluster pairs (Algorithm 4's evaluations that are too large for one
// warp): the batch schedule, duplicate dropping, and the fold of the tiles'
// partial results into the cache tables and this round's result table.  The
// evaluation kernels themselves are in hac_big.cuh.
#include "hac_big.cuh"

namespace {

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
    s.bmax2[t] = 0;  // +0.0f
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

}  // namespace

namespace hacg {

int big_prepare(const State &s, int r0, int m, cudaStream_t st) {
  k_big_dedup<<<1, BIG_BATCH, 0, st>>>(s, r0, m);
  k_big_tiles<<<1, BIG_BATCH, 0, st>>>(s, r0, m);
  CK(cudaGetLastError());
  return HAC_OK;
}

int launch_big(const State &s, int r0, cudaStream_t st) {
  return s.linkage == LK_COMPLETE ? launch_big_complete(s, r0, st)
                                  : launch_big_average(s, r0, st);
}

int big_finish(const State &s, int r0, int m, cudaStream_t st) {
  k_big_final<<<cdiv(m, 8), 256, 0, st>>>(s, r0, m);
  CK(cudaGetLastError());
  return HAC_OK;
}

}  // namespace hacg
