// Serving and batched runs: continuous batching of independent clusterings
// on engines that share one device state each (internal to the library; the
// C ABI is in include/hac.h).
#include "hac_impl.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

using namespace hacg;

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
                               const int32_t *sorted, const uint64_t *skey, int32_t *order,
                               int K, int nterm,
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
    s.mkey[c] = skey[p] & ((1ull << 40) - 1);  // the Morton key below the batch rank
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
        (rc = dalloc(&h, &s.bmax2, BIG_BATCH)) ||
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
        s, (const float *)e.stage, m, e.d_ai, na, h.vals[sc], h.keys[sc], ord, e.K, e.nterm, e.P,
        h.pcur, e.round, ward);
  else
    k_admit_layout<double><<<grid_for(m, TPB), TPB, 0, st>>>(
        s, (const double *)e.stage, m, e.d_ai, na, h.vals[sc], h.keys[sc], ord, e.K, e.nterm, e.P,
        h.pcur, e.round, ward);
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

void engine_loop_body(hac_server *srv, Engine *ep) {
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

// The engine thread: an exception (a failed host allocation) fails the
// engine's requests with a status instead of ending the process.
void engine_loop(hac_server *srv, Engine *ep) {
  try {
    engine_loop_body(srv, ep);
  } catch (const std::bad_alloc &) {
    engine_fail(srv, *ep, HAC_ENOMEM);
  } catch (...) {
    engine_fail(srv, *ep, HAC_EINTERNAL);
  }
}

}  // namespace

static int hac_server_create_body(int64_t points_per_engine, const hac_opts *opts,
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

static int hac_submit_body(hac_server_t srv, const void *points, int64_t n, int d, hac_dtype dt,
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
  double lo[MAXD], hi[MAXD], amax = 0.0;
  for (int k = 0; k < d; ++k) {
    lo[k] = INFINITY;
    hi[k] = -INFINITY;
  }
  for (int64_t i = 0; i < n * d; ++i) {
    const double x =
        dt == HAC_F32 ? (double)((const float *)points)[i] : ((const double *)points)[i];
    if (!std::isfinite(x)) return HAC_EINVAL;
    lo[i % d] = std::min(lo[i % d], x);
    hi[i % d] = std::max(hi[i % d], x);
    amax = std::max(amax, std::fabs(x));
  }
  // the FP32 copy is the input itself (FP32 input) or the recentred points
  if (srv->opt.precision == HAC_PREC_F32_RECHECK) {
    double ext = 0.0;
    for (int k = 0; k < d; ++k) ext = std::max(ext, 0.5 * (hi[k] - lo[k]));
    if ((dt == HAC_F32 ? amax : ext) >= FP32_COORD_LIMIT) return HAC_EINVAL;
  }
  // owned here until published in srv->reqs (a throwing copy or insert frees it)
  std::unique_ptr<SrvReq> r(new (std::nothrow) SrvReq());
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
  if (srv->err) return srv->err;
  const uint64_t tk = srv->next_ticket;
  if (n == 1) {  // nothing to merge
    r->ticket = tk;
    r->status = HAC_OK;
    r->t_done = r->t_submit;
    srv->reqs.emplace(tk, r.get());
    r.release();
    ++srv->next_ticket;
    *ticket = tk;
    return HAC_OK;
  }
  auto it = srv->engines.find(key);
  Engine *e = it == srv->engines.end() ? nullptr : it->second;
  if (!e) {
    // first request of this kind: its engine (device memory for cap points);
    // everything that can throw happens before its thread starts, so a
    // failure leaves no running engine unreachable from srv
    e = new (std::nothrow) Engine();
    if (!e) return HAC_ENOMEM;
    int rc = engine_init(*e, lk, d, dt, srv->cap, srv->opt);
    std::map<int, Engine *>::iterator slot;
    if (!rc) {
      try {
        slot = srv->engines.emplace(key, nullptr).first;
      } catch (...) {
        rc = HAC_ENOMEM;
      }
    }
    if (!rc) {
      try {
        e->thr = std::thread(engine_loop, srv, e);
      } catch (...) {
        srv->engines.erase(slot);
        rc = HAC_ENOMEM;
      }
    }
    if (rc) {
      engine_free(e);
      delete e;
      return rc;
    }
    slot->second = e;
  }
  // publish: the map insert and the queue append are undone together
  r->ticket = tk;
  r->eng = e;
  auto ri = srv->reqs.emplace(tk, r.get()).first;
  try {
    e->queue.push_back(r.get());
  } catch (...) {
    srv->reqs.erase(ri);
    return HAC_ENOMEM;
  }
  r.release();
  ++srv->next_ticket;
  *ticket = tk;
  g.unlock();
  srv->cv.notify_all();
  return HAC_OK;
}
}  // namespace

static int hac_cancel_body(hac_server_t srv, uint64_t ticket) {
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

static int hac_poll_body(hac_server_t srv, uint64_t ticket, hac_merge *out, int64_t cap,
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

static int hac_server_wait_body(hac_server_t srv, uint64_t ticket, double timeout_s) {
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

static int hac_server_stats_body(hac_server_t srv, hac_server_stats_t *out) {
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

static void hac_server_destroy_body(hac_server_t srv) {
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
static int hac_run_batch_body(hac_t *hs, int count, const hac_opts *opts) {
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

// ---------------------------------------------------------------------------
// C ABI: each entry point runs its body under abi_guard, so that a failed host
// allocation or thread start returns a status instead of ending the process.
// ---------------------------------------------------------------------------

extern "C" int hac_server_create(int64_t points_per_engine, const hac_opts *opts,
                                 hac_server_t *out) {
  return abi_guard([&] { return hac_server_create_body(points_per_engine, opts, out); });
}

extern "C" int hac_submit(hac_server_t srv, const void *points, int64_t n, int d, hac_dtype dt,
                          hac_linkage lk, double timeout_s, uint64_t *ticket) {
  return abi_guard([&] { return hac_submit_body(srv, points, n, d, dt, lk, timeout_s, ticket); });
}

extern "C" int hac_cancel(hac_server_t srv, uint64_t ticket) {
  return abi_guard([&] { return hac_cancel_body(srv, ticket); });
}

extern "C" int hac_poll(hac_server_t srv, uint64_t ticket, hac_merge *out, int64_t cap,
                        int64_t *n_written, double *latency_ms) {
  return abi_guard([&] { return hac_poll_body(srv, ticket, out, cap, n_written, latency_ms); });
}

extern "C" int hac_server_wait(hac_server_t srv, uint64_t ticket, double timeout_s) {
  return abi_guard([&] { return hac_server_wait_body(srv, ticket, timeout_s); });
}

extern "C" int hac_server_stats(hac_server_t srv, hac_server_stats_t *out) {
  return abi_guard([&] { return hac_server_stats_body(srv, out); });
}

extern "C" int hac_run_batch(hac_t *hs, int count, const hac_opts *opts) {
  return abi_guard([&] { return hac_run_batch_body(hs, count, opts); });
}

extern "C" void hac_server_destroy(hac_server_t srv) {
  try {
    hac_server_destroy_body(srv);
  } catch (...) {
  }
}
