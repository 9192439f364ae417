// Internal declarations of the GB300 HAC library (not part of the C ABI).
//
// Device state of one instance, laid out struct-of-arrays and indexed by
// cluster id (cid).  A merged cluster keeps min(cid_a, cid_b) (ParChain,
// Section 1 footnote), so every per-cluster array is sized n and a merge only
// retires the larger cid: no ids are ever allocated.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hacg {

constexpr int MAXD = 16;     // largest supported dimension
constexpr int FAN = 32;      // range-query tree: at most this many children per node
constexpr int MAXLEV = 10;   // tree levels of any n < 2^31 (tree_caps)
constexpr unsigned long long PRED_EMPTY = ~0ull;

// Device-side counters of one instance.
struct Counters {
  int32_t npairs;    // reciprocal pairs found this round
  int32_t nterm;     // terminals for the next search
  int32_t nactive;   // active clusters
  int32_t nmerges;   // merges made so far
  int32_t err;       // sticky error bits (ERR_*)
  int32_t nins;      // pair distances queued for the cache this round
  int32_t nbreq;     // big-pair requests queued by the search
  int32_t npend;     // terminals waiting for their big pairs
  int32_t ndone;     // instances that finished this round (entries of done_list)
  unsigned long long cluster_pairs, point_pairs, nodes, rechecks, searches, ltests, prows;
  unsigned long long cache_hits, cache_lw;
  unsigned long long big_pp, big_exact;  // point pairs / FP64 requests of the GPU-wide evaluation
  unsigned long long big_skip;  // of those, pairs complete linkage skipped by box bounds
  int32_t nrq;       // dense phase: pairs listed for an FP64 re-score this pass
  unsigned long long dense_pp, dense_rq_pp;  // dense phase: sweep / re-score point pairs
};

enum : int32_t { ERR_NONFINITE = 1, ERR_NO_NN = 2, ERR_STACK = 4, ERR_WINDOW = 8, ERR_TREE = 16 };

constexpr unsigned long long CKEY_EMPTY = ~0ull;
constexpr long long CACHE_MIN_PAIRS = 64;  // smaller pairs are cheaper to recompute
constexpr int CACHE_MAX_SLOTS = 256;

// cache key of neighbour `cid` at generation `gen`
__host__ __device__ inline unsigned long long ckey_of(int cid, int gen) {
  return ((unsigned long long)(unsigned)cid << 32) | (unsigned)gen;
}

// Everything a round's kernels read or write.  Arrays with [2] are double
// buffered across the point re-layout; `cur` selects the live one.
struct State {
  int64_t n;
  int d, dp;            // dimension and padded row stride (2, 4, 8 or 16)
  int linkage, prec;
  double abs_slack;     // absolute pruning slack (coordinate scale * 2^-18)
  float coord_scale;    // largest |coordinate| after recentring
  double p32_max;       // largest |coordinate| of the FP32 point copy
  float delta_pts;      // absolute error term of an FP32 point distance (0 for FP32 input)
  int pts32_exact;      // the FP32 point copy is the FP32 input itself
  // points, permuted into cluster-contiguous segments
  double *p64[2];
  float *p32[2];
  int32_t *plab[2];     // owning cid of each permuted point
  int32_t *seg[2];      // segment start of each cid
  // per-cid cluster state
  int32_t *csize;
  double *csum;         // coordinate sums (FP64), n x dp
  double *csq;          // sums of squared norms (FP64): a rigorous variance bound
  double *sse;          // sums of squared deviations from the centroid (FP64), merged
                        // exactly as the paper's variance update: avg-2 distances
  double *cent;         // centroids (FP64), n x dp
  float *cent32;        // centroid rounded to FP32, n x dp
  float *blo, *bhi;     // point bounding box, rounded outward to FP32, n x dp
  int32_t *succ;        // nearest-neighbour successor, -1 = terminal
  unsigned long long *pred;  // (f32 key rounded up) << 32 | cid, by WriteMin
  int32_t *mround;      // round in which the cid last took part in a merge
  int32_t *isterm;      // round in which the cid is a terminal
  uint8_t *alive;
  int32_t *rootof;      // retired cid -> surviving cid of its merge
  int32_t *reloff;      // retired cid -> offset of its points in the merged segment
  int32_t *osize;       // size of each cid just before this round's merge
  int32_t *partner;     // the other cid of this round's merge
  int32_t *gen;         // generation of each cid, bumped whenever it takes part in a merge
  // pair-distance cache (Section 5): cache_slots entries per cid; key =
  // neighbour cid << 32 | neighbour generation; value = distance (D units)
  // and its absolute error bound (0 for FP64 values)
  int cache_slots;
  int noprune;          // range-query ablation (HAC_FLAG_NO_PRUNE)
  unsigned long long *ckey;
  double *cval;
  float *cerr;
  // partial entries (Lance-Williams with one side unknown): 0 = the value is
  // D(owner, neighbour); c > 0 = it is D(first c points of the owner,
  // neighbour); c < 0 = D(last -c points of the owner, neighbour)
  int32_t *cpart;
  int ins_cap;          // queue of evaluated pairs to insert after the search
  int32_t *ins_i, *ins_j;
  double *ins_v;
  float *ins_e;
  // big pairs deferred by the search to the GPU-wide evaluation kernel
  int breq_cap;
  int32_t *breq_i, *breq_j, *breq_sa, *breq_na, *breq_sb, *breq_nb;
  uint8_t *breq_exact;   // 1 = FP64 value wanted, 0 = FP32 estimate
  // completion of a partial entry: the request evaluates the missing points
  // only; `cov` more points of side a are already covered by `base` (the sum
  // of their distances, average; their distance, complete) with error `berr`
  double *breq_base;
  int32_t *breq_cov;
  float *breq_berr;
  int32_t *bsched;       // tile schedule of the current batch (per-kind lists)
  int32_t *bmax2;        // complete linkage: largest squared distance found so far
                         // for each request of the batch (FP32 bits)
  double *bpart;         // per-tile partial results of the current batch
  int32_t *pend[2];      // terminals whose search deferred a pair
  // this round's big-pair results by unordered cid pair (cleared every round):
  // the re-run search reads them here even when a cache table had no room
  int side_cap;          // power of two
  unsigned long long *side_key;  // lo << 32 | hi, ~0 = empty
  double *side_val;
  float *side_err;
  // instances sharing this state (a server engine clusters many at once;
  // hac_run is the one-instance case): instance of each cid / position,
  // tree-node instance ranges, and per-instance parameters and progress
  int32_t *inst;        // instance slot of each cid
  int32_t *qinst;       // admission number of the instance at each position; it
                        // never decreases along `order`, so tree nodes keep tight
                        // [ninlo, ninhi] ranges of it
  int32_t *ninlo, *ninhi;
  int32_t *iseq;        // admission number of each instance slot
  int32_t *done_list;   // slots of the instances that finished this round
  int max_inst;
  float *islack;        // absolute pruning slack (coordinate scale * 2^-18)
  float *iscale;        // largest |coordinate| after recentring
  float *idpts;         // error term of FP32 point distances (0 for FP32 input)
  int32_t *irec;        // first merge-record slot (= first cid of the instance)
  int32_t *irecn;       // merge records written
  int32_t *iact;        // active clusters left
  int32_t *idone;       // 1 once one cluster is left
  int32_t *pos;         // position of each active cid in `order`
  double *Ekey;         // nearest-neighbour key of each terminal (linkage key space)
  int32_t *Ecid;
  // position-ordered copies of the search record of every active cluster,
  // rebuilt at each compaction so that a leaf scan reads 32 contiguous records
  float *q32, *qblo, *qbhi;  // FP32 centroid and box, K x dp
  double *q64;               // FP64 centroid, K x dp
  int32_t *qsz, *qseg;       // size and segment start
  float *qvar;               // variance (mean squared distance to the centroid), rounded up
  // lists
  int32_t *order[2];    // active cids in spatial order
  int32_t *term;        // terminal cids
  int32_t *blist;       // terminals left to the FP64 re-score of the exhaustive search
  // candidate lists of the exhaustive scan for average linkage (by position)
  int32_t *lpos, *lcnt;
  float *llb, *lub;
  int32_t *pair_lo, *pair_hi;
  double *pair_key;
  // dendrogram records
  int32_t *m_a, *m_b, *m_size, *m_round;
  double *m_h;
  // range-query tree, rebuilt every round over the active clusters in
  // position order: a level-0 node (a bucket) is a run of at most 32
  // positions, a level-L node a run of at most 32 level-(L-1) nodes, each run
  // one cell of the Morton-key hierarchy where the data allow (tree_caps,
  // build_tree).  Level L node j lives at index lvl_base[L] + j; its children
  // are [nch[chb[L] + j], nch[chb[L] + j + 1]) (positions for L = 0).
  float *nclo, *nchi;   // box of the children's FP32 centroids, nodes x dp
  float *nhmin, *nlmax; // min over children of box hi / max of box lo, nodes x dp
  int32_t *nnmin;       // min child cluster size
  int32_t *nch;         // first child of every node, plus one end entry per level
  int32_t *pbkt;        // bucket (level-0 node) of every position
  uint64_t *mkey;       // Morton key of each cluster's position at layout (cid)
  int32_t *tinfo;       // node count of every level, then TI_TOP, TI_FIXED
  int32_t lvl_base[MAXLEV + 1];
  int32_t chb[MAXLEV + 1];
  // dense phase (average linkage, one instance): once the active clusters
  // fit, the whole matrix of their pair distances (the Section 5 cache with
  // room for every pair), filled by one all-pairs sweep of the points and
  // updated by Lance-Williams after every round.  Each entry is kept as the
  // exact sum of its point distances (128-bit fixed point, so a merge adds
  // sums exactly) and as the mean distance that sum gives (FP64); in the FP32
  // mode an FP32-derived estimate carries the sign bit of the mean (its
  // magnitude is the estimate) and the top bit of the sum.
  int dense;            // 1 once the instance runs on the matrix
  int dk;               // matrix dimension: active clusters at the switch
  int dexp;             // exponent of the fixed-point unit of the sweep sums
  int dsk;              // the FP32 sweep scales coordinates by 2^dsk
  double dsl, dsh;      // 2^dexp and 2^(64 + dexp): a sum's low and high word scales
  double *dinv;         // 1 / size of the cluster at each matrix index
  double *dmat;         // dk x dk, row-major; diagonal +inf
  unsigned long long *dsum;  // 128-bit fixed-point sums of point distances of the
                             // pairs i < j, packed upper triangle (four limb words
                             // per pair; the top bit of the last marks an estimate)
  int32_t *dq;          // this round: matrix index of each active position
  uint8_t *dqm;         // after the merges: 1 if that cluster merged this round
  int32_t *didx;        // cid -> matrix index (the cid's position at the switch)
  int32_t *dcid;        // matrix index -> cid
  int drq_cap;          // FP64 re-score queue (pairs, lower index first)
  int32_t *drq_a, *drq_b, *drq_pre;
  unsigned long long *drq_acc;  // fixed-point sums, two words per pair
  int32_t *dpend[2];    // terminals whose search waits for re-scored pairs
  // scan scratch
  int32_t *bsum;        // 3 x nblocks block partial sums
  Counters *ctr;
  int cur;
};

// Query kernel arguments (by value).
struct QueryArgs {
  int d, linkage, round, K, nterm;
  double abs_slack;
  float coord_scale, delta_pts;
  const int32_t *term, *order, *pos, *csize, *seg;
  const double *cent, *p64;
  const float *cent32, *blo, *bhi, *p32;
  const unsigned long long *pred;
  const float *q32, *qblo, *qbhi;
  const double *q64;
  const int32_t *qsz, *qseg;
  const float *qvar;
  const double *sse;
  const float *nclo, *nchi, *nhmin, *nlmax;
  const int32_t *nnmin, *nch, *pbkt, *tinfo;
  int32_t lvl_base[MAXLEV + 1];
  int32_t chb[MAXLEV + 1];
  double *Ekey;
  int32_t *Ecid;
  Counters *ctr;
  // instances
  const int32_t *inst, *qinst, *ninlo, *ninhi;
  const float *islack, *iscale, *idpts;
  // pair-distance cache
  int cache_slots, ins_cap;
  const unsigned long long *ckey;
  const double *cval;
  const float *cerr;
  const int32_t *cpart;
  const int32_t *gen;
  int32_t *ins_i, *ins_j;
  double *ins_v;
  float *ins_e;
  // big-pair deferral (needs the cache): 0 = evaluate big pairs in the warp
  int defer;
  long long big_pairs, big_pairs64;
  long long warp_budget;  // point pairs a search evaluates itself before deferring more
  int noprune;            // ablation: every cluster of the instance is a candidate
  int side_cap;
  const unsigned long long *side_key;
  const double *side_val;
  const float *side_err;
  int breq_cap;
  int32_t *breq_i, *breq_j, *breq_sa, *breq_na, *breq_sb, *breq_nb;
  uint8_t *breq_exact;
  double *breq_base;
  int32_t *breq_cov;
  float *breq_berr;
  int32_t *pend_out;
  // candidate lists of the exhaustive scan (average linkage, high dimension),
  // indexed by the terminal's position: lcnt < 0 (or lcnt null) = use the tree
  int lcap;
  const int32_t *lpos, *lcnt;
  const float *lub;
};

// pairs of at least this many point pairs are evaluated by the whole GPU
constexpr long long BIG_PAIRS = 1ll << 16;
// FP64 point pairs cost ~64x more on this part: hand them over much earlier
constexpr long long BIG_PAIRS_F64 = 1ll << 13;
// point pairs one search evaluates in its own warp before it hands every
// further pair of at least BIG_MIN_PAIRS to the GPU-wide kernels
constexpr long long WARP_BUDGET = 1ll << 18;
constexpr long long BIG_MIN_PAIRS = 1ll << 12;
constexpr int SIDE_PROBES = 64;

__host__ __device__ inline unsigned side_hash(int lo, int hi, int cap) {
  return ((unsigned)lo * 2654435761u ^ (unsigned)hi * 0x85EBCA77u) & (unsigned)(cap - 1);
}

// error term stored with every cached FP32 estimate (0 marks an FP64 value)
constexpr float EST_MARK = 1e-30f;

// linkages whose cluster distance is O(1) from centroids, variances and
// sizes (Ward, avg-2): no point pairs, no cache, no point re-layout
__host__ __device__ inline bool closed_form(int linkage) { return linkage >= 2; }

// Node capacities of the range-query tree for K active clusters: level 0
// holds at most ceil(K / 8) + 1 buckets and level L at most
// ceil(cap[L-1] / 8) + 1 nodes; a level whose Morton-cell grouping would
// exceed its capacity (or whose keys are out of order) is cut into fixed runs
// of 32 instead, which always fit.  The last level has at most 32 nodes.
// Returns the number of levels (<= MAXLEV + 1).
__host__ __device__ inline int tree_caps(int K, int *cap) {
  int c = (int)(((long long)K + 7) / 8) + 1, L = 0;  // K + 7 may overflow an int
  if (cap) cap[0] = c;
  while (c > FAN) {
    c = (c + 7) / 8 + 1;
    ++L;
    if (cap) cap[L] = c;
  }
  return L + 1;
}

// The FP32 paths take coordinates (of the FP32 copy) below 2^40: squared
// differences then stay below 2^86 even for d = 16 and Ward's weights.  Runs
// over larger coordinates take the FP64 path in either precision mode.
constexpr double FP32_COORD_LIMIT = 1099511627776.0;  // 2^40

// tinfo entries after the per-level node counts
constexpr int TI_TOP = MAXLEV + 1;    // lowest level with at most 32 nodes (the root's children)
constexpr int TI_FIXED = MAXLEV + 2;  // bit L: level L was cut into fixed runs of 32
constexpr int TI_SIZE = MAXLEV + 3;

// launches the nearest-neighbour query of every terminal (hac_query.cu)
cudaError_t launch_query(const QueryArgs &a, int dp, int prec, cudaStream_t s);
// the same search done exhaustively with tiles of cluster records staged in
// shared memory (hac_brute.cu): closed-form linkages, FP32 + FP64 re-score,
// one instance; uses pend_out (nterm entries) and ctr->npend (zeroed first)
cudaError_t launch_brute(const QueryArgs &a, int dp, cudaStream_t s);
// candidate lists for average linkage: every terminal scans every active
// cluster's record (tiles in shared memory) and lists, by position, those
// whose centroid lower bound is within its least Jensen upper bound
// (at most lcap; lcnt = -1 if more, and the terminal searches the tree)
constexpr int BL_CAP = 256;
cudaError_t launch_cand_avg(const QueryArgs &a, int32_t *lpos, float *llb, int32_t *lcnt,
                            float *lub, int dp, cudaStream_t s);

}  // namespace hacg
