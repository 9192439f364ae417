/*
 * hac.h -- C ABI of the GB300 nearest-neighbor-chain HAC library.
 *
 * The library computes the exact hierarchical agglomerative clustering
 * dendrogram of n points in d <= 16 dimensions under complete, average
 * (Euclidean, "avg-1"), Ward, or average linkage on squared Euclidean
 * distances ("avg-2") (ParChain, arXiv 2106.04727, Table 1),
 * with the parallel nearest-neighbor-chain rounds of Algorithm 1: every round,
 * each terminal cluster finds its nearest active cluster (Algorithms 2-4,
 * range-pruned), all reciprocal-nearest-neighbor pairs merge at once, and the
 * cluster state is refreshed.  All compute runs in the library's own sm_103a
 * CUDA kernels on the current CUDA device; there is no CPU fallback.
 *
 * Conventions (fixed by the paper, Section 1 footnote and Fig. 1 caption):
 *   - a cluster's id (cid) is the smallest input index among its points;
 *     a merged cluster keeps min(cid_a, cid_b);
 *   - ties are broken lexicographically: a cluster's nearest neighbour is the
 *     candidate of least (distance, cid).
 *
 * Errors: every int-returning call returns HAC_OK (0) or a negative HAC_E*
 * code; hac_strerror() names it.  No call aborts the process.  A call that
 * fails leaves the handle usable unless it returns HAC_EDEVICE (then only
 * hac_destroy is valid).
 *
 * Threading: one handle must not be used by two host threads at once;
 * distinct handles are independent.
 */
#ifndef HAC_H_
#define HAC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define HAC_OK 0
#define HAC_EINVAL (-1)    /* bad argument: null pointer, n < 1, d outside 1..16,
                              non-finite coordinate, unknown enum value */
#define HAC_ENOMEM (-2)    /* device or host allocation failed */
#define HAC_EDEVICE (-3)   /* a CUDA call failed; the handle is unusable */
#define HAC_ETIMEOUT (-4)  /* opts->timeout_s or opts->max_rounds reached */
#define HAC_EPENDING (-5)  /* no dendrogram yet: hac_run has not completed */
#define HAC_ECAP (-6)      /* output buffer smaller than n - 1 records */
#define HAC_EINTERNAL (-7) /* an internal consistency check failed */
#define HAC_ECANCELED (-8) /* a served request was cancelled (hac_cancel) */

typedef struct hac_ctx *hac_t; /* opaque; owns all device memory of one instance */

/* HAC_AVERAGE_SQ: average linkage with the squared Euclidean metric ("avg-2",
 * Table 1): the mean squared point distance, reported as is (its heights are
 * in squared units); computed in O(1) from centroids, per-point variances and
 * sizes. */
typedef enum { HAC_COMPLETE = 0, HAC_AVERAGE = 1, HAC_WARD = 2, HAC_AVERAGE_SQ = 3 } hac_linkage;
typedef enum { HAC_F32 = 0, HAC_F64 = 1 } hac_dtype;
typedef enum {
  HAC_PREC_F64 = 0,         /* every distance in FP64 */
  HAC_PREC_F32_RECHECK = 1  /* bulk distances in FP32; candidates within the
                               stated FP32 error bound of the minimum are
                               re-scored in FP64, so nearest neighbours (and
                               hence the tree) are the FP64 ones.  Ward and
                               avg-2 tree searches (O(d) closed forms) run in
                               FP64 in both modes; their exhaustive scans
                               (d > 8) use the FP32 bulk.  hac_run and
                               hac_run_static run inputs whose FP32 copy has
                               a coordinate of 2^40 or more (FP32 input: the
                               input; FP64 input: the recentred points) in
                               FP64; an FP32 server refuses them (HAC_EINVAL) */
} hac_precision;

/* One dendrogram node: clusters cid_a < cid_b merged at `height` into a
 * cluster of `size` points (Algorithm 1, merge step). */
typedef struct {
  int64_t cid_a;
  int64_t cid_b;
  double height;
  int64_t size;
} hac_merge;

typedef struct {
  int precision;      /* hac_precision; default HAC_PREC_F64 */
  int cache_slots;    /* per-cluster pair-distance cache slots (Section 5), complete and
                         average only (at most 256); 0 = off.  The first run with a value
                         larger than any before allocates the tables (n * slots * 24
                         bytes) in the handle, releasing the smaller ones; a smaller value
                         reuses them.  hac_run_static ignores it. */
  int64_t max_rounds; /* 0 = unlimited; else HAC_ETIMEOUT after this many rounds */
  double timeout_s;   /* 0 = none; else HAC_ETIMEOUT once exceeded (checked per round) */
  void *stream;       /* cudaStream_t to run on; NULL = the handle's own stream */
  int flags;          /* HAC_FLAG_* bits; 0 = none */
} hac_opts;

/* Range-query ablation: every active cluster of the instance is a candidate
 * of every search (the pruning of Algorithms 2-3 and the summary upper bounds
 * are off).  Same dendrogram, much more work; for measuring what the range
 * query saves (hac_stats: cluster_pairs, point_pairs vs naive_pairs). */
#define HAC_FLAG_NO_PRUNE 1

typedef struct {
  int64_t rounds;            /* rounds of Algorithm 1 executed */
  int64_t merges;            /* merges made (n - 1 when complete) */
  int64_t nn_searches;       /* terminal nearest-neighbour searches, summed over rounds */
  int64_t cluster_pairs;     /* cluster-pair distance evaluations */
  int64_t point_pairs;       /* point-pair distance evaluations (the paper's D) */
  int64_t nodes_visited;     /* range-query tree nodes tested */
  int64_t rechecks;          /* FP64 re-scores made in HAC_PREC_F32_RECHECK mode */
  double ms_init;            /* layout + index build (Algorithm 1 initialisation) */
  double ms_nn;              /* nearest-neighbour search + chain update */
  double ms_merge;           /* reciprocal-pair filter + merges */
  double ms_update;          /* active/terminal refresh, point re-layout, index rebuild */
  double ms_total;           /* whole hac_run */
  int64_t device_bytes;      /* device memory held by the handle */
  double ms_query;           /* device time of the nearest-neighbour search kernel
                                alone (CUDA events around each launch) */
  int64_t query_launches;    /* launches of that kernel */
  int64_t query_bytes;       /* algorithmic bytes that kernel had to read: tree nodes
                                tested, leaf slots scanned, cluster records and point
                                rows of evaluated pairs (each counted once per use) */
  int64_t leaf_tests;        /* candidate clusters tested against the search ball */
  int64_t kernel_launches;   /* all kernels the library launched in the run */
  int64_t cache_hits;        /* pair distances taken from the cache instead of evaluated */
  int64_t cache_lw_entries;  /* cache entries derived by Lance-Williams after merges */
  double ms_big;             /* device time of the GPU-wide big-pair evaluation kernels */
  int64_t big_point_pairs;   /* point pairs evaluated by those kernels (also in point_pairs);
                                complete linkage skips chunks whose box bound cannot raise
                                the maximum, and those pairs are not counted */
  int64_t big_launches;      /* launches of those kernels */
  int64_t naive_pairs;       /* cluster pairs a search without range queries would
                                evaluate: terminals x (active clusters - 1), summed
                                over rounds */
  int64_t dense_k;           /* average linkage: clusters active when the run switched
                                to the dense matrix of all their pair distances (0 = it
                                did not) */
  int64_t dense_rounds;      /* rounds run on that matrix */
  int64_t dense_point_pairs; /* point pairs of the all-pairs sweep that filled it (also
                                in point_pairs) */
  int64_t dense_rechecks;    /* FP32 mode: matrix entries re-scored in FP64 */
  double ms_dense;           /* device time of the sweep */
} hac_stats_t;

/* Default options (FP64, no cache, no limits, own stream).  No counterpart in
 * the paper (the library's own run options). */
void hac_default_opts(hac_opts *opts);

/* Create an instance from HOST points (paper: Algorithm 1's input, Section 3;
 * every point starts as a singleton cluster whose cid is its input index,
 * Section 1 footnote): `points` is row-major n x d of type
 * `dt` (float or double), read during the call and not retained.  Allocates
 * all device memory the instance needs; the points are copied to the device.
 * HAC_EINVAL: points/out NULL, n < 1, d < 1 or d > 16, unknown dt/lk, or a
 * non-finite coordinate.  HAC_ENOMEM: device allocation failed. */
int hac_create(const void *points, int64_t n, int d, hac_dtype dt, hac_linkage lk, hac_t *out);

/* (Paper: as hac_create, Algorithm 1's input.)  As hac_create, but
 * `dev_points` is a DEVICE pointer (row-major n x d of
 * `dt`, on the current device) that the caller keeps owning; it is copied
 * device-to-device during the call.  Non-finite coordinates are reported by
 * hac_run as HAC_EINVAL. */
int hac_create_device(const void *dev_points, int64_t n, int d, hac_dtype dt, hac_linkage lk,
                      hac_t *out);

/* Run the whole clustering (paper: Algorithm 1 -- initialisation, then rounds
 * of nearest-neighbour search (Algorithms 2-4, Section 4), chain update,
 * reciprocal-pair filter, merges and the Section 5 cache update (Algorithm 5)
 * until one cluster is left).  Average linkage switches, once at most K
 * clusters are active, to the full matrix of their pair distances (the
 * Section 5 cache with room for every pair: 24 bytes per entry of the K x K
 * matrix, allocated once per handle; without room for it the run stays on
 * the range-query search).  K is 8,192 for d <= 3, 16,384 for d <= 8 and
 * 65,536 above, capped so that the matrix takes at most half of the device
 * memory free when the run starts; the environment variable HAC_DENSE_K,
 * read at hac_create, sets it instead (0 = never).  opts may be NULL (defaults).  Blocks until done.  May be called
 * again on the same handle: each call recomputes from the stored points.
 * HAC_ETIMEOUT if a limit in opts is hit (the handle stays usable). */
int hac_run(hac_t h, const hac_opts *opts);

/* Copy the n-1 merges of the last completed hac_run (paper: the merges of
 * Algorithm 1's merge step; heights are the Table 1 linkage values, cids as
 * in the Section 1 footnote; the sort order is this library's own, the paper
 * fixes none) to host array `out`
 * (capacity `cap` records), sorted by (height, size, cid_a).  *n_written
 * receives the count.  HAC_EPENDING before a completed run, HAC_ECAP if
 * cap < n - 1. */
int hac_dendrogram(hac_t h, hac_merge *out, int64_t cap, int64_t *n_written);

/* The round (0-based) of Algorithm 1 (paper: Section 3, one iteration of its
 * main loop) in which each merge of hac_dendrogram's output was made, in the
 * same order.  Same errors as hac_dendrogram. */
int hac_merge_rounds(hac_t h, int32_t *out, int64_t cap, int64_t *n_written);

/* Counters and phase times of the last hac_run (paper: Section 6, analysis of
 * the framework -- point_pairs is the count of distance computations the
 * paper calls D, cluster_pairs and the search counters its range-query
 * statistics).  HAC_EINVAL for a NULL handle or out. */
int hac_stats(hac_t h, hac_stats_t *out);

/* Free the instance and all its device memory.  NULL is a no-op.  No
 * counterpart in the paper. */
void hac_destroy(hac_t h);

/* Static description of a status code (never NULL; unknown codes get a
 * generic text).  No counterpart in the paper. */
const char *hac_strerror(int code);

/* Largest n accepted by hac_run_static. */
#define HAC_STATIC_MAX_N 4096

/* A whole clustering that allocates nothing (the paper has no counterpart;
 * this exists for callers that cannot call cudaMalloc when they need a
 * dendrogram, e.g. a serving process whose memory pool already owns every
 * byte of the GPU, or latency-sensitive code that must not risk the device
 * synchronisation that cudaMalloc/cudaFree can cause).
 *
 * Same dendrogram as hac_create + hac_run + hac_dendrogram on the same points
 * and options (with the dense matrix of average linkage off, HAC_DENSE_K=0;
 * with it on, the same tree and heights within the precision mode's stated
 * bound), computed by the same kernels, but all working memory comes
 * from a fixed 6 MiB device array inside the library, which every GPU that
 * loads the library holds until the process exits.  No cudaMalloc, cudaFree
 * or other allocating call is made.  The pair-distance cache needs memory, so
 * opts->cache_slots is ignored (no cache, hence no GPU-wide big-pair
 * evaluation), and the HAC_* environment overrides that hac_create reads
 * (HAC_BIG_PAIRS, HAC_BIG_PAIRS_F64, HAC_WARP_BUDGET, HAC_BRUTE, HAC_DENSE_K) do
 * not apply;
 * these change speed only, never the result.  HAC_FLAG_NO_PRUNE is honoured.
 *   dev_points  DEVICE pointer, row-major n x d of `dt`, on the current device;
 *               read only, owned by the caller.
 *   opts        may be NULL (defaults); opts->stream selects the stream
 *               (NULL = the legacy default stream).  Blocks until done.
 *   dev_out     DEVICE buffer of at least n - 1 hac_merge records, owned by the
 *               caller; receives the merges sorted by (height, size, cid_a).
 * Errors: HAC_EINVAL for n > HAC_STATIC_MAX_N (or the usual bad arguments,
 * including non-finite coordinates), HAC_ECAP if cap < n - 1, HAC_EDEVICE if
 * the array's device address cannot be obtained or a CUDA call fails.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing once the library's device
 * code is loaded).  Every call shares the one array and overwrites it, so
 * calls that overlap on the GPU (other host threads, other streams) race and
 * must be serialised by the caller. */
int hac_run_static(const void *dev_points, int64_t n, int d, hac_dtype dt, hac_linkage lk,
                   const hac_opts *opts, hac_merge *dev_out, int64_t cap);

/* ------------------------------------------------------------------------
 * Serving: many independent clusterings with continuous batching.
 *
 * The paper clusters one data set per run; a server (no counterpart in the
 * paper) keeps many requests resident on the GPU at once.  Requests of the
 * same linkage, dimension and input type share one ENGINE: one device state
 * for `points_per_engine` points, run by its own host thread on its own CUDA
 * stream.  Every round of Algorithm 1 is one launch per kernel for all of an
 * engine's resident requests; a nearest-neighbour search never leaves its own
 * request.  Between rounds, finished requests leave and queued ones are
 * admitted while their n fits in a free range of the engine's points (first
 * fit, in arrival order) and a request slot is free (4096 per engine), so
 * requests that arrive while others run join at the next round.  Engines of
 * different kinds run concurrently.  Each result is the dendrogram a lone
 * hac_create + hac_run + hac_dendrogram with the server's options gives for
 * the same points (cids local to the request, same canonical order), up to
 * the rounding of FP64 sums whose order depends on the device layout.
 * ------------------------------------------------------------------------ */
typedef struct hac_server *hac_server_t; /* opaque */

typedef struct {
  int64_t engines;         /* engines created so far */
  int64_t rounds;          /* rounds run, summed over engines */
  int64_t admitted;        /* requests admitted to an engine */
  int64_t completed;       /* requests that left an engine (finished, cancelled, timed out) */
  int64_t queued;          /* requests waiting for admission now */
  int64_t resident;        /* requests resident on the GPU now */
  int64_t max_resident;    /* most requests resident at once in one engine */
  int64_t device_bytes;    /* device memory held by all engines */
  int64_t kernel_launches; /* kernels launched by all engines */
  double ms_admit;         /* host wall time engines spent admitting requests */
  double ms_rounds;        /* ... running rounds (kernels, and waits on them) */
  double ms_harvest;       /* ... handing out finished requests */
} hac_server_stats_t;

/* (No counterpart in the paper, like every serving call below; each request
 * is one run of Algorithm 1.)  Create a server on the current CUDA device.  `points_per_engine` (2 ..
 * 2^29) sizes every engine, and bounds the n of a request.  An engine holds
 * about 0.35 KB (d <= 2) to 1.4 KB (d > 8) of device memory per point; with
 * opts->cache_slots > 0, complete and average engines add about 88 bytes
 * plus 24 bytes per slot per point and about 280 MiB of big-pair buffers.  An engine is
 * allocated when the first request of its kind arrives.  opts (may be NULL) gives precision
 * and cache_slots for every request; its stream, max_rounds and timeout_s
 * are ignored.  HAC_EINVAL for bad arguments, HAC_ENOMEM, HAC_EDEVICE. */
int hac_server_create(int64_t points_per_engine, const hac_opts *opts, hac_server_t *out);

/* (No counterpart in the paper.)  Queue a request (Algorithm 1's input, as
 * hac_create): HOST points, row-major n x d of `dt`, copied during the
 * call.  timeout_s > 0 sets a deadline from now: a request not finished by
 * then leaves at the next round boundary with HAC_ETIMEOUT.  *ticket names
 * it for hac_poll / hac_server_wait / hac_cancel.  Never blocks on the GPU,
 * except that the first request of a new kind allocates its engine.
 * HAC_EINVAL as for hac_create; HAC_ENOMEM if n > points_per_engine or the
 * engine cannot be allocated; after an engine failed, its code. */
int hac_submit(hac_server_t srv, const void *points, int64_t n, int d, hac_dtype dt,
               hac_linkage lk, double timeout_s, uint64_t *ticket);

/* (No counterpart in the paper.)  Cancel a request: a queued one leaves at once, a resident one at the next
 * round boundary; either then completes with HAC_ECANCELED.  HAC_OK also if
 * it had already finished (its result stays).  HAC_EINVAL: unknown ticket. */
int hac_cancel(hac_server_t srv, uint64_t ticket);

/* (No counterpart in the paper; the result is Algorithm 1's merges as in
 * hac_dendrogram.)  Non-blocking result of a request.  HAC_EPENDING while it runs.  Once it
 * has finished, the n-1 merges go to host array `out` (capacity `cap`;
 * HAC_ECAP if too small, ticket kept), *n_written receives their count,
 * *latency_ms (may be NULL) the time from hac_submit to completion, and the
 * ticket is released; a failed, cancelled or timed-out request returns its
 * code (HAC_ECANCELED, HAC_ETIMEOUT, HAC_EDEVICE, ...) and is released too.
 * HAC_EINVAL: unknown or already released ticket. */
int hac_poll(hac_server_t srv, uint64_t ticket, hac_merge *out, int64_t cap, int64_t *n_written,
             double *latency_ms);

/* (No counterpart in the paper.)  Block until the request has finished (hac_poll will not return
 * HAC_EPENDING) or timeout_s seconds passed (HAC_ETIMEOUT); timeout_s = 0
 * waits without limit.  HAC_EINVAL: unknown ticket. */
int hac_server_wait(hac_server_t srv, uint64_t ticket, double timeout_s);

/* (No counterpart in the paper.)  Counters of the server; returns the sticky error of a failed engine
 * (HAC_OK if none). */
int hac_server_stats(hac_server_t srv, hac_server_stats_t *out);

/* (No counterpart in the paper.)  Stop every engine after its current round, free all device memory and
 * every unreleased request.  NULL is a no-op. */
void hac_server_destroy(hac_server_t srv);

/* Cluster the points of `count` distinct handles together (the batched form
 * of hac_run, i.e. of Algorithm 1 per handle; the paper has no counterpart
 * for the batching).  Handles of the same linkage,
 * dimension and input type share one engine of a private server, so each
 * round is one launch per kernel for all of them; different kinds run
 * concurrently.  Afterwards each handle holds what hac_run(h, opts) would
 * leave: hac_dendrogram and hac_merge_rounds give the same merges in the same
 * rounds (heights up to the rounding of FP64 sums whose order depends on the
 * device layout).  hac_stats reports only rounds, merges, device_bytes and
 * ms_total (the batch's wall time).  opts may be NULL; its stream is ignored,
 * max_rounds must be 0, timeout_s applies to each handle.  Blocks until all
 * are done; allocates the engines for the call (about the size of the
 * handles' own state) and frees them before returning.  Returns HAC_OK, or
 * the first error of any handle (that handle then has no dendrogram;
 * HAC_EINVAL also for a NULL or repeated handle, a non-finite coordinate, or
 * in the FP32 + re-score mode a handle whose FP32 copy would hold a
 * coordinate of 2^40 or more, which hac_run runs in FP64 instead). */
int hac_run_batch(hac_t *hs, int count, const hac_opts *opts);

#ifdef __cplusplus
}
#endif

#endif /* HAC_H_ */
