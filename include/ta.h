/*
 * ta.h -- C ABI of the B300 trace-analysis library (libta.so).
 *
 * The library turns per-rank execution traces into the products the paper's
 * analysis layer derives from them (arxiv 2605.03561):
 *   - the rank x iteration x context tensor of exclusive time (Section V,
 *     the tri-dimensional model; iterations re-materialised from traces),
 *   - exclusive time per (rank, context) and inclusive time rolled up the
 *     calling context tree (Section II-A, inclusive/exclusive costs),
 *   - cross-rank statistics per context: min/max/mean/std, balance ratio,
 *     coefficient of variation, argmax rank, z-score outliers (Section VI-A,
 *     the group-by listing and Table IV; Section VI-B, outlier ranks),
 *   - the node/chassis/rack rollup of outlier ranks (Section VI-B),
 *   - the imbalance-derived potential speedup (Section VI-A, Table V),
 *   - pruning of the calling context tree on the summary profile, profiles
 *     of time windows and bottom-up calling contexts (Section III-A,
 *     Section VI-B), clusters of ranks by DBSCAN / K-Means with their node
 *     view (Section VI-B), and the DataFrame operation classes the paper
 *     benchmarks (Section IV) as column kernels,
 *   - a batched form (many trace sets in one CUDA graph) and a serving form
 *     (resident experiments, continuous batching of queries).
 *
 * Every computation runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions
 *   - Every call returns ta_status; no exception crosses the ABI.  After a
 *     non-OK status, ta_last_error_message() (thread-local) says why.
 *   - Inputs are borrowed: the library reads them during the call.
 *   - Outputs go to caller-owned buffers whose memory kind (host or device) is
 *     stated in the argument struct.  Every call below returns after its
 *     device work is complete (it synchronises the context's stream), so both
 *     host and device outputs are ready on return.
 *   - Sizes use the two-call pattern: a call whose output arrays are NULL only
 *     reports the sizes; too small a capacity returns TA_ERR_CAPACITY with
 *     the required size filled in and writes nothing.
 *   - Device memory the library needs is obtained from the allocator given to
 *     ta_set_allocator() (default: cudaMallocAsync on the context's stream).
 *   - Exactness: all times are integer nanoseconds (uint64).  Sums and moments
 *     are exact integers (sum of squares in 128 bits); only the final mean,
 *     std, cv, balance, z and speedup ratios are IEEE double, each a fixed
 *     sequence of correctly rounded operations on exactly converted integers.
 *     Loading requires R * (longest rank span) < 2^63 so that every such
 *     integer fits (TA_ERR_INVALID_ARG otherwise).
 */
#ifndef TA_H
#define TA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ta_status {
  TA_OK = 0,
  TA_ERR_INVALID_ARG = 1, /* bad pointer, size, subset, rank offsets, limits */
  TA_ERR_NOT_SORTED = 2,  /* a rank's timestamps decrease                     */
  TA_ERR_BAD_CTX = 3,     /* a sample's context id >= n_ctx                    */
  TA_ERR_BAD_CCT = 4,     /* parent array: not exactly one root, parent out of
                             range, or a cycle                                */
  TA_ERR_OOM = 5,         /* device allocation failed                         */
  TA_ERR_CAPACITY = 6,    /* caller buffer too small; required size filled in  */
  TA_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up               */
  TA_ERR_CUDA = 8,        /* CUDA runtime error                               */
  TA_ERR_STATE = 9        /* call not valid in the object's current state     */
} ta_status;

#define TA_NO_PARENT 0xFFFFFFFFu

typedef enum ta_mem_kind { TA_MEM_HOST = 0, TA_MEM_DEVICE = 1 } ta_mem_kind;
typedef enum ta_metric { TA_EXCLUSIVE = 0, TA_INCLUSIVE = 1 } ta_metric;

typedef struct ta_ctx ta_ctx;
typedef struct ta_experiment ta_experiment;

/* ------------------------------------------------------------ context ---- */

/* Create a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * stream is borrowed and must outlive the context.  Errors: INVALID_ARG
 * (out NULL), CUDA (no such device). */
ta_status ta_create(int device, void* cuda_stream, ta_ctx** out);
ta_status ta_destroy(ta_ctx* ctx);

/* Device memory callbacks.  alloc(bytes, stream, user) returns device memory
 * usable on `stream` or NULL; free(ptr, bytes, stream, user) releases it.
 * Pass NULLs to restore the default (cudaMallocAsync / cudaFreeAsync). */
typedef void* (*ta_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*ta_free_fn)(void* ptr, size_t bytes, void* stream, void* user);
ta_status ta_set_allocator(ta_ctx* ctx, ta_alloc_fn alloc, ta_free_fn free_fn, void* user);

/* Wait for all work issued on the context's stream. */
ta_status ta_sync(ta_ctx* ctx);

/* Thread-local text of the last error; never NULL. */
const char* ta_last_error_message(void);
const char* ta_status_string(ta_status s);

/* Number of kernel launches the library has issued on this context so far. */
uint64_t ta_kernel_launches(const ta_ctx* ctx);

/* Device time of the library's phases on this context, measured with CUDA
 * events recorded on the context's stream around each phase, accumulated
 * since the last reset; plus the units the iteration-tensor kernel processed
 * (samples read, entries and rows written) for bytes-per-launch accounting. */
typedef struct ta_profile {
  double validate_ms;
  double tensor_count_ms; /* tensor count pass + tile scan                 */
  double tensor_ms;       /* tensor write pass (the dominant kernel)       */
  double exclusive_ms, inclusive_ms;
  double stats_ms, topology_ms, speedup_ms;
  uint64_t tensor_launches, tensor_records, tensor_entries, tensor_rows;
  double interval_ms; /* time-window profiles (ta_interval_profile)      */
  /* what the time-window kernels read: edge samples (12 B each) and inner
     tensor entries (16 B each) */
  uint64_t interval_samples, interval_entries;
} ta_profile;
ta_status ta_get_profile(ta_ctx* ctx, ta_profile* out, int reset);

/* --------------------------------------------------------- ingestion ---- */

/* Execution traces (Section II-A: per rank a time-ordered list of samples,
 * each a timestamp and the calling context tree node it hit).
 *   rank_off[R+1]  CSR offsets into ts/ctx; rank r owns samples
 *                  [rank_off[r], rank_off[r+1]); rank_off[0] = 0,
 *                  non-decreasing, rank_off[R] = n_records; a rank may be
 *                  empty; a rank holds fewer than 2^32 samples.
 *   ts[N]          uint64 ns, non-decreasing within a rank (ties allowed).
 *   ctx[N]         uint32 context id < n_ctx.
 *   parent[C]      calling context tree; exactly one root with
 *                  parent = TA_NO_PARENT; every other parent < C; acyclic.
 *   marker_ctx     iteration marker context (< C): an iteration starts at
 *                  the first sample of every run of marker samples; samples
 *                  before a rank's first marker form its prologue row.
 *   mem_kind       where the four arrays live.
 *   flags          TA_LOAD_BORROW: device ts/ctx are used in place (no copy)
 *                  and must stay valid and unchanged until
 *                  ta_experiment_free() (arrays not 16-byte aligned are
 *                  copied instead); TA_LOAD_NO_INCLUSIVE: skip the
 *                  inclusive rollup; TA_LOAD_KEEP_TRACES: keep the copied
 *                  ts/ctx on the device after ingestion (by default they
 *                  are released), for ta_interval_profile.
 *   nnz_hint, rows_hint  optional first-try capacities of the tensor (0 =
 *                  library default); a too-small hint only costs a re-run.
 * A sample lasts until the next sample of its rank; a rank's last sample
 * lasts 0 ns but still counts as one sample. */
#define TA_LOAD_BORROW 1u
#define TA_LOAD_NO_INCLUSIVE 2u
#define TA_LOAD_KEEP_TRACES 4u

typedef struct ta_trace_desc {
  uint32_t n_ranks;
  uint32_t n_ctx;
  uint32_t marker_ctx;
  uint32_t mem_kind;
  uint64_t n_records;
  const uint64_t* rank_off;
  const uint64_t* ts;
  const uint32_t* ctx;
  const uint32_t* parent;
  uint32_t flags;
  uint32_t reserved;
  uint64_t nnz_hint;
  uint64_t rows_hint;
} ta_trace_desc;

/* Validate the traces (all of the rules above) and build the experiment's
 * resident products on the device: per-rank spans and iteration counts, the
 * iteration tensor, the exclusive CSR and (unless skipped) the inclusive CSR.
 * Beside the exclusive CSR it keeps each entry's iteration moments: the time
 * summed over the rank's iteration rows and the 128-bit sum of its squares.
 * They are kept only for ranks whose iteration rows all hold the same
 * contexts, and ta_potential_speedup reads them.  24 bytes per exclusive
 * entry plus 1 per rank; ta_prune_profiles drops them.
 * Synchronous: returns after the device work, with the first error found in
 * the order INVALID_ARG, BAD_CCT, BAD_CTX, NOT_SORTED (then OOM, TIMEOUT,
 * CUDA).  Host inputs are copied to the device first.  The experiment is
 * owned by the caller and released by ta_experiment_free(). */
ta_status ta_load_traces(ta_ctx* ctx, const ta_trace_desc* d, ta_experiment** out);
ta_status ta_experiment_free(ta_experiment* e);

typedef struct ta_experiment_info {
  uint32_t n_ranks, n_ctx, marker_ctx, max_depth; /* max_depth: deepest node */
  uint64_t n_records;
  uint64_t n_rows;       /* rows of the iteration tensor = R + sum n_iter   */
  uint64_t tensor_nnz;   /* (rank, iteration, ctx) entries                  */
  uint64_t excl_nnz;     /* (rank, ctx) entries of the exclusive CSR        */
  uint64_t incl_nnz;     /* (rank, ctx) entries of the inclusive CSR (0 if skipped) */
  uint64_t device_bytes; /* device memory held by the experiment           */
} ta_experiment_info;
ta_status ta_experiment_get_info(const ta_experiment* e, ta_experiment_info* info);

/* ------------------------------------------------- iteration tensor ---- */

/* The tri-dimensional model of Section V as CSR over (rank, iteration) rows.
 * Rank r owns rows [row_off_of_rank[r], row_off_of_rank[r+1]): its prologue
 * row (possibly empty) and then one row per iteration, n_iter[r] of them.
 * Row k owns entries [entry_off[k], entry_off[k+1]), context-ascending, one
 * per context with at least one sample in that row: e_time = summed sample
 * durations (ns), e_cnt = samples.
 *   n_iter[R], row_off_of_rank[R+1], entry_off[rows+1]  (rows_cap >= rows+1)
 *   e_ctx, e_time, e_cnt [nnz]                          (nnz_cap >= nnz)
 * Any array may be NULL to skip it; all NULL = sizes only. */
typedef struct ta_tensor_out {
  uint32_t mem_kind;
  uint32_t reserved;
  uint32_t* n_iter;
  uint64_t* row_off_of_rank;
  uint64_t* entry_off;
  uint32_t* e_ctx;
  uint64_t* e_time;
  uint32_t* e_cnt;
  uint64_t rows_cap; /* elements of entry_off                          */
  uint64_t nnz_cap;  /* elements of e_ctx / e_time / e_cnt             */
  uint64_t rows;     /* out                                            */
  uint64_t nnz;      /* out                                            */
} ta_tensor_out;
ta_status ta_iteration_tensor(ta_experiment* e, ta_tensor_out* o);

/* Per-(rank, context) CSR: rank r owns [off[r], off[r+1]), context-ascending.
 * Exclusive: time and samples in that context (Section V, profiles collapse
 * time).  Inclusive: the same summed over the context's subtree of the
 * calling context tree; present for every ancestor of a present context. */
typedef struct ta_csr_out {
  uint32_t mem_kind;
  uint32_t reserved;
  uint64_t* off; /* [R+1] */
  uint32_t* ctx;
  uint64_t* time;
  uint32_t* cnt;
  uint64_t nnz_cap;
  uint64_t nnz; /* out */
} ta_csr_out;
ta_status ta_exclusive(ta_experiment* e, ta_csr_out* o);
ta_status ta_inclusive_rollup(ta_experiment* e, ta_csr_out* o);

/* Zero-copy views of the resident products (device pointers owned by the
 * experiment, valid until ta_experiment_free). */
typedef struct ta_tensor_view {
  const uint32_t* n_iter;
  const uint64_t* row_off_of_rank;
  const uint64_t* entry_off;
  const uint32_t* e_ctx;
  const uint64_t* e_time;
  const uint32_t* e_cnt;
  const uint64_t* span; /* [R] ts_last - ts_first (0 for an empty rank) */
  uint64_t rows, nnz;
} ta_tensor_view;
typedef struct ta_csr_view {
  const uint64_t* off;
  const uint32_t* ctx;
  const uint64_t* time;
  const uint32_t* cnt;
  uint64_t nnz;
} ta_csr_view;
ta_status ta_tensor_get_view(const ta_experiment* e, ta_tensor_view* v);
ta_status ta_csr_get_view(const ta_experiment* e, uint32_t metric, ta_csr_view* v);

/* ---------------------------------------------- cross-rank statistics ---- */

/* Per context c over the rank set S (n = |S|; a rank without samples of c
 * counts as x = 0 -- absent ranks are idle ranks):
 *   n, present (ranks with >= 1 sample), min, max, argmax (lowest rank
 *   attaining max), s1 = sum x, s2 = sum x^2 (128-bit: s2_hi:s2_lo),
 *   mean = s1/n, std (ddof 1; 0 if n < 2), cv = std/mean (0 if mean = 0),
 *   balance = mean/max (1 if max = 0)          (Section VI-A, Table IV).
 * z-score of a present rank r: (n x_r - s1) / (n std) (0 if std = 0).
 * Outlier: a present rank whose z exceeds tau = tau_num / tau_den, decided
 * exactly in integers (no rounding) -- the high side only, slow ranks
 * (Section VI-B).  Outliers are listed sorted by (ctx, rank).
 *   ranks     sorted, unique rank ids, or NULL for all ranks;
 *   ctxs      sorted, unique context ids, or NULL for all C;
 *   mem_kind  of ranks/ctxs and of every output array. */
typedef struct ta_stats_args {
  uint32_t metric; /* ta_metric */
  uint32_t mem_kind;
  const uint32_t* ranks;
  uint32_t n_ranks_subset;
  uint32_t n_ctxs;
  const uint32_t* ctxs;
  uint32_t tau_num, tau_den; /* tau_den > 0 */
} ta_stats_args;

typedef struct ta_ctx_stats {
  uint32_t n, present, argmax, reserved;
  uint64_t min, max, s1, s2_lo, s2_hi;
  double mean, std, cv, balance;
} ta_ctx_stats;

typedef struct ta_outlier {
  uint32_t ctx, rank;
  double z;
} ta_outlier;

/* stats[n_ctxs or C] in the order of ctxs; outliers[outlier_cap];
 * z (optional) is laid out like the metric's CSR entries and receives the
 * z-score of each entry of a rank in S and a requested context, 0 elsewhere.
 * n_outliers is always set; if it exceeds outlier_cap the call returns
 * TA_ERR_CAPACITY after writing stats and z (outliers unspecified). */
typedef struct ta_stats_out {
  ta_ctx_stats* stats;
  ta_outlier* outliers;
  uint64_t outlier_cap;
  uint64_t n_outliers; /* out */
  double* z;
} ta_stats_out;
ta_status ta_context_stats(ta_experiment* e, const ta_stats_args* a, ta_stats_out* o);

/* --------------------------------------------------- topology rollup ---- */

/* Integer machine topology (Section VI-B: rank -> compute node via the
 * profile metadata, node -> chassis and rack via its Slingshot coordinate).
 * Chassis ids are global (not per rack). */
typedef struct ta_topology {
  uint32_t n_nodes, n_chassis, n_racks, mem_kind;
  const uint32_t* node_of_rank;    /* [R]       */
  const uint32_t* rack_of_node;    /* [n_nodes] */
  const uint32_t* chassis_of_node; /* [n_nodes] */
} ta_topology;

/* One context: its outlier ranks over S (as in ta_context_stats), then per
 * node: outlier ranks, sum of x over its ranks in S, ranks in S; a node is
 * flagged when it has >= min_ranks (>= 1) outlier ranks; per chassis and per
 * rack: flagged nodes, nodes, summed x; flagged_racks = racks with a flagged
 * node, ascending. */
typedef struct ta_topo_args {
  uint32_t metric;
  uint32_t ctx;
  uint32_t tau_num, tau_den;
  uint32_t min_ranks;
  uint32_t n_ranks_subset;
  const uint32_t* ranks; /* sorted unique or NULL; memory kind of ta_topo_out */
} ta_topo_args;

typedef struct ta_topo_out {
  uint32_t mem_kind;
  uint32_t n_flagged_racks; /* out */
  uint32_t* node_outliers;   /* [n_nodes]   */
  uint64_t* node_sum;        /* [n_nodes]   */
  uint32_t* node_ranks;      /* [n_nodes]   */
  uint8_t* node_flag;        /* [n_nodes]   */
  uint32_t* chassis_flagged; /* [n_chassis] */
  uint32_t* chassis_nodes;   /* [n_chassis] */
  uint64_t* chassis_sum;     /* [n_chassis] */
  uint32_t* rack_flagged;    /* [n_racks]   */
  uint32_t* rack_nodes;      /* [n_racks]   */
  uint64_t* rack_sum;        /* [n_racks]   */
  uint32_t* flagged_racks;   /* [n_racks]   */
} ta_topo_out;
ta_status ta_topology_rollup(ta_experiment* e, const ta_topology* t, const ta_topo_args* a,
                             ta_topo_out* o);

/* ------------------------------------------------- potential speedup ---- */

/* Section VI-A, Table V.  For contexts K (sorted unique, e.g. the GPU
 * kernels) over ranks S, using iterations i < I* = min over S of n_iter (the
 * prologue and later iterations are excluded; excluded_iterations counts the
 * latter).  With t[r][i][k] the tensor's time (0 if absent):
 *   A_k = sum_i max_r t, B_k = sum_i sum_r t, G_k = n A_k - B_k (exact),
 *   avg_mean = B_k / (n I*), avg_max = A_k / I*, savings_per_iter = G_k/(n I*),
 *   total_reduction = G_k / n, share = B_k / sum B,
 *   cv_across = mean over i of (std/mean over ranks of t[.][i][k]),
 *   cv_within = mean over r in S of (std/mean over i < I* of t[r][.][k]),
 * and totals: sum G, total reduction = sum G / n, t_app = app_time_ns or
 * (if 0) the longest rank span in S, speedup_fraction = sum G / (n t_app).
 * cv_across sums its terms in ascending i.  cv_within sums its per-rank
 * terms in a fixed pairwise order: level by level, v[2i] + v[2i+1], an odd
 * last term moving up.  Each per-rank term is computed as
 * sqrt(m / (m - 1)) sqrt(m q - s^2) / s from the exact sums s and q over
 * m = I* iterations.  That equals std/mean up to a few units in the last
 * place.  For ranks with exactly I* iterations whose iteration rows all hold
 * the same contexts, s and q come from the load's iteration moments; other
 * ranks read their tensor rows. */
typedef struct ta_speedup_args {
  uint32_t mem_kind; /* of ctxs / ranks / outputs */
  uint32_t n_ctxs;
  const uint32_t* ctxs;
  const uint32_t* ranks;
  uint32_t n_ranks_subset;
  uint32_t reserved;
  uint64_t app_time_ns;
} ta_speedup_args;

typedef struct ta_speedup_ctx {
  uint64_t A, B, G_lo, G_hi;
  double avg_mean, avg_max, savings_per_iter, total_reduction, share, cv_across, cv_within;
} ta_speedup_ctx;

typedef struct ta_speedup_total {
  uint32_t i_star, reserved;
  uint64_t excluded_iterations;
  uint64_t sum_G_lo, sum_G_hi;
  uint64_t t_app;
  double total_reduction;
  double speedup_fraction;
} ta_speedup_total;

typedef struct ta_speedup_out {
  ta_speedup_ctx* per_ctx;  /* [n_ctxs] */
  ta_speedup_total* total;  /* [1]      */
} ta_speedup_out;
ta_status ta_potential_speedup(ta_experiment* e, const ta_speedup_args* a, ta_speedup_out* o);

/* --------------------------------------------------------------- pruning --- */

/* Pruning of the calling context tree on the summary profile (Section III-A,
 * "Pruning Large Calling Context Trees": a strategy is evaluated once on the
 * summary profile, the aggregate of all parallel profiles, then propagated to
 * every parallel profile; Section VI-B removes library internals, line
 * statements and regions under 1 % of the total runtime).
 * The summary profile holds each context's inclusive time summed over all
 * ranks; the total is the root's.  Context c is kept iff
 *     summary[c] * keep_den >= total * keep_num      (exact integers)
 * and drop[c] is 0 (drop: optional per-context flags for classes the caller
 * removes by name, such as library internals or line statements).  Every
 * rank's exclusive and inclusive CSR is then compacted IN PLACE to the kept
 * contexts (order kept; a pruned context's time is not moved elsewhere), so
 * later calls and views see the pruned profiles; the iteration tensor is
 * not changed.  Needs the inclusive CSR (loaded without TA_LOAD_NO_INCLUSIVE).
 *   keep_num / keep_den  threshold fraction of the total (keep_den > 0; 1/100
 *                        is the paper's 1 %; 0/1 keeps every context).
 *   drop                 NULL or uint8[n_ctx] (nonzero: drop).
 *   kept                 NULL or uint8[n_ctx] out: 1 for kept contexts.
 *   summary              NULL or uint64[n_ctx] out: summary inclusive times.
 *   n_kept, excl_nnz, incl_nnz  out: kept contexts and the CSRs' new sizes.
 * mem_kind applies to drop, kept and summary.  Errors: INVALID_ARG (NULL, den
 * 0, mem kind), STATE (no inclusive CSR, or the experiment is registered with
 * a server, whose queries read its CSRs), OOM, CUDA. */
typedef struct ta_prune_args {
  uint32_t mem_kind;
  uint32_t keep_num;
  uint32_t keep_den;
  uint32_t reserved;
  const uint8_t* drop;
} ta_prune_args;

typedef struct ta_prune_out {
  uint8_t* kept;
  uint64_t* summary;
  uint32_t n_kept;
  uint32_t reserved;
  uint64_t excl_nnz;
  uint64_t incl_nnz;
} ta_prune_out;
ta_status ta_prune_profiles(ta_experiment* e, const ta_prune_args* a, ta_prune_out* o);

/* ------------------------------------------------ time-window slices ---- */

/* Per-rank profiles of the time window [t0, t1) (Section III-A: queries of
 * rank ranges and time ranges over the traces, which hold time-ordered
 * calling-context events and are searched by binary search on time).  Sample
 * i of a rank is in ctx_i during [ts_i, ts_{i+1}) (the rank's last sample
 * during [ts_i, ts_i]).  For ranks r0 <= r < r1 (relative index r - r0):
 *   exclusive: per context, time = the summed length of its samples'
 *              intervals inside the window, cnt = its samples whose ts lies
 *              in the window; a context is listed iff time > 0 or cnt > 0
 *              (the sample in progress at t0 gives time but no count).
 *   inclusive: the exclusive window profile rolled up the calling context
 *              tree as in ta_inclusive_rollup.
 * Over the whole time range this is ta_exclusive / ta_inclusive_rollup of
 * the same ranks, and adjacent windows add up exactly.  t1 <= t0 is an
 * empty window (every rank empty).
 * Needs the raw traces: loaded with TA_LOAD_KEEP_TRACES, or borrowed
 * (TA_LOAD_BORROW with aligned device arrays).  Each rank's window is found
 * by warp-cooperative 32-ary searches (of its iterations' start times, then
 * of one iteration's timestamps); iterations wholly inside the window are
 * taken from the iteration tensor, the samples of the partial iterations at
 * its edges one by one.  The first call builds an index of every tensor
 * row's first sample and its time (16 bytes per row, kept with the
 * experiment).  The result of the last call stays with the experiment in
 * device memory until a call with other arguments or ta_experiment_free, so
 * the second call of the two-call pattern only copies it out.
 *   o  as for ta_exclusive, over r1 - r0 ranks: off[r1 - r0 + 1]; NULL
 *      arrays = sizes only; nnz_cap too small = TA_ERR_CAPACITY (nnz set).
 * The inclusive window needs only the tree, not the experiment's inclusive
 * CSR.  Errors: INVALID_ARG (NULL, r0 > r1 or r1 > n_ranks, metric,
 * mem_kind), STATE (the traces were released after loading), OOM, CUDA. */
typedef struct ta_interval_args {
  uint64_t t0, t1;
  uint32_t r0, r1;
  uint32_t metric; /* ta_metric */
  uint32_t reserved;
} ta_interval_args;
ta_status ta_interval_profile(ta_experiment* e, const ta_interval_args* a, ta_csr_out* o);

/* Calling contexts of n contexts, bottom up (Section VI-B, "Obtaining
 * Calling Context": from a tree node up to the root, e.g. a communication
 * leaf to the solver call that issued it): chain i is
 * chain[off[i] .. off[i+1]) = ctxs[i], its parent, ..., the root; its length
 * is the node's depth + 1.
 *   mem_kind  of ctxs, off and chain.
 *   ctxs[n]   context ids (< n_ctx; any order, repeats allowed).
 *   off       [n + 1] out, or NULL (sizes only, with chain NULL).
 *   chain     [chain_cap] out, or NULL.
 *   total     out: off[n] (always set).
 * Errors: INVALID_ARG (NULL e/ctxs/total, mem_kind, a context id >= n_ctx),
 * CAPACITY (chain_cap < total; nothing written), OOM, CUDA. */
ta_status ta_call_chains(const ta_experiment* e, uint32_t mem_kind, const uint32_t* ctxs,
                         uint32_t n, uint64_t* off, uint32_t* chain, uint64_t chain_cap,
                         uint64_t* total);

/* ------------------------------------------------ clustering of ranks ---- */

/* Groups of ranks by their value of one context (Section VI-B: the ranks'
 * times of a communication call site clustered with DBSCAN, the groups
 * mapped to compute nodes, and K-Means over 2..5 groups as a stability
 * check).  The value of rank r is x_r = the metric's time of ctx on r, 0
 * where r has no sample of it (as in ta_context_stats).
 *   TA_CLUSTER_DBSCAN (eps in ns, min_pts >= 1): the eps-neighbourhood of a
 *     rank holds every rank of the subset whose value differs by at most eps,
 *     itself included; a rank with at least min_pts neighbours is a core;
 *     clusters are the connected components of cores (two cores are
 *     connected when they are neighbours); a non-core within eps of a core
 *     joins the cluster of its nearest core (equal distances: the cluster of
 *     smaller values); every other rank is noise (label -1).
 *   TA_CLUSTER_KMEANS (1 <= k <= 64; max_iter, 0 = 300): Lloyd's iteration
 *     in exact rational arithmetic.  Centroid j starts at the value at
 *     sorted position floor((2j + 1) n / (2k)).  Each assignment orders the
 *     clusters by centroid (stably) and gives every rank to the first cluster
 *     at the smallest distance; each update moves a non-empty cluster to its
 *     mean (an empty one keeps its centroid); the iteration stops when an
 *     assignment repeats the previous one or after max_iter updates.
 * Both give clusters that are ranges of the sorted values; they are numbered
 * in ascending order of value.
 *   ranks         sorted unique rank subset, or NULL for all ranks; labels
 *                 follow its order.
 *   node_of_rank  NULL, or the node of every rank of the experiment (< n_nodes):
 *                 then, when n_clusters <= 64, the node view is computed
 *                 (Section VI-B's node-level correlation): per cluster the
 *                 nodes holding one of its ranks, per pair i < j the nodes
 *                 holding ranks of both (pair_nodes[i * cluster_cap + j]),
 *                 and the nodes holding a noise rank.
 *   mem_kind      of ranks, node_of_rank and every output array.
 * Outputs: labels[n] (int32, or NULL), clusters[cluster_cap] (n, sum, min,
 * max of the cluster's values; mean = (double)sum / (double)n; centroid =
 * the mean for DBSCAN, the K-Means centroid S / c as (double)S / (double)c
 * of its unreduced sum S and count c), n_clusters, n_noise, iterations
 * (K-Means updates made), cluster_nodes[cluster_cap], pair_nodes
 * [cluster_cap * cluster_cap], noise_nodes and node_view (1 when the node
 * arrays were written).  More clusters than cluster_cap: TA_ERR_CAPACITY
 * after the labels (n_clusters set).  Errors: INVALID_ARG (NULL, method,
 * metric, ctx, subset, min_pts 0, k, a node id >= n_nodes), STATE
 * (inclusive metric without the inclusive rollup), CAPACITY, OOM, CUDA. */
#define TA_CLUSTER_DBSCAN 1u
#define TA_CLUSTER_KMEANS 2u
typedef struct ta_cluster_args {
  uint32_t method;          /* TA_CLUSTER_DBSCAN or TA_CLUSTER_KMEANS */
  uint32_t metric;          /* ta_metric                               */
  uint32_t ctx;
  uint32_t mem_kind;
  const uint32_t* ranks;
  uint32_t n_ranks_subset;
  uint32_t min_pts;         /* DBSCAN                                  */
  uint64_t eps;             /* DBSCAN, ns                              */
  uint32_t k;               /* K-Means                                 */
  uint32_t max_iter;        /* K-Means                                 */
  const uint32_t* node_of_rank;
  uint32_t n_nodes;
  uint32_t reserved;
} ta_cluster_args;
typedef struct ta_cluster_info {
  uint64_t n, sum, min, max;
  double mean, centroid;
} ta_cluster_info;
typedef struct ta_cluster_out {
  int32_t* labels;
  ta_cluster_info* clusters;
  uint32_t* cluster_nodes;
  uint32_t* pair_nodes;
  uint32_t cluster_cap;
  uint32_t n_clusters;  /* out */
  uint64_t n_noise;     /* out */
  uint32_t iterations;  /* out */
  uint32_t noise_nodes; /* out */
  uint32_t node_view;   /* out */
  uint32_t reserved;
} ta_cluster_out;
ta_status ta_cluster_ranks(ta_experiment* e, const ta_cluster_args* a, ta_cluster_out* o);

/* ------------------------------------------------ column operations ---- */

/* The operation classes the paper times its DataFrame backends with on
 * trace events (Section IV, Tables I-III: grouping, sorting, filtering,
 * merging; scalar compare, vector add, in-place multiply, reduction sum,
 * cumulative sum), as kernels over columns in device memory.  Every pointer
 * below is a device pointer; every call runs on the context's stream and
 * returns after its work is done.  n < 2^32 rows.  Errors: INVALID_ARG
 * (NULL with n > 0, n too large, ranges), OOM, CUDA. */

/* The trace events of ranks [r0, r1) of an experiment that kept its traces
 * (TA_LOAD_KEEP_TRACES or borrowed), as columns of n = rank_off[r1] -
 * rank_off[r0] rows in rank and time order: rank, ts, ctx and dur (the next
 * timestamp of the rank minus this one, 0 for a rank's last event).  Any
 * output may be NULL.  *n_out receives n.  STATE if the traces were
 * released. */
ta_status ta_events_table(ta_experiment* e, uint32_t r0, uint32_t r1, uint32_t* rank,
                          uint64_t* ts, uint32_t* ctx, uint64_t* dur, uint64_t* n_out);

/* Sorting: stable ascending sort of keys (LSD radix sort, 8-bit digits,
 * only as many passes as the largest key needs).  keys_out[n] and perm[n]
 * (perm[i] = the input row of the i-th smallest key) must not overlap keys. */
ta_status ta_col_sort(ta_ctx* ctx, const uint64_t* keys, uint64_t n, uint64_t* keys_out,
                      uint32_t* perm);

/* Filtering: the ascending row ids i with lo <= col[i] <= hi into
 * idx_out[n] (capacity n); *n_out (host) receives their number. */
ta_status ta_col_filter(ta_ctx* ctx, const uint64_t* col, uint64_t n, uint64_t lo, uint64_t hi,
                        uint32_t* idx_out, uint64_t* n_out);

/* Grouping: per segment s (rows [seg_off[s], seg_off[s+1]); seg_off[0] = 0,
 * non-decreasing, seg_off[n_seg] = n) and key (< n_keys), the sum of val
 * and the row count, keys ascending within a segment, as a CSR:
 * off_out[n_seg + 1], key_out / sum_out / cnt_out [out_cap].  A call with
 * key_out, sum_out and cnt_out NULL reports the size only; *n_out (host)
 * receives the number of groups; out_cap too small: CAPACITY.  Sums wrap
 * modulo 2^64. */
ta_status ta_col_group(ta_ctx* ctx, const uint64_t* seg_off, uint32_t n_seg, const uint32_t* key,
                       uint32_t n_keys, const uint64_t* val, uint64_t n, uint64_t* off_out,
                       uint32_t* key_out, uint64_t* sum_out, uint32_t* cnt_out,
                       uint64_t out_cap, uint64_t* n_out);

/* Merging: the join of a fact column with a dimension table on its row id,
 * out[i] = dim[key[i]] (every key < n_dim, else INVALID_ARG). */
ta_status ta_col_gather(ta_ctx* ctx, const uint32_t* key, uint64_t n, const uint32_t* dim,
                        uint32_t n_dim, uint32_t* out);

/* Scalar compare: mask[i] = col[i] > c.  Vector add: out[i] = a[i] + b[i].
 * In-place multiply: a[i] *= s.  Reduction sum: *sum (host) = sum of a.
 * Cumulative sum: out[i] = a[0] + ... + a[i].  Integer arithmetic modulo
 * 2^64. */
ta_status ta_col_compare(ta_ctx* ctx, const uint64_t* col, uint64_t n, uint64_t c, uint8_t* mask);
ta_status ta_col_add(ta_ctx* ctx, const uint64_t* a, const uint64_t* b, uint64_t n, uint64_t* out);
ta_status ta_col_scale(ta_ctx* ctx, uint64_t* a, uint64_t n, uint64_t s);
ta_status ta_col_sum(ta_ctx* ctx, const uint64_t* a, uint64_t n, uint64_t* sum);
ta_status ta_col_cumsum(ta_ctx* ctx, const uint64_t* a, uint64_t n, uint64_t* out);

/* ------------------------------------------------------ sharded form ---- */

/* One job's ranks split into contiguous shards, each loaded as its own
 * experiment (on its own GPU, or one after another): Section VI-B analyses
 * 100,000 ranks, the case sharding by rank serves.  Every per-rank product
 * (tensor, exclusive, inclusive) needs nothing from other shards.  The
 * cross-rank steps -- context statistics and outliers (Sections VI-A/B), the
 * rack rollup (Section VI-B) and the potential speedup (Section VI-A, Table
 * V) -- need one exchange of partials.  Every partial array below merges
 * element by element with SUM, MIN or MAX as stated, in any order or
 * grouping (an all-reduce, e.g. torch.distributed over NCCL), and the merge
 * is exact: integers only, 128-bit sums carried as four 32-bit limbs in
 * 64-bit words (limb l weighs 2^(32 l); a SUM of up to 2^32 shards cannot
 * overflow a limb).  The one exception is cv_within, a sum of FP64 terms:
 * merged across shards it agrees with the unsharded value to about 1e-15
 * relative per term added, not bit for bit.  The job's exactness contract is
 * the load contract applied to the whole job: n_total x longest span < 2^63.
 *
 * Protocol, with rank_base the global id of the shard's first rank and
 * n_total the job's rank count:
 *   1. ta_shard_stats_partials on every shard; merge sums (SUM), mins (MIN),
 *      maxs (MAX).
 *   2. ta_shard_stats_finalize with the merged arrays: every shard gets the
 *      job's per-context statistics and its own ranks' outliers (global rank
 *      ids, sorted by (ctx, rank); the shards' lists merged by (ctx, rank)
 *      are the job's list) and argmax candidates; merge the candidates (MIN)
 *      and write them with ta_shard_set_argmax.
 *   3. rack rollup: ta_shard_topology_partials on every shard (the same
 *      merged arrays), merge node_parts (SUM), ta_topology_finalize.
 *   4. speedup: ta_shard_speedup_bounds on every shard, merge (MIN, SUM,
 *      MAX); ta_shard_speedup_partials with the job's I*; merge (SUM, MAX,
 *      SUM); ta_speedup_finalize.
 * All arrays are device memory owned by the caller; calls run on the
 * experiment's (or context's) stream and return after their work. */

/* Reducible statistics partials of all n_ctx contexts over the shard's ranks
 * (a rank without the context counts 0, as in ta_context_stats). */
typedef struct ta_shard_stats_parts {
  uint64_t* sums; /* [6 n_ctx] SUM: per context present, S1 = sum x, S2 = sum x^2 as 4 limbs */
  uint64_t* mins; /* [n_ctx] MIN: min x over the shard's ranks */
  uint64_t* maxs; /* [n_ctx] MAX: max x */
} ta_shard_stats_parts;
ta_status ta_shard_stats_partials(ta_experiment* e, uint32_t metric, const ta_shard_stats_parts* out);

/* The merged partials every finishing call reads. */
typedef struct ta_shard_merged {
  uint32_t metric;
  uint32_t rank_base;       /* global id of this shard's first rank */
  uint32_t n_total;         /* ranks of the whole job */
  uint32_t tau_num, tau_den;
  const uint64_t* sums;     /* merged arrays of ta_shard_stats_parts */
  const uint64_t* mins;
  const uint64_t* maxs;
} ta_shard_merged;

/* Statistics of the whole job for every context (stats[n_ctx], argmax =
 * this shard's candidate until ta_shard_set_argmax), this shard's outliers
 * (global ids, sorted; TA_ERR_CAPACITY with n_outliers set when above
 * outlier_cap) and argmax[n_ctx]: the lowest global rank of this shard whose
 * value is the job's max (MIN-reducible; 0xFFFFFFFF: none here). */
typedef struct ta_shard_stats_out {
  ta_ctx_stats* stats;
  uint32_t* argmax;
  ta_outlier* outliers;
  uint64_t outlier_cap;
  uint64_t n_outliers; /* out */
} ta_shard_stats_out;
ta_status ta_shard_stats_finalize(ta_experiment* e, const ta_shard_merged* m, ta_shard_stats_out* o);
/* stats[c].argmax = argmax[c] for c < n_ctx (the merged candidates). */
ta_status ta_shard_set_argmax(ta_ctx* ctx, ta_ctx_stats* stats, const uint32_t* argmax,
                              uint32_t n_ctx);

/* Node partials of one context for the rack rollup (ta_topology_rollup over
 * the job): node_parts[3 n_nodes] SUM: per node its outlier ranks, sum of x
 * and ranks, over this shard's ranks; node_of_rank[shard R] maps the shard's
 * ranks to global node ids. */
ta_status ta_shard_topology_partials(ta_experiment* e, const ta_shard_merged* m, uint32_t ctx,
                                     const uint32_t* node_of_rank, uint32_t n_nodes,
                                     uint64_t* node_parts);
/* The rollup from merged node partials: flags (>= min_ranks outlier ranks),
 * chassis and rack counts and sums, flagged racks (t and o device, as in
 * ta_topology_rollup; t->node_of_rank unused). */
ta_status ta_topology_finalize(ta_ctx* ctx, const uint64_t* node_parts, const ta_topology* t,
                               uint32_t min_ranks, ta_topo_out* o);

/* bounds[3] (host): min n_iter (MIN), sum of n_iter (SUM) and longest span
 * (MAX) over the shard's ranks. */
ta_status ta_shard_speedup_bounds(ta_experiment* e, uint64_t* bounds);
/* Reducible speedup partials for contexts ctxs[nk] (device, sorted unique)
 * over iterations i < i_star (the job's I*): cells[5 i_star nk] SUM (per
 * (i, k): sum over ranks and the sum of squares as 4 limbs), cell_max[i_star
 * nk] MAX, within[nk] SUM (per context the shard's sum of its ranks' CV
 * terms, in the pairwise order of ta_potential_speedup). */
typedef struct ta_shard_speedup_parts {
  uint64_t* cells;
  uint64_t* cell_max;
  double* within;
} ta_shard_speedup_parts;
ta_status ta_shard_speedup_partials(ta_experiment* e, const uint32_t* ctxs, uint32_t nk,
                                    uint32_t i_star, const ta_shard_speedup_parts* out);
/* The speedup of the job from merged partials (outputs device, as in
 * ta_potential_speedup): excluded = sum of n_iter - n_total i_star, t_app =
 * app_time_ns or the merged longest span. */
ta_status ta_speedup_finalize(ta_ctx* ctx, uint32_t nk, uint32_t n_total, uint32_t i_star,
                              uint64_t excluded, uint64_t t_app,
                              const ta_shard_speedup_parts* merged, ta_speedup_ctx* per_ctx,
                              ta_speedup_total* total);

/* ------------------------------------------- allocation-free statistics ---- */

/* ta_context_stats over every context, for callers that must not allocate
 * device memory at call time -- for example a host runtime that manages all
 * device memory itself and hands libraries only buffers it already owns,
 * or a service whose device memory comes from a fixed budget that may not
 * grow.  It uses no allocator: its
 * temporaries live in one fixed device array inside this library (about 6 MB,
 * held by every GPU that loads the library until the process exits).  The
 * paper has no counterpart; this is an interface convenience.
 *   cuda_stream     stream to run on; the current device must be its device.
 *   off, ctx, time  a per-rank CSR on the device (e.g. ta_csr_get_view of an
 *                   experiment): rank r owns [off[r], off[r+1]), contexts
 *                   ascending, times in ns.  Checked on the device before
 *                   use: offsets that decrease return TA_ERR_INVALID_ARG, a
 *                   context id >= n_ctx returns TA_ERR_BAD_CTX (nothing is
 *                   computed).  The offsets must address the caller's arrays.
 *   n_ranks, n_ctx  R and C; n_ctx must not exceed 65536.
 *   ranks           sorted unique device rank ids, or NULL for all ranks.
 *   tau_num/tau_den outlier threshold, as in ta_context_stats.
 *   stats           device ta_ctx_stats[n_ctx] (context order).
 *   outliers        device ta_outlier[outlier_cap], sorted by (ctx, rank);
 *                   outlier_cap must not exceed 65536.
 *   n_outliers      host: set to the number of outliers (TA_ERR_CAPACITY if
 *                   above outlier_cap; then the outlier list is not written).
 * Results equal ta_context_stats with ctxs = NULL.  Returns after the work is
 * complete.  The first call on a device looks up the array's device address
 * (make that first call before any stream capture).  Every call reuses the
 * same array and resets what must start at zero; calls that overlap on the
 * GPU (other streams, other threads) race on it and must be serialised by the
 * caller.  Sizes above the limits return TA_ERR_INVALID_ARG. */
ta_status ta_context_stats_noalloc(void* cuda_stream, const uint64_t* off, const uint32_t* ctx,
                                   const uint64_t* time, uint32_t n_ranks, uint32_t n_ctx,
                                   const uint32_t* ranks, uint32_t n_ranks_subset,
                                   uint32_t tau_num, uint32_t tau_den, ta_ctx_stats* stats,
                                   ta_outlier* outliers, uint64_t outlier_cap,
                                   uint64_t* n_outliers);


/* ----------------------------------------------------- batched form ---- */

/* Many independent experiments (sets) analysed as one unit (the batched
 * execution form).  ta_batch_plan copies every set into one device arena
 * (ranks, samples and tree nodes concatenated; sample tiles never span two
 * sets), validates all of them, runs the analysis once to size every product
 * exactly, and captures the whole fixed launch sequence -- validation, the
 * iteration tensor (Section V), exclusive and inclusive CSR, and the
 * cross-rank statistics of the exclusive metric over all ranks of each set
 * (Section VI-A/B) -- in one CUDA graph.  Before capture an autotuner times
 * every launch shape of the tensor passes (4, 8 or 16 warps per CTA, 1 to the
 * resident maximum of CTAs per SM) on the batch's own data and keeps the
 * fastest (see ta_batch_info).  ta_batch_run replays that graph on
 * the context's stream (the inputs of the plan, already on the device, are
 * analysed again) and then sorts the outliers by set.
 *   sets[s]   as for ta_load_traces; parent ids and samples' context ids are
 *             local to their set; flags are ignored (every set is copied).
 *   args      tau = tau_num / tau_den (NULL: 3/1); outlier_cap = capacity of
 *             the outlier list over all sets (0: 2^20).
 * Every product of set s is the product ta_load_traces + ta_context_stats
 * (metric exclusive, all ranks, all contexts) -- and, when requested in
 * set_args, ta_potential_speedup and ta_topology_rollup -- would give for
 * that set alone;
 * ta_batch_get_set returns zero-copy device views with offsets relative to
 * the set (valid until ta_batch_free).  Errors: as ta_load_traces for any
 * set (the message names the set).  ta_batch_plan ends with one run; when
 * the outliers exceed outlier_cap, ta_batch_run returns TA_ERR_CAPACITY, the
 * info's n_outliers holds the full count, every set's outlier list is empty
 * and the other products are valid. */
typedef struct ta_batch ta_batch;
/* Optional per-set requests, computed for every set in the same graph:
 * the potential speedup (as ta_potential_speedup over all ranks of the set)
 * and the rack rollup of one context (as ta_topology_rollup, exclusive
 * metric, all ranks).  Host arrays, copied at plan time. */
typedef struct ta_batch_set_args {
  const uint32_t* speedup_ctxs;    /* sorted, unique set-local contexts; NULL = none */
  uint32_t n_speedup_ctxs;
  uint32_t topo_ctx;               /* rollup context (set-local)                     */
  uint64_t app_time_ns;            /* speedup denominator; 0 = longest rank span     */
  const uint32_t* node_of_rank;    /* [n_ranks]; NULL = no rollup                    */
  const uint32_t* rack_of_node;    /* [n_nodes]                                      */
  const uint32_t* chassis_of_node; /* [n_nodes]                                      */
  uint32_t n_nodes, n_chassis, n_racks;
  uint32_t topo_tau_num, topo_tau_den, topo_min_ranks;
} ta_batch_set_args;
typedef struct ta_batch_args {
  uint32_t tau_num, tau_den;
  uint64_t outlier_cap;
  const ta_batch_set_args* set_args; /* [n_sets] or NULL */
} ta_batch_args;
typedef struct ta_batch_info {
  uint32_t n_sets, n_ranks;
  uint64_t n_records, n_rows, tensor_nnz, excl_nnz, incl_nnz, n_outliers;
  uint64_t graph_nodes;   /* kernels, memsets and copies in the graph */
  uint64_t graph_kernels; /* kernel nodes among them                  */
  uint64_t device_bytes; /* arena owned by the batch                 */
  /* launch shape the autotuner chose for the tensor passes: warps per CTA
     and CTAs (count pass, write pass); trials run, the tile width (samples
     per tile: 4096 or 2048) and their total time */
  uint32_t count_warps, count_grid, write_warps, write_grid;
  uint32_t tune_trials, tile_width;
  double tune_ms;
} ta_batch_info;
typedef struct ta_batch_set_view {
  uint32_t n_ranks, n_ctx;
  ta_tensor_view tensor;       /* offsets relative to the set       */
  ta_csr_view exclusive;       /* off[n_ranks + 1] from 0           */
  ta_csr_view inclusive;
  const ta_ctx_stats* stats;   /* [n_ctx]                           */
  const ta_outlier* outliers;  /* sorted by (ctx, rank); local ids  */
  uint64_t n_outliers;
  /* potential speedup (NULL / 0 when not requested) */
  const ta_speedup_ctx* speedup; /* [n_speedup], in the request's order */
  const ta_speedup_total* speedup_total;
  uint32_t n_speedup, n_flagged_racks;
  /* rack rollup (NULL / 0 when not requested), as ta_topo_out */
  uint32_t n_nodes, n_chassis, n_racks, reserved;
  const uint32_t* node_outliers;
  const uint64_t* node_sum;
  const uint32_t* node_ranks;
  const uint8_t* node_flag;
  const uint32_t* chassis_flagged;
  const uint32_t* chassis_nodes;
  const uint64_t* chassis_sum;
  const uint32_t* rack_flagged;
  const uint32_t* rack_nodes;
  const uint64_t* rack_sum;
  const uint32_t* flagged_racks;
} ta_batch_set_view;
ta_status ta_batch_plan(ta_ctx* ctx, const ta_trace_desc* sets, uint32_t n_sets,
                        const ta_batch_args* args, ta_batch** out);
ta_status ta_batch_run(ta_batch* b);
ta_status ta_batch_free(ta_batch* b);
ta_status ta_batch_get_info(const ta_batch* b, ta_batch_info* info);
ta_status ta_batch_get_set(const ta_batch* b, uint32_t set, ta_batch_set_view* v);

/* ------------------------------------------------------ serving form ---- */

/* An interactive query server over resident experiments (the serving form).
 * Experiments loaded with ta_load_traces are registered with the server and
 * stay on the device (their derived products only).  Queries are submitted
 * from any host thread and answered asynchronously.  A worker thread admits
 * pending queries in arrival order as long as an in-flight slot and room in
 * the result, scratch and input-staging arenas are free (continuous
 * batching: queries that arrive while earlier batches run are packed into the
 * next batch); each batch is one descriptor upload, three kernel launches
 * over all of its queries (cut into per-chunk work items), and one download
 * of its results, and up to n_streams batches overlap on the device.
 * max_batch = 1 with n_streams = 1 runs one query per launch, one at a time
 * (the plain form the batching is measured against).
 *
 * Query kinds (slices and per-context views of the tri-dimensional model,
 * Sections V and VI; statistics as ta_context_stats, rollup as
 * ta_topology_rollup; time windows of the traces, Section III-A):
 *   TA_Q_STATS   statistics of context ctx over a rank subset (sorted, unique,
 *                host array, copied at submit), threshold tau:
 *                payload ta_q_stats = the ta_ctx_stats ta_context_stats gives
 *                for (ranks, ctxs = {ctx}) and the number of its outliers.
 *   TA_Q_SLICE   time of ctx in every (rank, iteration) cell of
 *                [r0, r1) x [i0, i1) (iteration rows only; 0 where absent or
 *                past the rank's last iteration): payload uint64 cells,
 *                row-major by rank.
 *   TA_Q_TOPK    the k ranks (1 <= k <= 1024) with the largest value of ctx
 *                over all ranks, equal values by lower rank, with x and the
 *                z-score over all ranks: payload uint64 count then
 *                ta_q_topk_entry[count].
 *   TA_Q_RACKS   rack rollup of ctx over all ranks (outlier rule tau,
 *                min_ranks) on the experiment's registered topology: payload
 *                ta_q_racks header, uint64 rack_sum[n_racks],
 *                uint32 rack_flagged[n_racks], uint32 rack_nodes[n_racks],
 *                uint32 flagged_racks[n_flagged_racks].
 *   TA_Q_WINDOW  exclusive time and samples of ctx in the time window
 *                [t0, t1) on every rank of [r0, r1), as ta_interval_profile
 *                (exclusive) would list them (0 where ctx is absent):
 *                payload uint64 time[r1 - r0] then uint64 cnt[r1 - r0].
 *                The experiment must have kept its traces
 *                (TA_LOAD_KEEP_TRACES or borrowed) when it was added; metric
 *                is ignored.
 * metric selects the exclusive or inclusive value (the inclusive rollup must
 * have been built).  Invalid queries are refused by ta_serve_submit
 * (TA_ERR_INVALID_ARG); a query larger than an arena returns
 * TA_ERR_CAPACITY. */
typedef struct ta_server ta_server;
#define TA_Q_STATS 1u
#define TA_Q_SLICE 2u
#define TA_Q_TOPK 3u
#define TA_Q_RACKS 4u
#define TA_Q_WINDOW 5u
typedef struct ta_serve_config {
  uint32_t max_batch;     /* queries per batch (0: 1024)                    */
  uint32_t n_streams;     /* batches in flight (0: 3)                       */
  uint32_t max_inflight;  /* admitted, unreleased queries (0: 8192)         */
  uint32_t reserved;
  uint64_t result_bytes;  /* device result arena + pinned mirror (0: 1 GiB) */
  uint64_t scratch_bytes; /* device scratch arena (0: 256 MiB)              */
  uint64_t staging_bytes; /* per-stream input staging (0: 32 MiB)           */
  uint64_t device_budget; /* resident experiment bytes (0: no limit)        */
} ta_serve_config;
typedef struct ta_query {
  uint32_t kind, experiment, metric, ctx;
  uint32_t tau_num, tau_den; /* STATS, RACKS        */
  uint32_t k;                /* TOPK               */
  uint32_t min_ranks;        /* RACKS              */
  uint32_t r0, r1, i0, i1;   /* SLICE              */
  const uint32_t* ranks;     /* STATS (host)        */
  uint32_t n_ranks;          /* STATS              */
  uint32_t reserved;
  uint64_t t0, t1;           /* WINDOW (r0, r1 too) */
} ta_query;
typedef struct ta_q_stats {
  ta_ctx_stats stats;
  uint64_t n_outliers;
} ta_q_stats;
typedef struct ta_q_topk_entry {
  uint32_t rank, reserved;
  uint64_t x;
  double z;
} ta_q_topk_entry;
typedef struct ta_q_racks {
  uint32_t n_racks, n_flagged_racks;
} ta_q_racks;
typedef struct ta_query_result {
  uint32_t status; /* ta_status of the query                            */
  uint32_t kind;
  uint64_t t_submit_ns, t_admit_ns, t_launch_ns, t_done_ns; /* steady clock */
  uint64_t bytes;   /* payload size                                      */
  const void* data; /* payload in the server's pinned host mirror, valid
                       until ta_serve_release of the ticket               */
} ta_query_result;
ta_status ta_serve_open(ta_ctx* ctx, const ta_serve_config* cfg, ta_server** out);
/* Waits for the batches on the device; pending queries are dropped. */
ta_status ta_serve_close(ta_server* s);
/* Registers a loaded experiment (which must outlive the server).  Admission
 * by memory: TA_ERR_OOM if its device bytes exceed what is left of
 * device_budget.  topo (host arrays, copied; may be NULL) enables rack
 * queries. */
ta_status ta_serve_add_experiment(ta_server* s, ta_experiment* e, const ta_topology* topo,
                                  uint32_t* experiment_id);
ta_status ta_serve_submit(ta_server* s, const ta_query* q, uint64_t* ticket);
/* Fills r when the query is done (waiting up to wait_ns; < 0 = forever);
 * TA_ERR_STATE while it is not. */
ta_status ta_serve_poll(ta_server* s, uint64_t ticket, int64_t wait_ns, ta_query_result* r);
/* Frees a finished query's result space and slot. */
ta_status ta_serve_release(ta_server* s, uint64_t ticket);
/* Open-loop replay: submits qs[i] at arrival_ns[i] after the start (host
 * steady clock) while a second thread collects results in order, writes
 * latency_ns[i] = done - arrival (queueing included) and releases them;
 * *wall_ns = start to last completion.  Returns the first failing status. */
ta_status ta_serve_replay(ta_server* s, const ta_query* qs, const uint64_t* arrival_ns,
                          uint64_t n, uint64_t* latency_ns, uint64_t* wall_ns);

#ifdef __cplusplus
}
#endif
#endif /* TA_H */
