/*
 * woodelf.h -- C ABI of the GB300 (sm_103a) Background-SHAP library.
 *
 * The library computes, for a decision-tree ensemble, a background matrix B (m rows)
 * and consumer rows C (n rows), the Background (interventional) Shapley value of every
 * feature for every consumer: the Shapley value (Eq. "s") of the game
 *     v_c(S) = (1/m) sum_{b in B} f(x^S),  x^S_i = c_i if i in S else b_i,
 * where f is the plain sum of the trees' leaf outputs (section "WOODELF Algorithm":
 * run per tree and sum).  It follows the paper's WOODELF route (Algorithm 3):
 *   set_background : per-leaf background decision-pattern counts (Algorithm 1 and
 *                    Eq. "bg_shap_derivation" step (d)), the Shapley pattern-pair
 *                    tables (Algorithm 2 with Formula "shap_simplified_formula"), and
 *                    their contraction s_{l,i} = w_l * M_{l,i} * f_l (step (f));
 *   explain        : consumer decision patterns, the lookup s_{l,i}[P[l][c]] and the
 *                    sum over leaves and trees (step (g)).
 *
 * Conventions (all entry points):
 *   - A row goes left at an inner node when x[feature] < threshold (strict float32
 *     compare; a NaN goes right) -- Def. "decision_tree".
 *   - Matrices are row-major float32 with a leading dimension (elements) >= the
 *     feature count.  phi is n x F row-major.
 *   - Pointers tagged WDF_MEM_DEVICE must be device memory of the context's GPU;
 *     WDF_MEM_HOST pointers are host memory (pinned memory gives asynchronous copies).
 *   - Every function returns a wdf_status and never throws; wdf_last_error() gives a
 *     thread-local message for the last failure on the calling thread.
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream).  Device work is
 *     enqueued on it and the call returns without waiting, except where stated.
 *   - The caller owns every buffer it passes; the library copies what it keeps.
 */
#ifndef WOODELF_H
#define WOODELF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WDF_OK = 0,
    WDF_EINVAL = 1,        /* malformed argument or call order */
    WDF_ENOMEM = 2,        /* a device or host allocation failed */
    WDF_ECUDA = 3,         /* a CUDA runtime call failed */
    WDF_EUNSUPPORTED = 4,  /* valid input the library does not handle (depth > 8, m == 0) */
    WDF_ETIMEOUT = 5,
    WDF_EBUSY = 6
} wdf_status;

/* Arithmetic of the contraction s = w * M * f (Eq. "bg_shap_derivation" step (f)). */
typedef enum {
    WDF_FP32 = 0,    /* FP32 operands, FP32 accumulation (CUDA cores) */
    WDF_TF32X3 = 1,  /* TF32 hi+lo split operands, three tensor-core products, FP32 accumulation */
    WDF_BF16X3 = 2,  /* BF16 hi+lo split operands, three tensor-core products, FP32 accumulation
                        (16 significant bits per operand: relative error about 2^-16 where a
                        background count exceeds 2^16 or a table value needs more bits) */
    WDF_BF16X6 = 3   /* BF16 hi+mid+lo split operands (exact for every FP32 value), the six
                        tensor-core products of total order <= 2, FP32 accumulation: FP32 accuracy */
} wdf_precision;

typedef enum { WDF_MEM_HOST = 0, WDF_MEM_DEVICE = 1 } wdf_memkind;

/* Which value of the game is computed (section "Beyond SHAP"): Shapley values
 * (Formula "shap_simplified_formula") or Banzhaf values (Formula
 * "banzhaf_simplified_formula"); only the pattern-pair table differs. */
typedef enum { WDF_SHAPLEY = 0, WDF_BANZHAF = 1 } wdf_metric;

typedef struct wdf_ctx wdf_ctx;
typedef struct wdf_ensemble wdf_ensemble;

typedef struct {
    int32_t n_features;      /* F */
    int32_t n_trees;         /* T */
    int32_t depth;           /* D: every tree is laid out as a complete tree of this depth */
    int32_t n_live_leaves;   /* leaves with a non-zero output after that layout */
    int32_t n_signatures;    /* distinct repeated-feature patterns of the live paths */
    int32_t has_background;  /* 1 after a successful wdf_set_background */
    int64_t device_bytes;    /* device memory the ensemble holds */
} wdf_info;

/* Context bound to one CUDA device.  Returns WDF_ECUDA if the device is absent.
 * wdf_ctx_destroy releases the caller's handle; the ensembles, batches and servers made
 * from the context hold it too, so they may be destroyed after it (the context is freed
 * with the last of them). */
wdf_status wdf_ctx_create(int32_t device, wdf_ctx **out);
void wdf_ctx_destroy(wdf_ctx *ctx);

/*
 * Load an ensemble (host arrays, copied).  Trees are stored back to back:
 * tree_offset[t] is the flat index of tree t's root, tree_offset[n_trees] the node
 * count.  Per node: feature (-1 for a leaf, else in [0, n_features)), threshold,
 * left/right child indices local to the tree (-1 for a leaf), value (leaf output).
 * Definition: Def. "decision_tree" (binary nodes, leaf outputs w_l, strict split).
 * WDF_EINVAL: offsets not increasing, a child index out of range, a node reached
 * twice or never, a feature out of range.  WDF_EUNSUPPORTED: a leaf deeper than 8
 * (patterns are 8-bit, section "Algorithmic Improvements" item 5).  Blocks until the
 * ensemble is resident on the device.
 */
wdf_status wdf_load_ensemble(wdf_ctx *ctx, int32_t n_features, int32_t n_trees, const int64_t *tree_offset,
                             const int32_t *feature, const float *threshold, const int32_t *left,
                             const int32_t *right, const float *value, wdf_ensemble **out);
void wdf_ensemble_destroy(wdf_ensemble *ens);
wdf_status wdf_ensemble_info(const wdf_ensemble *ens, wdf_info *out);

/*
 * Set the background B (m x F, leading dimension ldb) and run the consumer-independent
 * half of Algorithm 3: background pattern counts (step 1), pattern-pair tables (step
 * 2) and their contraction (step 3), in the given precision.  B is not retained; its
 * decision codes pass through a buffer the ensemble keeps (up to 2^20 rows of codes).
 * Calls on one ensemble must not overlap on the GPU.
 * WDF_EUNSUPPORTED: m == 0 (an empty background is the path-dependent variant).
 * precision WDF_TF32X3 / WDF_BF16X3 / WDF_BF16X6 runs the contraction on the tensor cores (tcgen05,
 * TMEM accumulators) and then waits for the stream to check the kernel's bounded waits:
 * WDF_ETIMEOUT if one expired.  WDF_FP32 is stream-ordered without waiting; a later
 * wdf_explain on the same stream sees the result.
 */
wdf_status wdf_set_background(wdf_ensemble *ens, const float *B, int64_t m, int64_t ldb, wdf_memkind kind,
                              wdf_precision precision, void *stream);

/* The background in shards (for background rows split across devices or arriving in
 * parts): step 1 of Algorithm 3 produces joint pattern counts that are plain sums over
 * the background rows (Eq. "bg_shap_derivation" step (d)), so the counts of disjoint
 * shards add up to the counts of their union.
 * wdf_background_counts_size: the number of u32 counts (T * 2^(D-2) * 2^(D+1)); -1 for
 * a null ensemble.
 * wdf_background_counts: ADDS the counts of rows B (DEVICE memory, m x F, stride ldb)
 * into counts (DEVICE memory, wdf_background_counts_size u32, zeroed by the caller
 * before the first shard).  Shares the ensemble's code buffer with wdf_set_background:
 * calls on one ensemble must not overlap on the GPU.
 * wdf_set_background_counts: finishes the background from summed counts (DEVICE
 * memory) of m_total rows in total, exactly as wdf_set_background would from all the
 * rows at once (the same counts give the same tables, folded vectors and results).
 * WDF_EUNSUPPORTED for m_total < 1 or more than 2^32 - 1 rows. */
int64_t wdf_background_counts_size(const wdf_ensemble *ens);
wdf_status wdf_background_counts(wdf_ensemble *ens, const float *B, int64_t m, int64_t ldb, uint32_t *counts,
                                 void *stream);
wdf_status wdf_set_background_counts(wdf_ensemble *ens, const uint32_t *counts, int64_t m_total,
                                     wdf_precision precision, void *stream);

/*
 * Path-Dependent values (section "Efficient Path-Dependent SHAP Equation"): the
 * baseline pattern frequencies come from the nodes' covers (the number of training rows
 * that reached each node) instead of a background, Eq. "path_dependent_estimation":
 * f_l[p_b] = product over the path of r_i = cover(n_{i+1}) / cover(n_i) where bit i of
 * p_b is 1 and of 1 - r_i where it is 0.
 * wdf_set_covers: one cover per input node, indexed like the arrays of
 * wdf_load_ensemble (host, copied); WDF_EINVAL if one is negative or not finite.  A
 * node of zero cover gives its children ratio 0.  Synchronous.
 * wdf_set_path_dependent: replaces the background state by the path-dependent one
 * (then wdf_explain gives path-dependent values and wdf_expected_value the expected
 * output under the covers).  WDF_EINVAL without covers.  Stream-ordered like
 * wdf_set_background.
 */
wdf_status wdf_set_covers(wdf_ensemble *ens, const double *cover);
wdf_status wdf_set_path_dependent(wdf_ensemble *ens, wdf_precision precision, void *stream);

/* Select Shapley (the default) or Banzhaf values: rebuilds the pattern-pair tables
 * (Algorithm 2 with the metric's cube formula, section "Beyond SHAP"; Algorithm 3's
 * function v).  The background must be set again afterwards.  Synchronous. */
wdf_status wdf_set_metric(wdf_ensemble *ens, wdf_metric metric);

/*
 * phi[c, i] for the n consumer rows C (leading dimension ldc) into phi (leading
 * dimension ldphi >= F): Algorithm 3 step 4 / Eq. "bg_shap_derivation" step (g).
 * C and phi live in the same memory kind.  WDF_EINVAL if no background was set.
 * Device kind: asynchronous; the rows' decision codes (one or two bytes per code column
 * and row, at most 2^20 rows at a time) live in a temporary stream-ordered allocation,
 * so calls on different streams never share scratch memory.  Host kind: copies
 * through the ensemble's device staging buffers and returns once phi is written on the
 * host.  phi of a row does not depend on the other rows of the call (the same
 * floating-point additions in the same order).
 */
wdf_status wdf_explain(wdf_ensemble *ens, const float *C, int64_t n, int64_t ldc, wdf_memkind kind,
                       float *phi, int64_t ldphi, void *stream);

/* Pairwise interaction values of the same game (section "Beyond SHAP"): Shapley
 * interaction values phi_ij = phi_{j|i=1} - phi_{j|i=0} (Def. "shap_iv_def", computed
 * per cube with Table "table_shap_iv") when the metric is WDF_SHAPLEY, Banzhaf
 * interaction values (Def. "banzhaf_iv_def", Formula
 * "banzhaf_simplified_formula_interactions") when it is WDF_BANZHAF.
 * C: n x F consumer rows (DEVICE memory, row stride ldc >= F).  out: DEVICE memory, row
 * r of the result at out + r * ldo (ldo >= F * F), F x F row-major per row: symmetric,
 * out[i][j] = out[j][i] = the value of the pair (i, j), diagonal 0.  FP32 results from
 * an FP32 contraction of FP64-built tables; the additions into one element come from
 * many threads, so the last bits may change between runs.  Stream-ordered; takes a
 * temporary stream-ordered allocation (pair tables and per-leaf pair vectors).
 * WDF_EINVAL without a background (or path-dependent frequencies), for null pointers
 * or short strides. */
wdf_status wdf_explain_interactions(wdf_ensemble *ens, const float *C, int64_t n, int64_t ldc, float *out,
                                    int64_t ldo, void *stream);

/* E_b f(b), the value of the empty coalition, in FP64 (efficiency property, Appendix
 * B: sum_i phi_i(c) = f(c) - E_b f(b)).  Waits for the background to be processed. */
wdf_status wdf_expected_value(const wdf_ensemble *ens, double *out, void *stream);

/*
 * Global attribution over n explained rows (device pointers): mean_abs[i] =
 * (1/n) sum_c |phi[c,i]| and mean[i] = (1/n) sum_c phi[c,i], accumulated in FP64 in a
 * fixed order (the paper's global attribution combines many local attributions,
 * section "Introduction"), so the result does not depend on scheduling.  With packed
 * rows (ldphi == n_features <= 512, 16-byte aligned phi) short runs of 8 values are
 * first summed as exact-error FP32 pairs (TwoSum; within 2^-42 of the run's exact sum)
 * and each pair is then added in FP64.  mean_abs and mean are device arrays of F
 * doubles.  Asynchronous.
 */
wdf_status wdf_global_attribution(wdf_ctx *ctx, const float *phi, int64_t n, int64_t ldphi, int32_t n_features,
                                  double *mean_abs, double *mean, void *stream);

/*
 * Ragged batches (project addition; the paper runs one tree ensemble at a time).
 * A batch groups ensembles of one context -- any depths 2..8 and feature counts -- so a
 * single call explains many requests against them with ONE CUDA-graph launch: the graph
 * copies a packed work description (one memcpy) and runs, per depth class on parallel
 * branches, an encode kernel (the requests' decision codes into a device arena the
 * batch keeps and grows as needed) and a persistent consumer kernel over (ensemble,
 * request, tile of consumer rows) work items.  Per-row results equal those of
 * wdf_explain bit for bit.
 *
 * wdf_batch_create: the ensembles must outlive the batch; their backgrounds may be set
 * (or reset) later but before wdf_batch_explain.
 * wdf_batch_explain: request i explains n[i] rows at C[i] (device memory, row stride
 * ldc[i]) against ensembles[ensemble_index[i]] into phi[i] (device, stride ldphi[i]).
 * Stream-ordered and asynchronous; the caller may reuse its request arrays on return.
 * WDF_EINVAL for an index out of range, a missing background or bad sizes.
 * wdf_batch_autotune: runs each depth class's kernel on the given requests with every
 * consumer-tile size that fits (32, 64, 128 rows), reps timed runs each, and keeps the
 * fastest per class (phi is written with valid results).  cache_path (nullable): a text
 * file of "depth features code_bytes tile_rows ms" lines (features and decision-code
 * bytes per row of the class, rounded up to 32) read first and appended to.  Synchronous.  wdf_batch_tile_rows reports the tile size of a depth class (-1 if
 * the batch has none).
 */
typedef struct wdf_batch wdf_batch;
wdf_status wdf_batch_create(wdf_ctx *ctx, int32_t n_ensembles, wdf_ensemble *const *ensembles, wdf_batch **out);
void wdf_batch_destroy(wdf_batch *batch);
wdf_status wdf_batch_explain(wdf_batch *batch, int32_t n_requests, const int32_t *ensemble_index,
                             const float *const *C, const int64_t *n, const int64_t *ldc, float *const *phi,
                             const int64_t *ldphi, void *stream);
wdf_status wdf_batch_autotune(wdf_batch *batch, int32_t n_requests, const int32_t *ensemble_index,
                              const float *const *C, const int64_t *n, const int64_t *ldc, float *const *phi,
                              const int64_t *ldphi, int32_t reps, const char *cache_path, void *stream);
wdf_status wdf_batch_tile_rows(const wdf_batch *batch, int32_t depth, int32_t *tile_rows);

/*
 * Continuous-batching server (project addition).  Requests in host memory queue in
 * arrival order and are served in parts of at most 8192 rows.  Whenever one of n_slots
 * execution slots is free, a scheduler thread fills a wave by taking one part from each
 * queued request in turn (round robin, so a large request does not hold back the ones
 * behind it) until the wave has max_wave_requests parts, about 16M rows x trees of
 * work, or the next part's device buffers (2 * rows * F * 4 bytes) would exceed
 * device_budget_bytes; it runs the wave as copies in, ONE batch launch
 * (wdf_batch_explain) and copies out on the slot's stream.  Waves of different slots
 * overlap on the GPU.  With four or more slots, slot 0 is an express slot: it takes only
 * requests of at most 2^20 rows x trees of remaining work, in waves of at most 2^22
 * rows x trees, so small requests do not queue behind large parts.  A request whose next part does not fit the remaining
 * budget is passed over for smaller ones at most 8 fills in a row; then the fill stops
 * at it until memory frees up.  A request completes with its last part.  Every ensemble
 * must have its background set and must outlive the server.  A request's phi equals
 * what wdf_explain gives for the same rows, whatever shares its waves.
 * wdf_server_submit: C (n x F, row stride ldc) is read and phi (row stride ldphi)
 * written asynchronously: both must stay valid until wdf_server_wait / _poll reports the
 * ticket done.  WDF_ENOMEM if one part of the request (min(n, 8192) rows) alone exceeds
 * the budget, WDF_EBUSY while shutting down.  wdf_server_wait: WDF_ETIMEOUT if not done
 * within timeout_ms (the request stays queued or in flight).  A request whose wave
 * failed on the device is reported done with WDF_ECUDA, only after its slot's stream
 * has finished with its buffers.
 * wdf_server_request_ms: the latency (submit to completion, milliseconds) of a completed
 * request; WDF_EINVAL for an unknown or unfinished ticket.
 * wdf_server_stats: latency percentiles are over requests completed since creation or
 * the last wdf_server_reset_stats, measured from submit to completion; rows_per_s over
 * the span from the first submit to the last completion.  wdf_server_reset_stats also
 * forgets the tickets of completed requests (later waits, polls and latency queries on
 * them return WDF_EINVAL), which keeps a long-running server's bookkeeping bounded.  wdf_server_destroy finishes
 * every queued request first.
 */
typedef struct wdf_server wdf_server;
typedef struct {
    int64_t submitted, completed, queued, waves, rows_completed;
    double p50_ms, p99_ms, max_ms, rows_per_s;
    int64_t device_bytes_in_use, device_budget;
} wdf_serving_stats;
wdf_status wdf_server_create(wdf_ctx *ctx, int32_t n_ensembles, wdf_ensemble *const *ensembles,
                             int64_t device_budget_bytes, int32_t n_slots, int32_t max_wave_requests,
                             wdf_server **out);
wdf_status wdf_server_submit(wdf_server *server, int32_t ensemble_index, const float *C, int64_t n, int64_t ldc,
                             float *phi, int64_t ldphi, uint64_t *ticket);
wdf_status wdf_server_wait(wdf_server *server, uint64_t ticket, int64_t timeout_ms);
wdf_status wdf_server_poll(wdf_server *server, uint64_t ticket, int32_t *done);
wdf_status wdf_server_request_ms(wdf_server *server, uint64_t ticket, double *ms);
wdf_status wdf_server_stats(wdf_server *server, wdf_serving_stats *out);
wdf_status wdf_server_reset_stats(wdf_server *server);
void wdf_server_destroy(wdf_server *server);

/*
 * wdf_global_attribution without any device allocation.  The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory when they need the
 * reduction -- code running under a framework whose caching allocator already holds the
 * GPU's memory (a raw cudaMalloc there can fail), or latency-critical loops where an
 * allocation or free may block the host or synchronise the device.
 * Same arguments and the same result (same kernels, same summation order) as
 * wdf_global_attribution, with the device index in place of a context.  The FP64
 * partial sums live in a fixed 2 MiB array of device memory inside the library (held on
 * every GPU that loads the library until the process exits); WDF_EINVAL when
 * ceil(n / 4096) * n_features * 2 exceeds its 262,144 doubles (for 127 features: up to
 * about 4.2 million rows).  Calls share that array and it keeps the last call's
 * contents: calls that overlap on the GPU race and must be ordered (e.g. one stream).
 * The first call on a device looks up the array's address with that device current;
 * make it before any stream capture begins.  stream must belong to `device`.
 * Asynchronous.
 */
wdf_status wdf_global_attribution_noalloc(int32_t device, const float *phi, int64_t n, int64_t ldphi,
                                          int32_t n_features, double *mean_abs, double *mean, void *stream);

/*
 * Inspection, used by the tests.
 * wdf_debug_leaf_hist: the background pattern counts vc[l][p_b] (Eq.
 * "bg_shap_derivation" step (d)) of every leaf of the complete depth-D layout, as
 * uint32 [T][2^D][2^D] on the host (out_elems must be >= T * 4^D); leaf q of tree t is
 * the q-th leaf from the left, pattern bits root first.  Synchronous.
 * wdf_debug_pair_table: the FP64 pattern-pair table of one path shape, built on the
 * device (Algorithm 2 + Formula "shap_simplified_formula" or
 * "banzhaf_simplified_formula", unit leaf weight): out[p_b][k * 2^D + p_c] for path
 * position k, where first[k] is the first path position holding the same feature as
 * position k (first[k] == k for a new feature); the value of a feature is stored at
 * its first position, later ones hold 0.  Host output of 2^D * D * 2^D doubles.
 * Synchronous.
 */
wdf_status wdf_debug_leaf_hist(const wdf_ensemble *ens, uint32_t *out, int64_t out_elems);
wdf_status wdf_debug_pair_table(wdf_ctx *ctx, int32_t depth, const int32_t *first, wdf_metric metric, double *out);

/* Failure-detection hook for tests (process-wide, not thread-safe against concurrent
 * contractions): the first mbarrier wait of every CTA of later tensor-core contractions
 * polls at most `polls` times (polls <= 0 restores the normal limit of 2^22 polls).  A
 * wait that gives up makes wdf_set_background (or wdf_set_background_counts,
 * wdf_set_path_dependent) return WDF_ETIMEOUT with the background left unset; the kernel
 * still waits at the normal limit for its own tensor-core work before it frees its
 * tensor memory and returns, so the context stays usable.  The paper has no
 * counterpart: this exists so that the bounded waits can be shown to end in an error
 * status without faulting or hanging the GPU. */
void wdf_debug_contract_wait_limit(int32_t polls);

/* Number of kernels this library has launched in the process so far (all devices).
 * Benchmarks read it before and after a timed region. */
int64_t wdf_launch_count(void);

/* Consumer-kernel timing (process-wide; a measurement aid with no counterpart in the
 * paper).  wdf_explain_timing(1) makes every later wdf_explain bracket each launch of
 * its consumer kernel (Algorithm 3 step 4, one launch per 2^20 rows) with a pair of CUDA
 * events on the call's stream; wdf_explain_timing(0) stops; either call forgets the
 * pairs recorded so far.  wdf_explain_timing_read waits for the recorded pairs, writes
 * their summed milliseconds and their count (the launches timed), and forgets them.
 * Reading while another thread is inside wdf_explain returns only the pairs that call
 * has finished recording.  WDF_EINVAL for null outputs, WDF_ECUDA if an event fails. */
wdf_status wdf_explain_timing(int32_t enable);
wdf_status wdf_explain_timing_read(double *ms, int64_t *launches);

const char *wdf_last_error(void);
const char *wdf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* WOODELF_H */
