/*
 * dfdm.h -- C ABI of the GB300 fast directional matrix-vector product.
 *
 * The library computes g = A v for the Helmholtz matrix of Eq. (1) of
 * Of & Watschinger, "Complexity Analysis of a Fast Directional
 * Matrix-Vector Multiplication":
 *
 *     A[j,k] = exp(i kappa |x_j - y_k|) / (4 pi |x_j - y_k|),
 *
 * x_j in P_T (targets), y_k in P_S (sources), by the fast directional method
 * of Sect. 2 (Alg. 4) over uniform box cluster trees (Alg. 1), the block
 * partition of Alg. 2, and the directions of Alg. 3 / Def. 3 / Def. 5.
 * A coincident (bitwise equal) target/source pair contributes 0, the zero
 * diagonal of Sect. 4.
 *
 * Conventions shared by every call:
 *   - Every call returns a dfdm_status; none aborts or exits.  On an error,
 *     dfdm_last_error() returns a description (thread-local, never NULL).
 *   - Points are N x 3 row-major doubles (x0 y0 z0 x1 y1 z1 ...).
 *   - Complex vectors are interleaved (re, im) pairs: complex128 = 2 doubles
 *     (precision DFDM_FP64), complex64 = 2 floats (tensor-core precision).
 *   - Streams are passed as `void*` holding a cudaStream_t (NULL = the
 *     legacy default stream).  Device work is ordered on that stream.
 *   - The caller owns every buffer it passes; the plan owns all device
 *     tables it creates and frees them in dfdm_plan_destroy.
 */
#ifndef DFDM_H
#define DFDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DFDM_OK = 0,
  DFDM_ERR_INVALID_ARG = 1, /* bad pointer, size, parameter or point      */
  DFDM_ERR_OOM = 2,         /* device or host allocation failed           */
  DFDM_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  DFDM_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up          */
  DFDM_ERR_NUMERIC = 5,     /* a scale or value left its representable range */
  DFDM_ERR_UNSUPPORTED = 6  /* valid input the library does not handle yet */
} dfdm_status;

typedef enum {
  /* Every phase in FP64 on the CUDA cores. */
  DFDM_FP64 = 0,
  /* Coupling (M2L) products on the tcgen05 tensor cores with operands split
   * into two FP16 terms (hi + lo, three products hi*hi + hi*lo + lo*hi) and
   * FP32 accumulation, local expansions summed in FP64; the other phases in
   * FP32 with FP64 argument reduction of kappa |x - y| and of the
   * plane-wave phases.  Orders 2..6. */
  DFDM_TC_FP16X3 = 1
} dfdm_precision;

typedef struct {
  int order;        /* Chebyshev nodes per axis, o = m + 1 (m: degree of Eq. 4); 2..10 */
  int max_depth;    /* tree depth cap D (Alg. 1 never refines below it); 0..10   */
  int n_max;        /* Alg. 1 leaf size; 0 = refine every non-empty box to D     */
  double eta2;      /* eta_2 of (A1), (A3); default 5 (Sect. 4)                  */
  int l_hf;         /* largest high-frequency level (Eq. 11); -2 = default rule:
                       largest l with kappa * w_l > 2 (w_l = box side), else -1 */
  int root_mode;    /* 0: root cube [root_lo, root_lo + root_side]^3;
                       1: smallest power-of-two cube on a dyadic corner that
                          holds P_T and P_S                                      */
  double root_lo[3];
  double root_side;
  int precision;    /* dfdm_precision                                            */
  int nrhs_max;     /* largest nrhs dfdm_apply will be called with (>= 1)        */
} dfdm_params;

/* Counters of a plan (Table 1 quantities and sizes). */
typedef struct {
  int64_t n_targets, n_sources;
  int32_t depth;            /* p = depth of both trees (uniform)              */
  int32_t l_hf;             /* largest high-frequency level used              */
  int64_t n_coupling;       /* N_C: admissible blocks (t,s) in L+, both boxes non-empty */
  int64_t n_stored_coupling;/* N_SC: distinct (level, box offset) operators   */
  int64_t n_near_blocks;    /* inadmissible leaf blocks in L-                 */
  int64_t nf_entries;       /* sum over L- of #t^ * #s^ (nearfield entries)   */
  int64_t n_leaves_t, n_leaves_s; /* non-empty leaf boxes                     */
  int64_t device_bytes;     /* device memory held by the plan                 */
  int32_t level_dirs[16];   /* direction slots per level (|D_used(l)|)        */
  int64_t level_coupling[16]; /* N_C per level                                */
  int32_t level_offsets[16];  /* N_SC per level                               */
} dfdm_stats;

typedef struct dfdm_plan_s *dfdm_plan;

/* Fills *p with the defaults: order 5, max_depth 6, n_max 0, eta2 5,
 * l_hf -2 (rule), root_mode 0 with the unit cube [0,1]^3, DFDM_FP64,
 * nrhs_max 1.  Returns DFDM_ERR_INVALID_ARG for p == NULL. */
dfdm_status dfdm_params_default(dfdm_params *p);

/* Builds both trees (Alg. 1, Morton-keyed, Sect. 2.1), the partition
 * (Alg. 2 / Def. 2, stored as per-level box-offset tables), the directions
 * (Alg. 3, Def. 3, Def. 5) and every operator the apply needs (coupling
 * matrices once per level and offset, 8 reference transfer matrices per
 * level, directional phase diagonals: Sect. 2.7).
 *
 * targets, sources: HOST pointers, n_t x 3 and n_s x 3 doubles; copied.
 * kappa > 0.  Errors: INVALID_ARG for kappa <= 0 or not finite, n < 1,
 * non-finite coordinates, points outside the root cube (root_mode 0),
 * order outside 2..10, max_depth outside 0..10, eta2 <= 0;
 * UNSUPPORTED for the tensor-core form at orders above 6, and when the two
 * trees are not both of uniform depth (all leaves
 * on one level p; always true for n_max = 0); OOM; CUDA.
 * On success *out receives the plan; on failure *out is NULL.  The work is
 * done on `stream`; the call returns after it finished. */
dfdm_status dfdm_plan_create(const double *targets, int64_t n_t,
                             const double *sources, int64_t n_s, double kappa,
                             const dfdm_params *params, void *stream,
                             dfdm_plan *out);

/* g = A v by Alg. 4 (S2M, M2M, M2L, L2L, L2T, nearfield), for nrhs
 * right-hand sides.  x: DEVICE pointer, nrhs vectors of n_s complex values
 * in the caller's source order, vector r at x + r * n_s (complex128 for
 * DFDM_FP64, complex64 for DFDM_TC_FP16X3).  y: DEVICE pointer, nrhs
 * vectors of n_t complex values in the caller's target order, overwritten.
 * 1 <= nrhs <= params.nrhs_max.  Asynchronous on `stream`; no host sync.
 * Errors: INVALID_ARG (NULL, nrhs), CUDA, NUMERIC (a moment scale left the
 * FP16 range; reported by the next call of dfdm_plan_check). */
dfdm_status dfdm_apply(dfdm_plan plan, const void *x, void *y, int nrhs,
                       void *stream);

/* The same product with HOST buffers: copies x to the device, applies, and
 * copies y back, all on `stream`; returns after y is on the host. */
dfdm_status dfdm_apply_host(dfdm_plan plan, const void *x_host, void *y_host,
                            int nrhs, void *stream);

/* Synchronises `stream` and reports a device-side error flag raised by an
 * earlier apply (a bounded wait that gave up: TIMEOUT; a scale overflow:
 * NUMERIC), then clears it. */
dfdm_status dfdm_plan_check(dfdm_plan plan, void *stream);

/* Copies the plan's counters into *st (host). */
dfdm_status dfdm_plan_stats(dfdm_plan plan, dfdm_stats *st);

/* Device time of the phases of Alg. 4, summed over the dfdm_apply calls made
 * since timing was turned on or last read (and over their right-hand sides),
 * from CUDA events recorded on each apply's stream (milliseconds).  m2l_ms[l]
 * is the multiplication phase of level l; launches counts the library's kernel
 * launches of those applies, applies the applies. */
typedef struct {
  double s2m_ms, m2m_ms, split_ms, l2l_ms, l2t_ms, near_ms, total_ms;
  double m2l_ms[16];
  int64_t launches;
  int64_t applies;
} dfdm_timing;

/* Turns per-phase event timing of later applies on (enable != 0) or off and
 * drops any segments not yet read.  Timing adds event records to the stream
 * but no synchronisation; the events of consecutive applies accumulate until
 * dfdm_plan_timing reads them. */
dfdm_status dfdm_plan_set_timing(dfdm_plan plan, int enable);

/* Waits for the events of the applies since timing was turned on or last
 * read, fills *t with their sums and starts a new accumulation.  Returns
 * INVALID_ARG when timing is off or no apply ran since then.
 * dfdm_plan_autotune drops segments not yet read. */
dfdm_status dfdm_plan_timing(dfdm_plan plan, dfdm_timing *t);

/* Launch shapes chosen by dfdm_plan_autotune and what they measured. */
typedef struct {
  int m2l_nsplit[16]; /* per level l: chunks the M2L operator lists of a tile
                         are cut into (0: the level has no M2L)            */
  int p2p_threads;    /* nearfield block size (0: small-leaf kernel, fixed) */
  int p2p_chunks;     /* nearfield target chunks per leaf                   */
  double rule_ms;     /* one product with the built-in rule (0: from cache) */
  double tuned_ms;    /* one product with the chosen shapes (0: from cache) */
  int products;       /* products timed (0: from cache)                    */
  int from_cache;     /* 1: taken from cache_path without timing           */
} dfdm_tuning;

/* Measured tuner of the tensor-core form's launch shapes: how many chunks
 * every level's M2L operator lists are cut into (Alg. 4, multiplication
 * phase) and the nearfield's block size and target chunks per leaf.  A few
 * candidates per level (the built-in rule's first) are timed on whole
 * products of x with CUDA events on `stream` (per-level M2L and nearfield
 * times, the better of two products per candidate, after one untimed
 * product); the fastest per level and for the nearfield are kept, and
 * later applies use them, unless the tuned product is slower than the
 * rule's, in which case the rule stays.  The result does not depend on the
 * shapes beyond the rounding order of sums.
 * x: DEVICE pointer, one right-hand side (complex64, n_s values).
 * cache_path (may be NULL): a JSON-lines file.  A line whose "key" equals
 * this plan's shape key (device name, SM count, order, depth, per level the
 * grid, direction slots and operator list length, leaf count and sizes) is
 * applied without timing; otherwise the result is appended as one line.
 * out (may be NULL) receives the choice.  Synchronises the stream.
 * Errors: INVALID_ARG (NULL plan or x, an FP64 plan, cache_path not
 * writable, a cache line that does not parse), CUDA, OOM, TIMEOUT. */
dfdm_status dfdm_plan_autotune(dfdm_plan plan, const void *x,
                               const char *cache_path, void *stream,
                               dfdm_tuning *out);

/* Exports one level of one tree for bit-exact comparison with Alg. 1:
 * which = 0 targets, 1 sources; 0 <= level <= depth.  With keys == NULL only
 * *nboxes is set.  Otherwise keys/begin/end must hold *nboxes entries: the
 * Morton key of every non-empty box on the level (x in bit 0, Sect. 2.1
 * child order bx + 2 by + 4 bz), in ascending key order, and its [begin, end)
 * range in the sorted point order.  perm (n points, may be NULL) receives the
 * original index of every sorted point: points are sorted by their leaf's
 * key, and within a leaf by ascending original index (a box above the leaf
 * level holds the runs of its leaves in key order). */
dfdm_status dfdm_plan_export_tree(dfdm_plan plan, int which, int level,
                                  int64_t *nboxes, int64_t *keys,
                                  int64_t *begin, int64_t *end,
                                  int64_t *perm);

/* Exports the coupling structure of one level: for target boxes of parity
 * alpha = (ax, ay, az) (bit i = box coordinate i mod 2), the offsets
 * d = t - s (integer box units) of all admissible blocks of Alg. 2 whose
 * parent pair is inadmissible, and the index of c_(l)(t,s) (Def. 3) in
 * D^(l) for each (0 on low-frequency levels).  alpha_index = ax + 2 ay + 4 az.
 * With offsets == NULL only *count is set; else offsets holds 3 * *count
 * int32 and dirs *count int32.  level 0 .. depth. */
dfdm_status dfdm_plan_export_offsets(dfdm_plan plan, int level,
                                     int alpha_index, int32_t *count,
                                     int32_t *offsets, int32_t *dirs);

/* Rows of the exact product of Eq. (1) by direct summation in FP64 on the GPU
 * (the direct computation Sect. 4 compares the method with):
 *     y[r] = sum_k A[rows[r], k] x[k],  r = 0 .. nrows-1,
 * a coincident target/source pair contributing 0.  No plan is needed.
 * targets (n_t x 3), sources (n_s x 3): DEVICE doubles, row-major; x: DEVICE
 * complex128, n_s entries; rows: DEVICE int64, nrows entries; y: DEVICE
 * complex128, nrows entries, overwritten.  A row index outside [0, n_t)
 * gives NaN in its y entry.  The sources are split into chunks summed by
 * separate blocks; the partial sums go to a scratch array of at most
 * 64 x nrows complex128 that this call allocates and frees in stream order
 * (cudaMallocAsync / cudaFreeAsync on `stream`).  Asynchronous on `stream`.
 * Errors: INVALID_ARG (NULL pointer, n_t, n_s or nrows < 1, kappa not > 0),
 * OOM, CUDA. */
dfdm_status dfdm_direct_rows(const double *targets, int64_t n_t,
                             const double *sources, int64_t n_s, double kappa,
                             const void *x, const int64_t *rows, int64_t nrows,
                             void *y, void *stream);

/* dfdm_direct_rows for callers that must not allocate device memory.
 *
 * The paper has no counterpart of this call; it exists for users of the
 * library.  Some callers cannot allocate device memory at the moment they
 * need these rows: a process whose device memory is reserved by another
 * framework's caching allocator (a fresh allocation would fail or fragment
 * that pool), or a latency-bound loop that must not let an allocation call
 * synchronise or stall the device.  This variant computes exactly what
 * dfdm_direct_rows computes, with the same arguments and the same kernel,
 * and allocates nothing: its partial sums go to a fixed scratch array that
 * the library places in device memory when it is loaded, 2^18 complex128
 * entries (4 MiB) that every GPU using the library keeps until the process
 * exits.  The caller still provides every input and output buffer.
 *
 * Limit: nrows <= 262144 (2^18); larger requests return DFDM_ERR_INVALID_ARG
 * and touch nothing.  The first call on each device looks up the scratch
 * array's device address (with that device current) and caches it; make that
 * first call before any stream capture on the device.  All calls share the
 * one array, which keeps the last call's partial sums (every entry a call
 * reads it first writes, so nothing needs clearing): two calls whose work
 * overlaps on a GPU (other streams, other threads) race on it and must be
 * ordered by the caller.  Asynchronous on `stream`.  Errors as
 * dfdm_direct_rows, plus CUDA if the address lookup fails. */
dfdm_status dfdm_direct_rows_noalloc(const double *targets, int64_t n_t,
                                     const double *sources, int64_t n_s,
                                     double kappa, const void *x,
                                     const int64_t *rows, int64_t nrows,
                                     void *y, void *stream);

/* Frees the plan and everything it owns; NULL is allowed. */
dfdm_status dfdm_plan_destroy(dfdm_plan plan);

/* Counts of the block partition (Alg. 2) for a uniform tree of depth
 * `depth` whose every box is occupied on both sides -- Sect. 4's tensor grid
 * with n_max = 512 is one -- from the planner's per-level offset tables alone
 * (host only: no points, no GPU): *n_coupling = N_C (admissible blocks of
 * Alg. 2), *n_stored_coupling = N_SC (distinct (level, offset) coupling
 * matrices), *near_leaf_pairs = inadmissible leaf pairs (nearfield blocks).
 * root_side = side of the root cube; l_hf: -2 = the default rule.  Any output
 * pointer may be NULL.  Errors: INVALID_ARG. */
dfdm_status dfdm_uniform_counts(double kappa, double eta2, double root_side,
                                int depth, int l_hf, int64_t *n_coupling,
                                int64_t *n_stored_coupling,
                                int64_t *near_leaf_pairs);

/* Partially pivoted adaptive cross approximation of one coupling matrix,
 * A ~ U V^* (Sect. 2.7, closing remark; host only, a set-up step).  a: host,
 * m x n complex128, row-major.  Step k takes the residual of one row, its
 * largest entry as pivot column, and the residual of that column; the
 * approximation stops once |u_k| |v_k| <= tol ||S_k||_F (S_k the current
 * approximation, the k-th term kept; tol >= 0, 0 runs to max_rank) or at
 * max_rank columns.  u: host m x max_rank complex128, v: host n x max_rank
 * complex128, both row-major, column l holding u_l and v_l (a ~ u v^*);
 * columns from *rank on are zero.  u and v may be NULL when max_rank is 0.
 * Errors: INVALID_ARG, OOM. */
dfdm_status dfdm_aca(const void *a, int m, int n, double tol, int max_rank,
                     void *u, void *v, int *rank);

/* The coupling structure of one level of such a uniform tree, in the format
 * of dfdm_plan_export_offsets (offsets d = t - s and direction indices for
 * targets of parity alpha_index), from the planner alone (host only).
 * Errors: INVALID_ARG (arguments as dfdm_uniform_counts, level outside
 * 0..depth, alpha_index outside 0..7, *count too small). */
dfdm_status dfdm_uniform_offsets(double kappa, double eta2, double root_side,
                                 int depth, int l_hf, int level,
                                 int alpha_index, int32_t *count,
                                 int32_t *offsets, int32_t *dirs);

/* ---------------------------------------------------------------- batches
 * Many independent products, each of Sect. 2 for its own P_T, P_S and kappa
 * (the paper treats one problem at a time; the batched form is this
 * library's).  One plan per problem; dfdm_batch_apply issues every plan's
 * apply on a set of worker streams, the problems placed largest first on the
 * least-loaded stream (estimated flops: 8 n^2 N_C + 20 nearfield entries),
 * and captures all of it once into a CUDA graph; later applies with the same
 * vector pointers and nrhs replay that graph with one launch. */
typedef struct {
  const double *targets; /* HOST, n_t x 3 doubles (copied at create)          */
  int64_t n_t;
  const double *sources; /* HOST, n_s x 3 doubles (copied at create)          */
  int64_t n_s;
  double kappa;          /* > 0                                               */
  int max_depth;         /* tree depth of this problem; -1 = params->max_depth */
} dfdm_problem;

typedef struct dfdm_batch_s *dfdm_batch;

/* Creates one plan per problem with *params (max_depth per problem as
 * above; params->n_max must be 0: uniform trees).  nstreams worker streams
 * (0 = 4, at most 64, never more than nprob).  Plans are built one after the
 * other on `stream`; returns after all are built.  Errors as
 * dfdm_plan_create (the message names the problem), INVALID_ARG for
 * nprob < 1 or a bad nstreams, CUDA if a stream or event cannot be made. */
dfdm_status dfdm_batch_create(int nprob, const dfdm_problem *probs,
                              const dfdm_params *params, int nstreams,
                              void *stream, dfdm_batch *out);

/* Applies every problem: y[i] = A_i x[i] for nrhs right-hand sides, x[i]
 * and y[i] DEVICE pointers laid out as in dfdm_apply.  The graph's launch is
 * ordered on `stream` (work inside it runs on the batch's own streams, after
 * everything issued earlier on `stream`, and `stream` waits for all of it).
 * The first call, or a call whose pointers or nrhs differ from the captured
 * ones, captures a new graph: that call must not itself be inside a stream
 * capture.  Errors: INVALID_ARG, CUDA; device-side errors through
 * dfdm_batch_check. */
dfdm_status dfdm_batch_apply(dfdm_batch b, void *const *x, void *const *y,
                             int nrhs, void *stream);

/* dfdm_plan_check on every plan; returns the first error found. */
dfdm_status dfdm_batch_check(dfdm_batch b, void *stream);

/* Borrows problem i's plan (stats, exports, timing); owned by the batch. */
dfdm_status dfdm_batch_plan(dfdm_batch b, int i, dfdm_plan *out);

/* Worker stream count, the stream of every problem (nprob ints, may be
 * NULL) and the kernel launches the captured graph holds (may be NULL). */
dfdm_status dfdm_batch_info(dfdm_batch b, int *nstreams, int *stream_of,
                            int64_t *launches);

/* Frees the batch, its graph, streams and plans; NULL is allowed. */
dfdm_status dfdm_batch_destroy(dfdm_batch b);

/* ------------------------------------------------------- parameter selector
 * A small perceptron that picks a plan's Chebyshev order and high-frequency
 * level for a requested accuracy.  The paper fixes one order for all levels
 * (m = 4 in Sect. 4) and l_hf by its rule (Eq. 11); the selector is the
 * library's own addition, trained on errors the method itself measures
 * against direct sums.  Network: 4 -> 64 -> 64 -> 64 -> 2, tanh on the
 * hidden layers, linear output; every parameter enters the products rounded
 * to FP16, sums in FP32.  Parameters are a flat float vector of
 * dfdm_selector_param_count() = 8770 entries: W1 (64 x 4, row-major), b1 (64),
 * W2 (64 x 64), b2, W3 (64 x 64), b3, W4 (2 x 64), b4 (2).  Features of one
 * level l (4 floats): l / 10, log2(kappa sqrt(3) w_l) / 8,
 * log2(1 + n / 8^l) / 16, -log10(tol) / 10, with w_l = root_side / 2^l and n
 * points.  Outputs (2 floats): (order - 2) / 8 and a direction flag (> 0.5:
 * the level is treated as high-frequency).  Unless stated, pointers are HOST
 * pointers; the calls run their kernels on `stream` (device scratch is
 * allocated and freed in stream order) and return after the results are on
 * the host.  Errors: INVALID_ARG, OOM, CUDA. */
int dfdm_selector_param_count(void);

/* The 4 features of level `level` (out: 4 floats). */
dfdm_status dfdm_selector_features(double kappa, double root_side, int level,
                                   int64_t n_points, double tol, float *out);

/* y (n x 2) = network(theta; x (n x 4)). */
dfdm_status dfdm_selector_forward(const float *theta, const float *x,
                                  int64_t n, float *y, void *stream);

/* Loss L = (1/n) sum_i 1/2 |network(x_i) - t_i|^2 (t: n x 2) and its
 * gradient w.r.t. theta (grad: 8770 floats; the FP16 rounding of the
 * weights is passed straight through). */
dfdm_status dfdm_selector_grad(const float *theta, const float *x,
                               const float *t, int64_t n, float *grad,
                               float *loss, void *stream);

/* Full-batch Adam (beta1 0.9, beta2 0.999, eps 1e-8, step size lr) for
 * `epochs` steps from theta0; theta_out receives the trained parameters and
 * losses (epochs floats, may be NULL) the loss before each step.  All
 * computed by the library's GPU kernels; deterministic. */
dfdm_status dfdm_selector_train(const float *theta0, const float *x,
                                const float *t, int64_t n, int epochs,
                                float lr, float *theta_out, float *losses,
                                void *stream);

/* Fills p->order and p->l_hf for a product with wave number kappa over
 * n_points points at relative accuracy tol: the network is evaluated on the
 * features of levels min(2, D) .. D (D = p->max_depth, root side
 * p->root_side); order = the mean predicted order over those levels,
 * rounded (a plan has one order; clamped to 2..10), l_hf = the deepest level
 * flagged high-frequency (-1 if none).
 * Errors: INVALID_ARG, NUMERIC (a non-finite network output), OOM, CUDA. */
dfdm_status dfdm_select_params(const float *theta, double kappa, double tol,
                               int64_t n_points, dfdm_params *p, void *stream);

/* Description of the last error on this thread (never NULL). */
const char *dfdm_last_error(void);

/* Library version string (never NULL). */
const char *dfdm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DFDM_H */
