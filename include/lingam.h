/*
 * lingam.h -- C ABI of the GB300 (sm_103a) DirectLiNGAM / VarLiNGAM library.
 *
 * The library computes the causal-ordering step of DirectLiNGAM as described
 * in AcceleratedLiNGAM (arXiv 2403.03772): Algorithm 1 ("search_causal_order")
 * repeated inside the DirectLiNGAM loop of Sec. 2.2, the least-squares
 * adjacency of Sec. 1, and VarLiNGAM (Sec. 3.2).  All arithmetic runs in the
 * library's own CUDA kernels; there is no CPU fallback.
 *
 * Conventions for every call
 *   - Data X is [n samples][d variables] (the paper's "dataset [m, dim]"):
 *     LINGAM_ROW_MAJOR: element (s, i) at X[s*ld + i], ld >= d;
 *     LINGAM_COL_MAJOR: element (s, i) at X[i*ld + s], ld >= n.
 *     X may be a device pointer or a host pointer (pinned or pageable); the
 *     library detects which and copies host data to its own device workspace.
 *   - The caller owns every input and output buffer.  The context owns its
 *     device workspace and its captured CUDA graphs.
 *   - Work is ordered on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Calls that return host outputs synchronise before returning.
 *   - One context per host thread; a context is not thread-safe.
 *   - No call throws or aborts.  Errors come back as lingam_status; the text
 *     of the last error is available from lingam_last_error().
 *   - Status meanings: ARG = invalid size/pointer/layout; NONFINITE = NaN or
 *     Inf in the input; DEGENERATE = a variance reached zero relative to the
 *     variable's original variance (<= 1e-12 relative), or two residualised
 *     variables became perfectly correlated (1 - rho^2 <= 1e-12), or d > n;
 *     CUDA = a CUDA runtime error; OOM = device allocation failed; TIMEOUT =
 *     a bounded device-side wait expired (the kernel gave up and returned).
 */
#ifndef LINGAM_GB300_H
#define LINGAM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lingam_stream_t; /* same type as cudaStream_t */
typedef struct lingam_ctx lingam_ctx;         /* opaque */

typedef enum {
    LINGAM_OK = 0,
    LINGAM_ERR_ARG = 1,
    LINGAM_ERR_NONFINITE = 2,
    LINGAM_ERR_DEGENERATE = 3,
    LINGAM_ERR_CUDA = 4,
    LINGAM_ERR_OOM = 5,
    LINGAM_ERR_TIMEOUT = 6
} lingam_status;

/* Arithmetic of the ordering step.
 *   FP32  -- entropy moments in FP32 with the accurate CUDA expf/log1pf, FP64
 *            covariance (Gram), FP64 residual data, rank-1 downdate and OLS.
 *   MIXED -- covariance on the tensor cores (single-instance calls; exact
 *            7-bit BF16 digit planes scaled per 64 samples, FP64
 *            recombination, about 4e-11 relative error), entropy moments
 *            with the hardware ex2/lg2
 *            approximations and compensated summation; FP64 downdate and OLS.
 *   FP64  -- every moment in FP64 (small problems; GB300 FP64 is slow).
 *   DF    -- every moment in double-float (pairs of FP32 numbers, about
 *            2^-46 relative error per term) on the FP32 pipe, near-ties
 *            re-scored in FP64: near-FP64 results at a fraction of its cost.
 * In the FP32 and MIXED forms a step whose top scores lie within the FP32
 * error bound of each other re-scores its candidates in double-float, and
 * the candidates still within that bound of each other in FP64, before the
 * argmax is taken; steps with at most 32 remaining variables are scored in
 * double-float throughout. */
typedef enum {
    LINGAM_PREC_FP32 = 0,
    LINGAM_PREC_MIXED = 1,
    LINGAM_PREC_FP64 = 2,
    LINGAM_PREC_DF = 3
} lingam_precision;

typedef enum { LINGAM_ROW_MAJOR = 0, LINGAM_COL_MAJOR = 1 } lingam_layout;

typedef struct {
    int32_t precision;     /* lingam_precision */
    int32_t profile;       /* 1: time every launch of the pair-moment kernel
                              with CUDA events (read back by lingam_get_stats) */
    double tie_scale;      /* multiplies the FP32 and double-float error
                              bounds that select the candidates re-scored in
                              the next tier; 0 means 1.0 */
    int32_t conditional_rescore; /* 1: a single-instance graph puts each step's
                              re-score launches under a conditional node
                              that a kernel after the step's select sets, so steps
                              decided by their FP32 scores skip them (fewer
                              launches; Nsight Compute cannot profile the
                              kernel nodes of such a graph); 0 (default):
                              plain graph */
    int32_t reserved[7];
} lingam_opts;

/* Create a context on CUDA device `device`.  opts may be NULL (FP32, no
 * profiling).  *ctx receives the handle (NULL on failure). */
lingam_status lingam_create(lingam_ctx **ctx, int device, const lingam_opts *opts);

/* Release the context, its workspace and its graphs.  NULL is allowed. */
lingam_status lingam_destroy(lingam_ctx *ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next
 * call on the same context.  ctx == NULL gives the last creation error. */
const char *lingam_last_error(const lingam_ctx *ctx);

/* Change the precision of later calls (lingam_precision). */
lingam_status lingam_set_precision(lingam_ctx *ctx, int32_t precision);

/*
 * DirectLiNGAM causal order (Algorithm 1 inside the loop of Sec. 2.2).
 *   X          FP32 data (FP64 when the context precision is FP64), n x d
 *              in `layout` with leading dimension `ld`; read only.
 *   order_out  host int32[d]: original variable indices, most exogenous
 *              first (the paper's causal order K).
 *   scores_out optional host double[d*d]: row t holds the step-t scores
 *              M(i) = -sum_j min(0, I(i,j))^2 (Algorithm 1's k_list) at the
 *              original indices, NaN for variables already ordered; row d-1
 *              holds 0 for the last variable.
 * Requires 1 <= d <= n, n >= 2.  d == 1 returns [0].
 */
lingam_status lingam_causal_order(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                  int64_t ld, int32_t layout, int32_t *order_out,
                                  double *scores_out, lingam_stream_t stream);

/*
 * Weighted adjacency by least squares on the causal order (Sec. 1): row k of
 * B holds the OLS coefficients of x_k regressed on every variable that
 * precedes k in `order` (data centred, so the intercept drops out); all other
 * entries are 0.  B[i*d + j] = effect of x_j on x_i.
 *   order      host int32[d], a permutation of 0..d-1.
 *   B_out      double[d*d], host memory, or device memory if B_on_device.
 * Computed as B = I - L^{-1} where the order-permuted covariance is L D L^T,
 * all in FP64.
 */
lingam_status lingam_fit_adjacency(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                   int64_t ld, int32_t layout, const int32_t *order,
                                   double *B_out, int32_t B_on_device, lingam_stream_t stream);

/*
 * VarLiNGAM (Sec. 3.2): least-squares VAR(lags) with intercept on the time
 * series Xt ([T][d] in `layout`), DirectLiNGAM on the n = T - lags residual
 * innovations, B0 by least squares on that order, and B_tau = (I - B0) M_tau.
 *   order_out  host int32[d]; B0_out host double[d*d]; Btau_out host
 *              double[lags*d*d] (tau = 1..lags, each d x d, B[i*d+j] =
 *              effect of x_j(t - tau) on x_i(t)).  B0_out/Btau_out may be NULL.
 * Xt is FP32.  Requires lags >= 1 and T - lags > lags*d + d.
 */
lingam_status varlingam_fit(lingam_ctx *ctx, const void *Xt, int64_t T, int64_t d, int64_t ld,
                            int32_t layout, int32_t lags, int32_t *order_out, double *B0_out,
                            double *Btau_out, lingam_stream_t stream);

/*
 * Many independent DirectLiNGAM problems in one call (bootstrap resamples
 * and problems of uneven size).  Instance k orders the FP32 data X (row-major
 * [n_src][ld], ld >= d) restricted to the rows rows[0..n) when rows != NULL
 * (sampling with replacement is allowed; rows is a host int32 array), or to
 * its first n rows when rows == NULL (then n <= n_src).
 *   orders_out[k]  host int32[d_k]
 *   B_out[k]       optional host double[d_k*d_k] adjacency of instance k
 *                  (B_out itself may be NULL).
 * All instances advance through their ordering steps together in one CUDA
 * graph.  Returns the first failing instance's status; *failed_index (may be
 * NULL) receives its index or -1.
 */
typedef struct {
    const void *X;        /* FP32 row-major data, device or host */
    int64_t n_src;        /* rows available in X */
    int64_t n;            /* rows used (length of rows[] when rows != NULL) */
    int64_t d;
    int64_t ld;
    const int32_t *rows;  /* optional host int32[n] row indices into X */
} lingam_instance;

lingam_status lingam_causal_order_batch(lingam_ctx *ctx, const lingam_instance *inst,
                                        int32_t count, int32_t *const *orders_out,
                                        double *const *B_out, int32_t *failed_index,
                                        lingam_stream_t stream);

/*
 * Scores of the first ordering step only, for parity checks: I_out optional
 * host double[d*d] with I(i, j) of Algorithm 1 at original indices (diagonal
 * 0); M_out optional host double[d] with M(i); eps_out optional host
 * double[d*d] with the bound on |I_out - I_exact| that the library uses to
 * pick the candidates it re-scores (from its moment-error model in the FP32
 * and MIXED forms, a fixed 1e-12 in DF, 0 in FP64).  Same data rules as
 * lingam_causal_order.
 */
lingam_status lingam_step_measures(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                   int64_t ld, int32_t layout, double *I_out, double *M_out,
                                   double *eps_out, lingam_stream_t stream);

/*
 * Sparse weighted adjacency on a causal order.  The paper only says the
 * adjacency comes from "regressing" each variable on the ones before it
 * (Sec. 1); this is the pruned reading: for every variable k with
 * predecessors P, the adaptive lasso of Zou (2006) in covariance form,
 *     min_b 1/2 b'C_PP b - b'C_Pk + lam sum_j w_j |b_j|,  w_j = |b_ols_j|^-gamma,
 * on the centred FP64 covariance C = Xc'Xc/n, at lam_i = lam_max
 * eps^(i/(n_lambda-1)), i = 0..n_lambda-1 (lam_max = (1 + 1e-9) max_j
 * |C_jk| / w_j).  Each point is the exact minimiser, the path being followed
 * by homotopy (the lasso form of LARS: joins and drops of the active set,
 * the active Gram's inverse updated in place); the lam with the smallest
 * BIC = n log(RSS/n) + df log n (first minimum) gives row k.  Variables with
 * b_ols_j = 0 keep b_j = 0.  LINGAM_ERR_DEGENERATE if the active Gram stops
 * being positive definite or a row's path does not end within 20 q + 100
 * events (q predecessors).
 *   X, n, d, ld, layout, order: as lingam_fit_adjacency.
 *   gamma > 0 (1 is usual), 2 <= n_lambda <= 1000, 0 < eps < 1 (60, 1e-6
 *   are the library's test settings).
 *   B_out: double[d*d], host memory, or device memory if B_on_device.
 */
lingam_status lingam_prune_adjacency(lingam_ctx *ctx, const void *X, int64_t n, int64_t d,
                                     int64_t ld, int32_t layout, const int32_t *order,
                                     double gamma, int32_t n_lambda, double eps, double *B_out,
                                     int32_t B_on_device, lingam_stream_t stream);

/*
 * Total causal effects (Sec. 4.2 ranks nodes "by measuring the total causal
 * effects"): for the linear acyclic model x = B x + e, T = (I - B)^-1, so
 * T[i*d + j] is the effect on x_i of a unit change in e_j: the sum over every
 * directed path j -> i of the product of the edge weights (T[i][i] = 1).
 *   B      double[d*d] (host or device), B[i*d + j] = edge j -> i, zero unless
 *          j precedes i in `order` (else LINGAM_ERR_ARG).
 *   order  host int32[d], a permutation of 0..d-1 (a causal order of B).
 *   T_out  double[d*d], host memory, or device memory if T_on_device.
 * FP64: forward substitution of the unit lower triangular I - B in the order.
 */
lingam_status lingam_total_effects(lingam_ctx *ctx, const double *B, int64_t d,
                                   const int32_t *order, double *T_out, int32_t T_on_device,
                                   lingam_stream_t stream);

/*
 * Total effects in the time-unrolled VarLiNGAM graph (Sec. 3.2, 4.2) over the
 * q = (lags+1) d nodes [x(t-lags), ..., x(t-1), x(t)] (node s*d + i is
 * variable i in slice s, oldest slice first): B0 acts within every slice,
 * B_tau from slice s - tau to slice s.  B0 (double[d*d]) and Btau
 * (double[lags*d*d], as varlingam_fit writes them) may be host or device
 * memory; order is B0's causal order (host int32[d]).  T_out: double[q*q].
 */
lingam_status varlingam_total_effects(lingam_ctx *ctx, const double *B0, const double *Btau,
                                      int64_t d, int32_t lags, const int32_t *order,
                                      double *T_out, int32_t T_on_device,
                                      lingam_stream_t stream);

/*
 * Influence of every node from total effects T (double[q*q], host or device;
 * Sec. 4.2 Table 2): exert_out[j] = sum_{i != j} |T[i][j]|, receive_out[i] =
 * sum_{j != i} |T[i][j]| (host double[q] each, optional); the rank outputs
 * (host int32[q], optional) list the nodes by descending score, equal scores
 * to the smaller index, so their first k entries are the top-k nodes.
 */
lingam_status lingam_influence(lingam_ctx *ctx, const double *T, int64_t q, double *exert_out,
                               double *receive_out, int32_t *exert_rank_out,
                               int32_t *receive_rank_out, lingam_stream_t stream);

/*
 * Edge statistics over bootstrap resamples (the adjacency matrices of a
 * batch, host or device double[d*d] each): prob_out[i*d + j] = fraction of the
 * count matrices with |B[i][j]| > threshold, mean_out[i*d + j] = their mean
 * (host double[d*d] each).  threshold >= 0.
 */
lingam_status lingam_bootstrap_edge_stats(lingam_ctx *ctx, const double *const *B, int32_t count,
                                          int64_t d, double threshold, double *prob_out,
                                          double *mean_out, lingam_stream_t stream);

/*
 * Tile shapes and split schedules of the FP32 pair-moment kernel, by range of
 * the number p of remaining variables.  Bucket b covers
 * p_max[b-1] < p <= p_max[b] (p_max ascending; the last bucket also covers
 * every larger p).  tile[b] indexes the kernel's tile configurations
 * (0 .. LINGAM_PAIR_TILES-1, described by lingam_pair_tile_info); ctas_per_sm[b] is
 * the number of CTAs per SM the sample splits aim for; ms[b] the kernel time
 * measured at the probe size p_probe[b] with n_probe samples.  One table per
 * form that runs the FP32 kernel (precision FP32 or MIXED).
 */
typedef struct {
    int32_t count;            /* buckets in use, 1..8 */
    int32_t precision;        /* LINGAM_PREC_FP32 or LINGAM_PREC_MIXED */
    int32_t p_max[8];
    int32_t tile[8];
    int32_t ctas_per_sm[8];
    int32_t p_probe[8];
    double ms[8];
    int64_t n_probe;
} lingam_tuning;

/*
 * Autotuner: times every tile configuration with three split schedules on
 * synthetic standardised data of n samples (capped at 131072) at probe sizes
 * p = 64, 128, ..., up to min(d, 2048), each probe launched as `instances`
 * copies in one batch (1 for single problems; the batch size for
 * lingam_causal_order_batch, within 2 GB of scratch), and keeps the fastest
 * per bucket for the context's current precision form (FP32 or MIXED; other
 * forms return LINGAM_ERR_ARG).  Later calls of that form use the table.
 * *out (optional) receives it.  Allocates and frees its own scratch;
 * invalidates the cached step graph.
 */
lingam_status lingam_autotune(lingam_ctx *ctx, int64_t n, int64_t d, int32_t instances,
                              lingam_tuning *out);

/* Install a table (for example one saved from an earlier lingam_autotune on
 * the same GPU model) for the form t->precision; checks its entries. */
lingam_status lingam_set_tuning(lingam_ctx *ctx, const lingam_tuning *t);

/* Current table of form `precision` (the untuned default is one bucket,
 * tile 0, 4 CTAs per SM). */
lingam_status lingam_get_tuning(const lingam_ctx *ctx, int32_t precision, lingam_tuning *out);

/*
 * Prior knowledge of ancestry for the following ordering calls on ctx
 * (lingam_causal_order, lingam_causal_order_batch, varlingam_fit on the
 * innovations).  prior: host int8 [d][d] row-major, copied; prior[i*d + j] =
 * 1 if x_j is known to be an ancestor of x_i (a directed path j -> i), 0 if
 * known not to be, -1 if unknown; the diagonal is ignored.  NULL or d = 0
 * clears it.  The paper has no prior knowledge; the rule follows the
 * DirectLiNGAM literature's use of such a matrix: at each step a variable may
 * be chosen only if no remaining variable is a known ancestor of it, and
 * only among the known-exogenous remaining variables (every other remaining
 * one known not to be an ancestor) when there are any; the scores M(i) are
 * unchanged.  Every input of a later ordering call must have this d
 * (LINGAM_ERR_ARG otherwise), and knowledge that leaves no variable to choose
 * makes that call return LINGAM_ERR_ARG.  LINGAM_ERR_ARG here for entries
 * outside {-1, 0, 1} or d outside 1..6000.
 */
lingam_status lingam_set_prior_knowledge(lingam_ctx *ctx, const int8_t *prior, int64_t d);

/*
 * Pair sharding of one ordering over several ranks (one process and GPU per
 * rank).  Algorithm 1's work per step is the p (p - 1) ordered pairs, which
 * are independent (Sec. 3.1 parallelises over them); only the p-vector of
 * scores M(i) joins them.  With a shard set, a context computes the pair
 * moments and the score terms only for the pairs its rank owns
 * (lingam_shard_owner), so its M(i) and error bounds E(i) are partial sums;
 * after each step's scoring the library calls
 *
 *     int allreduce(double *buf, int64_t count, void *user)
 *
 * with buf = [partial M (p values) | partial E (p values)], count = 2 p, on
 * the host.  It must replace buf with the element-wise sums over all ranks,
 * identical bit for bit on every rank (for example gather the partials and
 * add them in rank order), and return 0; a non-zero return fails the call
 * with LINGAM_ERR_CUDA.  Every rank then takes the same decisions: the
 * argmax, the re-score tiers (candidate rows recomputed in full on every
 * rank) and the regress-out are replicated, so all ranks return the same
 * order.  One exchange of 2 p doubles per step.
 *
 *   rank, nranks  0 <= rank < nranks; nranks = 1 removes the shard.
 *   allreduce     required when nranks > 1; user is passed through.
 * Applies to lingam_causal_order (without a score history) and
 * lingam_step_measures (which returns the rank's partial first-step M, no
 * exchange, and I(i, j) only for owned entries).  A sharded context refuses
 * batched calls and score histories with LINGAM_ERR_ARG.
 */
typedef int (*lingam_allreduce_fn)(double *buf, int64_t count, void *user);
lingam_status lingam_set_shard(lingam_ctx *ctx, int32_t rank, int32_t nranks,
                               lingam_allreduce_fn allreduce, void *user);

/* Owner rank of the ordered pairs (i, j) and (j, i) of positions i, j < p at a
 * step with p remaining variables over nranks ranks: the positions are cut
 * into blocks of 16 and the unordered block pairs, taken row by row over the
 * upper triangle, into nranks contiguous ranges of about p (p - 1) / nranks
 * ordered pairs each.  No context or GPU needed; -1 for arguments out of
 * range (p = 1 has no pairs: rank 0). */
int32_t lingam_shard_owner(int64_t i, int64_t j, int64_t p, int32_t nranks);

/*
 * Input gate for the single-instance calls (lingam_causal_order,
 * lingam_step_measures).  (The paper has no counterpart: a runtime facility.)
 * With a gate set, each such call first waits on the device until *flag is
 * non-zero, and only then reads X, so a producer that cannot share a stream
 * with the caller (another process, a copy engine driven elsewhere, the host
 * writing mapped memory) can release the input by setting the flag after
 * its data are written (with release ordering at system scope, e.g. a
 * __threadfence_system() before the store, or a stream-ordered copy).
 *
 *   flag       4-byte aligned uint32 in device, managed or mapped (pinned,
 *              cudaHostAllocMapped / registered-mapped) host memory, owned by
 *              the caller and valid while the gate is set; NULL removes the
 *              gate.  The library only reads it.
 *   timeout_s  bound on each wait, 0 < timeout_s <= 60.
 * When a wait runs out, the call returns LINGAM_ERR_TIMEOUT (its outputs are
 * not valid) and the context stays usable: the next call waits again.  A
 * flag that is not device-readable memory, a misaligned flag or a timeout
 * outside the range is LINGAM_ERR_ARG.
 */
lingam_status lingam_set_input_gate(lingam_ctx *ctx, const uint32_t *flag, double timeout_s);

/* Number of pair-kernel tile configurations. */
#define LINGAM_PAIR_TILES 33

/*
 * Shape of tile configuration `tile` (no context or GPU needed): out[9] =
 * {pairs per warp along i, along j, warps along i, along j, TMA ring stages,
 * groups of 4 samples per lane and iteration (one MUFU lg2 per 4 x groups
 * samples in the fast form), chunks of 256 samples between compensated
 * folds, paired-FP32 (f32x2) arithmetic 0/1, chunks per TMA ring stage of the
 * streamlined block (0: the original one-chunk-per-stage block)}.  LINGAM_ERR_ARG for a tile
 * outside 0 .. LINGAM_PAIR_TILES-1 or a null out.
 */
lingam_status lingam_pair_tile_info(int32_t tile, int32_t *out);

/* Counters of the last lingam_causal_order / batch call on ctx. */
typedef struct {
    double total_ms;          /* device time of the whole call (events) */
    double pair_ms;           /* summed pair-moment kernel time (profile=1) */
    int64_t pair_launches;    /* pair-moment kernel launches timed */
    double pair_units;        /* residual-samples those launches processed */
    int32_t refined_steps;    /* steps whose first scores left candidates */
    int32_t genuine_ties;     /* steps whose FP64 top-2 gap <= 1e-9 max|M| */
    int32_t candidates_max;   /* largest candidate set re-scored */
    int32_t graph_nodes;      /* kernel nodes in the step graph */
    double graph_build_ms;    /* capture + instantiate time (0 if cached) */
    int32_t fp64_candidates;  /* candidates re-scored in FP64 over the run */
    int32_t df_candidates;    /* candidates re-scored in double-float */
    int32_t cond_nodes;       /* kernel nodes of graph_nodes inside conditional
                                 re-score blocks (run only at steps that leave
                                 candidates after their first scores) */
    int32_t cond_bodies;      /* those blocks (one per step of a single-instance
                                 graph; 0 for batches and sharded calls) */
    int32_t reserved[2];
    double score_ms;          /* summed score + select time (profile=1) */
    double refine_ms;         /* summed re-score passes (profile=1) */
    double regress_ms;        /* summed regress-out + downdate (profile=1) */
} lingam_stats;

lingam_status lingam_get_stats(const lingam_ctx *ctx, lingam_stats *out);

/*
 * Throughput probes of the units the entropy kernel is bound by, measured on
 * the context's device: which = 0 FP32 FMA (flop/s, 2 per FMA), 1 MUFU ex2
 * (op/s), 2 MUFU lg2 (op/s), 3 FP64 FMA (flop/s).  *ops_per_s receives the
 * rate and *sm_clock_mhz the average SM clock seen by the probe (from
 * clock64 over the globaltimer).
 */
lingam_status lingam_peak_probe(lingam_ctx *ctx, int32_t which, double *ops_per_s,
                                double *sm_clock_mhz);

/*
 * First-step scores for callers that must not allocate device memory.
 *
 * (The paper has no counterpart: this is a packaging variant of the FP64
 * pair-moment kernel for constrained callers.)  Every other entry point needs
 * a context, and lingam_create allocates device workspace.  Some callers
 * cannot do that while they run: code invoked from inside a device-memory
 * allocator or pool (cudaMalloc would re-enter it), plugins of applications
 * that reserve nearly all device memory up front, and services that forbid
 * cudaMalloc/cudaFree on their serving path because those calls can
 * synchronise the device.  This call needs no context and allocates nothing:
 * its scratch is a fixed ~66 KB array built into the library, present on
 * every GPU that loads the library until the process exits.
 *
 *   X      device pointer, FP64, row-major [n][ld], ld >= d (read only).
 *   M_out  device pointer, double[d]: M(i) = -sum_j min(0, I(i,j))^2 of the
 *          first ordering step, computed in FP64 (what lingam_step_measures
 *          returns in M_out).
 *   stream the call is ordered on it and synchronises it before returning.
 * Limits: 2 <= d <= 64 (the scratch array's size), 2 <= n <= 2^30; anything
 * else returns LINGAM_ERR_ARG without touching the GPU.  NaN/Inf input gives
 * LINGAM_ERR_NONFINITE, a zero variance or |rho| = 1 LINGAM_ERR_DEGENERATE.
 * Each call looks up the array's device address with the caller's device
 * current.  Under CUDA's lazy module loading the first call on a device loads
 * the library's device code there, and that load can allocate device memory
 * (for the code and the array): make one call on each device before entering
 * a region where allocation is forbidden, and before any stream capture.
 * Later calls allocate nothing.  All calls on one GPU share the array (the
 * call clears what must start at zero), so calls that overlap in time on the
 * same GPU race and must be serialised by the caller.  Cost: each unordered
 * pair re-reads its two columns three times from row-major X, one row per
 * lane, so a call makes about 3 d^2 strided passes over n samples; it is
 * meant for small d, not for throughput.
 */
lingam_status lingam_step_scores_noalloc(const double *X, int64_t n, int64_t d, int64_t ld,
                                         double *M_out, lingam_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* LINGAM_GB300_H */
