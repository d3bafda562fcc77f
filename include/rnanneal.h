/*
 * rnanneal.h -- C ABI of the GB300 (sm_103a) library for parallel simulated
 * annealing over the integer parameters of ternary discrete-logic models of
 * regulatory networks (arXiv 2506.19866).
 *
 * The problem (Sections 2.1-2.3): a directed network of N nodes with states
 * s_i in {0,1,2}; each edge j -> i carries weight w in {0,1,2}, polarity
 * p in {-1,0,1} and threshold t in {1,2} (Section 2.1); each node carries
 * speed u ({1..6} slow, {10,11,12} fast), memory m in {0,1,2} and step size
 * d in {1,2} (Section 2.2).  Given initial states, sparse time courses R and
 * the observation mask, find the parameter vector
 *     x = [w(E), p(E), t(E), u(N), m(N), d(N)],  P = 3E + 3N  (Section 2.3)
 * minimising the gradient-weighted Manhattan distance y between the simulated
 * trajectories S(x) and R, subject to the structural constraints of
 * Section 2.5.3, with the parallel annealing loop of Table 1.
 *
 * Conventions shared by every entry point:
 *   - Every function returns RN_OK (0) or a negative RN_E* code; the message
 *     of the last failure on a context is rn_last_error(ctx).  A failing call
 *     leaves the context's previous state usable unless the code is
 *     RN_ECUDA, after which the context should be destroyed.
 *   - Host arrays are read during the call and copied; the library keeps no
 *     pointer to them.  Output host arrays are written before the call returns.
 *   - Arrays are dense, row-major, in the shapes given ([C][T][N] means
 *     index (c * T + t) * N + i).  Edge order is the caller's order and defines
 *     the layout of x.
 *   - The context owns all device memory it allocates.  Work runs on the
 *     stream given to rn_create (NULL: the library creates its own), so a
 *     caller may pass the CUDA stream its framework is using.
 *   - Contexts are not thread-safe; one context per host thread.
 *   - The step generator is Philox4x32-10 (Salmon et al., SC'11) keyed by the
 *     64-bit seed; step g of chain k uses counter (g_lo, g_hi, k, 0): word 0
 *     picks the parameter, word 1 its new value, word 2 decides acceptance.
 *     Results are bit-identical across runs, devices and call splittings.
 */
#ifndef RNANNEAL_H
#define RNANNEAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RN_OK 0
#define RN_EINVAL (-1)        /* bad argument, shape or value */
#define RN_ECONSTRAINT (-2)   /* Section 2.5.3 constraints cannot hold / do not hold */
#define RN_ENOMEM (-3)        /* device or host allocation failed */
#define RN_ECUDA (-4)         /* a CUDA call failed */
#define RN_ETIMEOUT (-5)      /* a device-side wait gave up (error flag set by a kernel) */
#define RN_ESTATE (-6)        /* call made in the wrong order (e.g. anneal before init) */
#define RN_EUNSUPPORTED (-7)  /* shape outside what the compiled kernels cover */

typedef struct rn_ctx rn_ctx;

/* Annealing schedule (Table 1 and Section 2.4.1).  Level l runs at
 * T_l = T0 * alpha^l (repeated multiplication in double precision) for
 * iters_per_level proposals per chain.  reset_to_best: each level starts from
 * the chain's x_best (Table 1, first lines of the while loop).  global_sync:
 * each level ends with the serial argmin of Table 1 -- the lowest delta_best
 * over all chains of a network (lowest chain index on ties) is copied into
 * every chain's x_best.  The paper's runs use T0 = 1000, alpha = 0.99,
 * iters_per_level = 5000, reset_to_best = global_sync = 1; one proposal per
 * level with both flags 0 is a plain geometric anneal.  Acceptance of a
 * candidate with dE = delta_cand - delta_cur > 0 is r < thr(T_l, dE) with
 * thr = min(floor(exp(-dE / T_l) * 2^32), 2^32 - 1) computed on the host. */
typedef struct {
    double T0;
    double alpha;
    int64_t iters_per_level;
    int32_t reset_to_best;
    int32_t global_sync;
    /* Exact early rejection (an addition to Table 1, off when 0): the
     * acceptance word r is drawn before the simulation, so the largest
     * acceptable dE is known up front (the thresholds do not increase with dE);
     * a candidate's simulation stops once its partial score, which never
     * decreases, exceeds delta_cur plus that dE.  Such a candidate would be
     * rejected anyway: chains, scores and counters are bit-identical to the
     * full simulation.  Networks above 512 nodes and the batched launch
     * (see rn_batch_config) simulate in full. */
    int32_t early_reject;
    /* Grouped level synchronisation (the group-wise reduction that Section 4.5
     * proposes in place of one reduction over all threads): with global_sync,
     * chains k*sync_group .. (k+1)*sync_group - 1 form group k (the last group
     * may be shorter), and the level-end argmin and broadcast run within each
     * group.  0 means one group of all the network's chains. */
    int32_t sync_group;
} rn_schedule;

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t the
 * library should use (NULL: create one).  Fails with RN_ECUDA if the device
 * cannot be used or is not an sm_103 part. */
int rn_create(rn_ctx **out, int device, void *stream);

/* Free every device buffer and the context itself.  NULL is accepted. */
int rn_destroy(rn_ctx *ctx);

/* Message of the last failure on ctx ("" if none).  Valid until the next call
 * on ctx.  NULL ctx gives the message of the last rn_create failure. */
const char *rn_last_error(const rn_ctx *ctx);

/* Register a network (Section 2.1 topology, Section 2.2 speed classes).
 *   src, dst   [E] node indices of each edge (0 <= index < N).
 *   fast       [N] 1 = fast node (u in {10,11,12}), 0 = slow (u in {1..6}).
 *   frozen     [P] 1 = parameter j is fixed at frozen_val[j] and never
 *              proposed, or NULL (everything free).
 *   frozen_val [P] values of the fixed parameters (ignored where frozen = 0),
 *              or NULL iff frozen is NULL.
 * Rejected with RN_EINVAL: N < 1, E < 1, N > 65535, P = 3E + 3N above
 * 2^31 - 1, an index out of range,
 * a self-loop, a duplicate edge, a node without an in-edge or an out-edge
 * (the constraints of Section 2.5.3 could never hold), a fixed value outside
 * its domain.  On success *net_id receives the network's handle.
 * Shapes the kernels cover (calls that need the device -- rn_init_chains,
 * rn_evaluate, rn_anneal -- return RN_EUNSUPPORTED otherwise):
 *   N <= 512, in-degree <= 16: a warp per chain (register tables up to 128
 *     nodes, shared-memory tables above);
 *   otherwise N <= 4096, in-degree <= 31: a block of 256 threads per chain
 *     (at least 2 nodes per thread; node state in registers up to 2048
 *     nodes), provided the chain's tables fit one block's shared memory
 *     (227 KiB: 1 KiB per table row, where nodes ranked by in-degree fill
 *     slots of 256 and each slot has as many rows as its largest in-degree
 *     rounded up to 4, plus 4 bytes per node up to 2048 nodes and 52 above;
 *     the chain's x joins them there when it fits; e.g. 2000 nodes at mean
 *     in-degree 6, or about 2900 nodes at in-degree 2). */
int rn_load_network(rn_ctx *ctx, int32_t n_nodes, int32_t n_edges, const int32_t *src,
                    const int32_t *dst, const uint8_t *fast, const uint8_t *frozen,
                    const int8_t *frozen_val, int32_t *net_id);

/* Attach experimental data to a network (Section 2.3).
 *   n_cond     C >= 1 conditions; a condition is an initial state plus an
 *              optional set of knocked-out nodes (held at 0, never updated).
 *   n_times    1 <= T <= 128 time points including t0 (T - 1 update steps).
 *   init       [C][N] initial states, 0..2.
 *   knockout   [C][N] 1 = knocked out in that condition, or NULL.
 *   ref        [C][T][N] reference data R, 0..2 (ignored where unobserved).
 *   observed   [C][T][N] 1 = entry observed.
 * The weight of an entry is observed * (|G| + 1), with G the difference of R
 * to the previous time point of the same condition where both are observed
 * and 0 otherwise (0 in row t0).  Replaces earlier data and invalidates the
 * chains' objective values (call rn_init_chains again).  RN_EINVAL if the
 * largest possible score, sum of 2 W over the entries, reaches 2^30, or if
 * C * T * N exceeds 2^31. */
int rn_load_timecourse(rn_ctx *ctx, int32_t net, int32_t n_cond, int32_t n_times,
                       const uint8_t *init, const uint8_t *knockout, const uint8_t *ref,
                       const uint8_t *observed);

/* Create n_chains >= 1 annealing chains for a network and evaluate them.
 *   seed   Philox key of every draw of these chains.
 *   x0     [n_chains][P] starting vectors (checked: domains, fixed values,
 *          constraints -> RN_EINVAL / RN_ECONSTRAINT), or NULL to draw them on
 *          the device: each free x_j is dom_j[floor(r * |dom_j| / 2^32)] with r
 *          word (j & 3) of Philox(seed; j >> 2, 0, chain, 1); then every node
 *          without an activating in-edge gets one (p = +1, w = 1 + (r1 & 1) on
 *          the floor(r0 * n / 2^32)-th eligible in-edge, r = Philox(seed; i, 0,
 *          chain, 3)), then every node without a nonzero out-edge gets one
 *          (w = 1 + (r1 & 1), r = Philox(seed; i, 1, chain, 3)).  A network
 *          whose fixed parameters make this impossible gives RN_ECONSTRAINT.
 * Sets x_best = x_cur = x0, delta_best = delta_cur = y(x0), global step 0. */
int rn_init_chains(rn_ctx *ctx, int32_t net, int32_t n_chains, uint64_t seed, const int8_t *x0);

/* Precompute the acceptance-threshold tables of a schedule for global steps
 * 0 .. total_steps - 1 and keep them on the device, so that later rn_anneal
 * calls with an identical schedule inside that range do no host work and
 * return without waiting for the device.  Optional: rn_anneal computes the
 * tables it needs when they are not cached.  The cache covers every network
 * loaded so far (their largest possible dE). */
int rn_prepare_schedule(rn_ctx *ctx, const rn_schedule *sched, int64_t total_steps);

/* Advance every chain of every initialised network by `sweeps` proposal
 * steps (global steps g .. g + sweeps - 1, continuing from earlier calls).
 * Per step and chain (Table 1): draw r; GetCandidate picks the
 * floor(r0 * n_free / 2^32)-th free parameter and the floor(r1 * n_alt / 2^32)-th
 * of its alternative values (ascending, != current, keeping both constraints
 * of Section 2.5.3); with no alternative the step is a null move and nothing
 * is simulated; otherwise the candidate is simulated over every condition and
 * scored, and accepted iff dE <= 0 or r2 < thr(T_l, dE).  x_best follows
 * strict improvements.  Asynchronous on the context stream except for the
 * small threshold-table upload.  With several launches in one call (the
 * batched launch and the networks it does not take, see below), cached tables
 * (rn_prepare_schedule) and no global_sync, the networks with launches of their
 * own run on up to four side streams of the context, most work first: they
 * wait for the work already queued on the context stream, run beside one
 * another and beside the batched launch once it is tuned, and the call makes
 * the context stream wait for all of them (events; the host does not block),
 * so later work on the context stream is ordered after the whole call.  Networks without chains are skipped;
 * RN_ESTATE if no network of the context has chains.  RN_EINVAL for sweeps < 0,
 * iters_per_level < 1, sync_group < 0, or T0 or alpha not positive and finite. */
int rn_anneal(rn_ctx *ctx, const rn_schedule *sched, int64_t sweeps);

/* Best vector over a network's chains: lowest delta_best, lowest chain index
 * on ties.  x [P] (may be NULL), *score, *chain (may be NULL).  Synchronises
 * the context stream. */
int rn_get_best(rn_ctx *ctx, int32_t net, int8_t *x, int32_t *score, int32_t *chain);

/* Objective y of n parameter vectors (Simulate() of Table 1), host buffers.
 *   x      [n][P] vectors (domains are checked; constraints are not required).
 *   score  [n] out.
 *   traj   [n][C][T][N] out: simulated trajectories S, or NULL. */
int rn_evaluate(rn_ctx *ctx, int32_t net, int32_t n, const int8_t *x, int32_t *score,
                uint8_t *traj);

/* As rn_evaluate with device pointers (x_dev [n][P], score_dev [n],
 * traj_dev [n][C][T][N] or NULL) and no host synchronisation: the work is
 * queued on the context stream.  Values outside a domain give undefined
 * scores (not checked).  Each buffer must be device (or managed) memory of the
 * context's device holding its full size within one allocation; a host
 * pointer, another device's memory or a short buffer is refused with
 * RN_EINVAL before anything is launched. */
int rn_evaluate_device(rn_ctx *ctx, int32_t net, int32_t n, const int8_t *x_dev,
                       int32_t *score_dev, uint8_t *traj_dev);

/* Number of parameters P = 3E + 3N of a network. */
int rn_n_params(rn_ctx *ctx, int32_t net, int32_t *n_params);

/* Update scheme of a network (Section 2.2 names three): 0 = priority updating
 * (the paper's, the default): only the eligible nodes of maximum priority
 * u * (tau - last) move at a step; 1 = synchronous updating: every eligible
 * node moves at every step; 2 = asynchronous updating: at step tau of condition
 * c only node selected[c][tau] (-1: none) may move, if eligible (the others
 * keep counting toward their memory m); eligibility, m and d as before.
 *   selected  [C][T] node drawn by the caller for each step (entry tau = 0 is
 *             unused), for scheme 2 only (else ignored); needs the time course
 *             loaded first (RN_ESTATE).
 * Under schemes 1 and 2 the speeds u have no effect, so GetCandidate no longer
 * proposes them (they keep their values).  A new rn_load_timecourse drops
 * scheme 2 (back to 0).  The network's chains must be initialised again
 * (RN_ESTATE until rn_init_chains).  RN_EINVAL for another scheme or a node
 * outside -1 .. N-1. */
int rn_set_update_scheme(rn_ctx *ctx, int32_t net, int32_t scheme, const int32_t *selected);

/* Checkpoint / parity access to the chain state of a network (host buffers,
 * each may be NULL): x_cur, x_best [n][P]; d_cur, d_best [n];
 * counters [n][3] = accepted moves, accepted uphill moves (dE > 0), null
 * moves; *step = next global step.  rn_set_chain_state restores all of them
 * (every pointer required, vectors checked as in rn_init_chains), so that a
 * resumed run continues bit-identically. */
int rn_get_chain_state(rn_ctx *ctx, int32_t net, int8_t *x_cur, int32_t *d_cur, int8_t *x_best,
                       int32_t *d_best, int64_t *counters, int64_t *step);
int rn_set_chain_state(rn_ctx *ctx, int32_t net, int32_t n_chains, uint64_t seed,
                       const int8_t *x_cur, const int32_t *d_cur, const int8_t *x_best,
                       const int32_t *d_best, const int64_t *counters, int64_t step);

/* Annealing statistics of a network, for acceptance-rate profiles such as
 * the paper's (Section 3):
 *   stats[0] accepted moves, stats[1] accepted uphill moves (dE > 0),
 *   stats[2] null moves, each summed over the network's chains since
 *   rn_init_chains (or as restored by rn_set_chain_state);
 *   stats[3] chains; stats[4] the next global step.
 * A level's counts are the difference of two calls around the rn_anneal that
 * runs it; its acceptance rate is accepted / (chains * steps - null).
 * Synchronises the context stream.  RN_EINVAL for a NULL stats, RN_ESTATE if
 * the network has no chains. */
int rn_get_stats(rn_ctx *ctx, int32_t net, int64_t stats[5]);

/* Self-test of the failure path of the device-side waits (an addition of this
 * library; the paper has none).  The annealing kernels' work queue waits, with
 * an iteration limit, for the previous chunk of a chain; a wait that gives up
 * sets the context's device flag and its kernel returns, and the next call
 * that checks the flag fails with RN_ETIMEOUT.  This call runs that same wait
 * in one warp, with a short limit (4096 polls), on a counter that nothing
 * advances, and returns what the flag check reports: RN_ETIMEOUT, with
 * rn_last_error naming the wait, when the path works.  The flag is cleared, so
 * the context stays usable.  RN_ECUDA if the wait did not give up and report
 * it; an earlier failure on the context stream is reported first. */
int rn_selftest_wait(rn_ctx *ctx);

/* Number of kernels this context has launched since rn_create. */
int rn_launch_count(rn_ctx *ctx, int64_t *count);

/* Batched annealing.  When two or more networks of a context have chains, a
 * warp per chain and at least two conditions (and the schedule has no
 * global_sync), rn_anneal advances all of them in one persistent launch over
 * every chain; the other networks with chains (one condition, or above 512
 * nodes) get their own launches in the same call.  Results are bit-identical
 * to annealing each network alone.  The first batched call tunes the launch on the real
 * batch (table path per network and warps per block), timing each candidate
 * for a few steps from the current state, which is restored afterwards.
 * Candidate c = 3 * w + p (c < 6): table paths p = 0 register tables where
 * they fit, shared-memory tables elsewhere; p = 1 the same with the hybrid
 * path (table words in shared memory, node state in registers) for networks of
 * 129-256 nodes; p = 2 shared-memory tables for all; warps per block 4 (w = 0)
 * or 2 (w = 1); the warps with a region large enough for any network are the
 * work share of those networks.  c = 6, 7: p = 0 with 4 / 2 warps per block,
 * every warp with a large region.  c = 8, 9: phased launches, one kernel per
 * table path in sequence (the paths of p = 0, and of p = 1 with the hybrid
 * path also for networks of 257-320 nodes), so that an SM never
 * runs two paths' code at once; each phase's warp region fits its own path's
 * largest network, and each phase takes the warps per block (4 or 2) its trial
 * ran faster with (a phased candidate's trial time is the sum of its phases').
 * With the threshold tables cached by rn_prepare_schedule, the launch (all
 * phases) is captured once in a CUDA graph and replayed.  This reports the
 * configuration in use:
 *   info[0] networks in the batch (0: no batch yet)
 *   info[1] warps per block (phased: of the phase with the most chains)
 *   info[2] networks on a large warp region (shared-memory or hybrid tables)
 *   info[3] 1 if calls replay a CUDA graph
 *   info[4] networks on the hybrid path
 *   info[5] the candidate in use (-1: not tuned yet)
 *   info[6] kernels of the batched launch: 1, or the phases of a phased one
 *   trial_ms[10] (may be NULL) milliseconds of the candidates' trials (0 when
 *   the candidate was pinned by rn_batch_tune). */
int rn_batch_config(rn_ctx *ctx, int32_t info[7], double trial_ms[10]);

/* Pin the batched launch to candidate `config` (0 .. 9, see rn_batch_config)
 * instead of timing the candidates, or return to autotuning with -1.  Takes
 * effect at the next batched rn_anneal call (a pinned phased candidate still
 * times its phases' warps per block).  RN_EINVAL outside -1 .. 9. */
int rn_batch_tune(rn_ctx *ctx, int32_t config);

/* For callers that cannot let a library allocate device memory -- an
 * application that owns every byte of the GPU through its own memory pool or
 * fixed arena and must not see cudaMalloc/cudaFree behind its back, or that
 * has sized its device memory up front -- this one entry point performs the
 * level-end step of the annealing loop (the lowest delta_best over the chains,
 * lowest chain index on ties, copied with its vector into every chain) on the
 * caller's own device buffers, without a context and without allocating.  It
 * is an addition of this library for such callers; the paper has no
 * counterpart to it beyond the serial argmin of Table 1 it performs.
 *   x_best     device [n_chains][row_bytes] vectors; row w is copied (n_params
 *              bytes) into every other row.
 *   d_best     device [n_chains] objectives; entry w is copied into every other.
 *   n_chains   1 .. 1,048,576: the call keeps its partial minima in one fixed
 *              8 KiB device array, sized for at most that many chains; more
 *              are rejected with RN_EINVAL.
 *   row_bytes  stride of x_best rows (>= n_params).
 *   stream     cudaStream_t to queue the three kernels on (NULL: legacy default).
 * The call queues its work and returns; it calls no cudaMalloc, cudaFree or
 * allocating routine.  The fixed array is a file-scope device array that every
 * GPU loading the library holds until the process exits.  On the first call
 * for a device, the call resolves that array's device address with the device
 * current (cudaGetSymbolAddress, which may also load the library's device code
 * on that device); make that first call before any stream capture.  Every
 * call shares the array and leaves its contents behind; nothing in it needs to
 * start at zero, because each call writes every slot before reading it.  Calls
 * whose work overlaps on the GPU (two streams, or two host threads) race on
 * the array: order them on one stream.  The resolved address is kept for the
 * life of the process; after a cudaDeviceReset of that device it would be
 * stale, so the call is not supported after such a reset.  Before launching,
 * the call checks that x_best and d_best are device (or managed) memory of the
 * current device spanning the bytes above within their allocations.  Errors:
 * RN_EINVAL for a NULL pointer, a host pointer, another device's memory, a
 * buffer shorter than its span or a size out of range; RN_ECUDA if the device
 * cannot be used; the message is rn_last_error(NULL). */
int rn_level_sync_noalloc(int8_t *x_best, int32_t *d_best, int32_t n_chains, int64_t row_bytes,
                          int32_t n_params, void *stream);

/* ---- Learned proposal screen ------------------------------------------------
 * An addition of this library to the method of Table 1 (the paper has no
 * surrogate): a small MLP on the one-hot encoding of x ranks K candidate moves
 * per chain and step so that only the best-ranked few are simulated exactly.
 * The exact simulator alone decides acceptance (Metropolis as in Table 1), so
 * the surrogate changes which moves are tried, never what a move scores.
 *
 * Model: onehot(x) concatenates one block per parameter j of |dom_j| inputs
 * (domains ascending as in Sections 2.1-2.2; width D = sum |dom_j|), and
 *     a1 = b1 + W1^T onehot(x),  h1 = relu(a1)        W1 [D][H1]
 *     a2 = b2 + W2^T h1,         h2 = relu(a2)        W2 [H1][H2]
 *     y  = b3 + w3 . h2                               w3 [H2]
 * FP32 master weights; the matrix products run on BF16 tensor-core GEMMs with
 * FP32 accumulation (W1, W2 and h1 rounded to BF16, h2 and y in FP32).
 * Training minimises mean (y - target)^2 with Adam on the FP32 masters. */

/* Create the screen of a network: hidden widths h1, h2 (multiples of 256, at
 * most 1024), a device training set of `capacity` pairs (>= 1).  Weights
 * start at zero (rn_mlp_set_weights).  Out: *mlp_id, *onehot_width = D. */
int rn_mlp_create(rn_ctx *ctx, int32_t net, int32_t h1, int32_t h2, int64_t capacity,
                  int32_t *mlp_id, int32_t *onehot_width);

/* FP32 weights, host arrays in the layouts above (W1 [D][h1] row-major, W2
 * [h1][h2]); set resets the Adam state. */
int rn_mlp_set_weights(rn_ctx *ctx, int32_t mlp, const float *W1, const float *b1,
                       const float *W2, const float *b2, const float *w3, float b3);
int rn_mlp_get_weights(rn_ctx *ctx, int32_t mlp, float *W1, float *b1, float *W2, float *b2,
                       float *w3, float *b3);

/* Predictions y[n] of the vectors x[n][P].  Here and in the calls below that
 * take host vectors, every value must lie in its parameter's domain
 * (RN_EINVAL otherwise); the constraints of Section 2.5.3 are not required. */
int rn_mlp_forward(rn_ctx *ctx, int32_t mlp, int32_t n, const int8_t *x, float *y);

/* Loss (mean squared error) and its gradients with respect to every weight,
 * for the n (1 .. 65536) pairs (x[n][P], target[n]); output layouts as in
 * rn_mlp_get_weights.  Any output may be NULL. */
int rn_mlp_gradients(rn_ctx *ctx, int32_t mlp, int32_t n, const int8_t *x, const float *target,
                     float *loss, float *gW1, float *gb1, float *gW2, float *gb2, float *gw3,
                     float *gb3);

/* Training set: append pairs from the host (targets as given), or the current
 * state of every chain of the network (x_cur, target = delta_cur / n_obs with
 * n_obs the observed entries of the time course).  The set is a ring: beyond
 * its capacity the oldest pairs are overwritten.  *count (may be NULL) = pairs
 * held after the call. */
int rn_mlp_add_samples(rn_ctx *ctx, int32_t mlp, int32_t n, const int8_t *x, const float *target,
                       int64_t *count);
int rn_mlp_log_chains(rn_ctx *ctx, int32_t mlp, int64_t *count);

/* `steps` Adam steps (learning rate lr, beta1 0.9, beta2 0.999, eps 1e-8) on
 * minibatches of `batch` pairs (a multiple of 128, at most 65536) drawn
 * uniformly with replacement from the training set by Philox4x32-10 keyed by
 * `seed` (counter (step, 0, row, 8)).  Where the training set's targets
 * spread less than 1/16 of their mean level, they are standardised by their
 * mean and standard deviation for the steps (the output layer w3, b3 is mapped
 * to that scale before -- unless it has never been trained -- and back after,
 * so predictions stay in the targets' units).  *loss (may be NULL): mean
 * squared error of the last minibatch, on the standardised scale when the
 * targets were standardised.  The first step is launched directly; the
 * launches of the next one are captured once per call in a CUDA graph on the
 * context's stream and replayed for the remaining steps, so the call must not
 * be made while that stream is being captured (RN_ECUDA). */
int rn_mlp_train(rn_ctx *ctx, int32_t mlp, int32_t steps, int32_t batch, float lr, uint64_t seed,
                 float *loss);

/* Screened annealing of the screen's network for `sweeps` steps (schedule as
 * in rn_anneal; reset_to_best and global_sync are not supported here).  Step g
 * of chain k draws K candidates: candidate 0 from Philox counter
 * (g_lo, g_hi, k, 0) exactly as rn_anneal's proposal, candidate c >= 1 from
 * (g_lo, g_hi, k, 16 + c) (words 0 and 1, GetCandidate of Table 1).  With
 * probability eps (word 3 of counter tag 0 below eps * 2^32) only candidate 0
 * is simulated; otherwise the `top` candidates of lowest predicted y (distinct
 * moves, lowest index on ties) are simulated exactly and the one of lowest
 * exact score (first on ties) goes to the Metropolis test of Table 1 with
 * word 2 of counter tag 0.  A step with no candidate is a null move.  With
 * eps = 1 the chains are bit-identical to rn_anneal's.  K: 1 .. 32;
 * top: 1 .. 4 (<= K).  Covers every network the annealing kernels cover (a
 * warp or a block of threads per chain); RN_EUNSUPPORTED if one chain's x and
 * constraint counters exceed a block's shared memory.  The layer-2 input rows
 * of the K candidates, relu(A1 + W1[new] - W1[old]), go through device memory
 * unless rn_mlp_set_hidden_mode selects forming them inside the GEMM. */
int rn_anneal_screened(rn_ctx *ctx, int32_t mlp, const rn_schedule *s, int32_t K, int32_t top,
                       double eps, int64_t sweeps);

/* How a screened step forms the layer-2 GEMM's input rows, the hidden rows
 * relu(A1 + W1[new] - W1[old]) of every chain's K candidates (an addition of
 * this library, no counterpart in the paper).  mode 1 (the default): the
 * propose kernel writes the BF16 rows to device memory and the tcgen05 GEMM
 * reads them back by TMA (M x H1 x 2 bytes each way per step).  mode 0: the
 * propose kernel writes only each candidate's two W1 row indices, and producer
 * warps of the GEMM form the rows in shared memory from A1 and the gathered W1
 * rows; it saves the round trip through memory but measured slower on GB300
 * (each SM's L2 intake for the row gathers and B tiles exceeds the MMAs' pace).
 * Both give bit-identical predictions and chains; layers wider than 512 and
 * fewer than 8 candidates always use mode 1.  RN_EINVAL for another mode or an
 * unknown screen. */
int rn_mlp_set_hidden_mode(rn_ctx *ctx, int32_t mlp, int32_t mode);

/* Wait for all queued work on the context stream; reports device-side errors. */
int rn_synchronize(rn_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
