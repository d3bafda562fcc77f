/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for the parallel
 * simulated-annealing parameter search over ternary discrete-logic models of
 * regulatory networks (arXiv 2506.19866).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library uses this file; the
 * two implementations share no code.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it.  Every function follows the paper's
 * steps in its order and notation, with no blocking, fusion or reordering:
 *
 *   orc_simulate        Sections 2.1 (image K_i) and 2.2 (priority update)
 *   orc_weights         Section 2.3, gradient matrix G, weight |G| + 1
 *   orc_score_*         Section 2.3, objective y
 *   orc_propose         Table 1 GetCandidate + Section 2.5.3 constraints
 *   orc_threshold       Table 1 acceptance criterion A = exp(-dE / T)
 *   orc_anneal          Table 1, the parallel simulated-annealing loop
 *   orc_init_chain      Section 2.4.2 / 2.5.3: a valid random x0 per thread
 *   orc_philox4x32_10   Philox4x32-10 (Salmon et al., SC'11), the per-chain
 *                       counter-based generator that replaces the paper's
 *                       per-thread xoroshiro128+ (Section 4.2)
 *   orc_bruteforce      exhaustive minimum over all valid parameter vectors
 *   orc_mlp             the learned proposal screen (an MLP on the one-hot
 *                       parameter vector) in FP64: forward, MSE loss, gradients
 *
 * Where the paper is silent or its extracted text is garbled, the readings
 * below are used (each is also stated at the function that applies it):
 *   - the objective is the SUM over all entries of |S - R| (.) (|G| + 1);
 *   - G is taken per condition from consecutive time points, and is 0 unless
 *     both entries are observed; unobserved entries have weight 0; row t0
 *     carries weight 1 when observed;
 *   - the target of node i is clamp(K_i, 0, 2) (node bias 0);
 *   - memory m: a node may move once it has been told to move in the same
 *     direction for m + 1 consecutive steps (this one included);
 *   - priority u_i * (tau - last_i), last_i = 0 before the first update; all
 *     eligible nodes whose priority equals the maximum update together;
 *   - a knocked-out node is 0 at every time point and never updates;
 *   - GetCandidate draws one free index uniformly, then one value uniformly
 *     among the domain values != current that keep both constraints true; if
 *     there is none the step is a null move and nothing is simulated;
 *   - acceptance: dE <= 0, or r < floor(exp(-dE / T) * 2^32) with r a uniform
 *     32-bit word (the "delta_cand < delta_best" clause of Table 1 is implied,
 *     as delta_cur >= delta_best always holds); x_best moves on strict
 *     improvement only.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- layout -- */

int32_t orc_n_params(const orc_net *net) { return 3 * net->n_edges + 3 * net->n_nodes; }

/* Parameter j of x = [w(E), p(E), t(E), u(N), m(N), d(N)] (Section 2.3, x). */
enum { K_W = 0, K_P, K_T, K_U, K_M, K_D };

static int kind_of(const orc_net *net, int32_t j, int32_t *index)
{
    int32_t E = net->n_edges, N = net->n_nodes;
    if (j < E) { *index = j; return K_W; }
    if (j < 2 * E) { *index = j - E; return K_P; }
    if (j < 3 * E) { *index = j - 2 * E; return K_T; }
    if (j < 3 * E + N) { *index = j - 3 * E; return K_U; }
    if (j < 3 * E + 2 * N) { *index = j - 3 * E - N; return K_M; }
    *index = j - 3 * E - 2 * N;
    return K_D;
}

/* Domains, ascending: Section 2.1 (w, p, t) and Section 2.2 (u, m, d). */
int32_t orc_domain(const orc_net *net, int32_t j, int8_t vals[6])
{
    int32_t idx;
    int n = 0;
    switch (kind_of(net, j, &idx)) {
    case K_W: vals[0] = 0; vals[1] = 1; vals[2] = 2; n = 3; break;
    case K_P: vals[0] = -1; vals[1] = 0; vals[2] = 1; n = 3; break;
    case K_T: vals[0] = 1; vals[1] = 2; n = 2; break;
    case K_U:
        if (net->fast[idx]) { vals[0] = 10; vals[1] = 11; vals[2] = 12; n = 3; }
        else { for (int k = 0; k < 6; k++) vals[k] = (int8_t)(k + 1); n = 6; }
        break;
    case K_M: vals[0] = 0; vals[1] = 1; vals[2] = 2; n = 3; break;
    default: vals[0] = 1; vals[1] = 2; n = 2; break;
    }
    return n;
}

static int is_frozen(const orc_net *net, int32_t j) { return net->frozen && net->frozen[j]; }

/* Parameters GetCandidate may pick: the free ones, less the speeds u under the
 * synchronous scheme, where they have no effect. */
static int is_proposable(const orc_net *net, int32_t j)
{
    int32_t idx;
    if (is_frozen(net, j)) return 0;
    return !((net->sync || net->async_sel) && kind_of(net, j, &idx) == K_U);
}

/* ------------------------------------------------------------ generator -- */

/* Philox4x32-10: ten rounds of the Philox S-box on a 4x32-bit counter with a
 * 2x32-bit key (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11).  Round: multiply words 0 and 2 by the two round
 * multipliers, then cross the high halves with words 1 and 3 and the key;
 * the key advances by the two Weyl constants between rounds. */
void orc_philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform index in [0, n) from a 32-bit word: floor(r * n / 2^32). */
static uint32_t pick(uint32_t r, uint32_t n) { return (uint32_t)(((uint64_t)r * n) >> 32); }

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t r[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    orc_philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), ctr, r);
}

/* ----------------------------------------------------------- simulation -- */

/* Simulate one condition c for T time points (Sections 2.1-2.2); writes the
 * simulated matrix S (Section 2.3) as S[tau * N + i] for tau = 0..T-1.
 *
 * Every node that is not knocked out reads only the states before the step:
 *   K_i   = sum over edges j -> i of (s_j // t_ji) * w_ji * p_ji     (2.1)
 *   tgt_i = clamp(K_i, 0, 2); the node is told to move iff tgt_i != s_i
 *   cnt_i = consecutive steps told to move in the same direction    (2.2, m)
 *   eligible iff cnt_i >= m_i + 1; priority u_i * (tau - last_i)    (2.2)
 * All eligible nodes at the maximum priority then move by
 * min(d_i, |tgt_i - s_i|) toward tgt_i at the end of the step.  Under the
 * synchronous scheme (net->sync) every eligible node has the same priority,
 * so all of them move; under the asynchronous scheme (net->async_sel) only the
 * step's selected node may move (the others keep counting toward m). */
int32_t orc_simulate(const orc_net *net, const orc_tc *tc, const int8_t *x, int32_t c, uint8_t *S)
{
    const int32_t N = net->n_nodes, E = net->n_edges, T = tc->n_times;
    if (net->async_sel && (c >= net->n_cond_sel || net->n_times_sel != T)) return ORC_EINVAL;
    const int8_t *w = x, *p = x + E, *t = x + 2 * E;
    const int8_t *u = x + 3 * E, *m = x + 3 * E + N, *d = x + 3 * E + 2 * N;
    const uint8_t *ko = tc->knockout ? tc->knockout + (size_t)c * N : NULL;

    int32_t *s = calloc((size_t)N, sizeof *s), *cnt = calloc((size_t)N, sizeof *cnt);
    int32_t *dir = calloc((size_t)N, sizeof *dir), *last = calloc((size_t)N, sizeof *last);
    int32_t *K = calloc((size_t)N, sizeof *K), *prio = calloc((size_t)N, sizeof *prio);
    int32_t *move = calloc((size_t)N, sizeof *move);
    if (!s || !cnt || !dir || !last || !K || !prio || !move) {
        free(s); free(cnt); free(dir); free(last); free(K); free(prio); free(move);
        return ORC_ENOMEM;
    }

    for (int32_t i = 0; i < N; i++) {
        s[i] = (ko && ko[i]) ? 0 : tc->init[(size_t)c * N + i];
        S[i] = (uint8_t)s[i];
    }
    for (int32_t tau = 1; tau < T; tau++) {
        for (int32_t i = 0; i < N; i++) K[i] = 0;
        for (int32_t e = 0; e < E; e++)
            K[net->dst[e]] += (s[net->src[e]] / t[e]) * w[e] * p[e];

        int32_t pmax = 0;
        for (int32_t i = 0; i < N; i++) {
            prio[i] = 0;
            move[i] = 0;
            if (ko && ko[i]) continue;
            int32_t tgt = K[i] < 0 ? 0 : (K[i] > 2 ? 2 : K[i]);
            int32_t diff = tgt - s[i];
            if (diff == 0) {
                cnt[i] = 0;
                dir[i] = 0;
                continue;
            }
            int32_t drv = diff > 0 ? 1 : -1;
            cnt[i] = (drv == dir[i]) ? cnt[i] + 1 : 1;
            dir[i] = drv;
            const int selected =
                !net->async_sel || net->async_sel[(size_t)c * net->n_times_sel + tau] == i;
            if (cnt[i] >= m[i] + 1 && selected) {
                int32_t mag = diff > 0 ? diff : -diff;
                prio[i] = (net->sync || net->async_sel) ? 1 : u[i] * (tau - last[i]);
                move[i] = drv * (d[i] < mag ? d[i] : mag);
            }
            if (prio[i] > pmax) pmax = prio[i];
        }
        if (pmax > 0) {
            for (int32_t i = 0; i < N; i++) {
                if (prio[i] == pmax) {
                    s[i] += move[i];
                    last[i] = tau;
                    cnt[i] = 0;
                    dir[i] = 0;
                }
            }
        }
        for (int32_t i = 0; i < N; i++) S[(size_t)tau * N + i] = (uint8_t)s[i];
    }
    free(s); free(cnt); free(dir); free(last); free(K); free(prio); free(move);
    return ORC_OK;
}

/* Weight of each entry, W = observed * (|G| + 1) (Section 2.3): G is 0 in
 * row t0 and R_t - R_{t-1} below it, taken per condition and only where both
 * entries are observed. */
void orc_weights(const orc_net *net, const orc_tc *tc, uint8_t *W)
{
    const int32_t N = net->n_nodes, T = tc->n_times, C = tc->n_cond;
    for (int32_t c = 0; c < C; c++)
        for (int32_t tau = 0; tau < T; tau++)
            for (int32_t i = 0; i < N; i++) {
                size_t k = ((size_t)c * T + tau) * N + i;
                if (!tc->observed[k]) { W[k] = 0; continue; }
                int32_t G = 0;
                if (tau > 0 && tc->observed[k - N]) G = (int32_t)tc->ref[k] - (int32_t)tc->ref[k - N];
                W[k] = (uint8_t)((G < 0 ? -G : G) + 1);
            }
}

/* Objective y = sum |S - R| (.) (|G| + 1) (Section 2.3) of trajectories
 * traj[C][T][N]. */
int32_t orc_score_trajectory(const orc_net *net, const orc_tc *tc, const uint8_t *traj)
{
    const int32_t N = net->n_nodes, T = tc->n_times, C = tc->n_cond;
    size_t n = (size_t)C * T * N;
    uint8_t *W = malloc(n ? n : 1);
    if (!W) return ORC_ENOMEM;
    orc_weights(net, tc, W);
    int64_t y = 0;
    for (size_t k = 0; k < n; k++) {
        int32_t e = (int32_t)traj[k] - (int32_t)tc->ref[k];
        y += (int64_t)W[k] * (e < 0 ? -e : e);
    }
    free(W);
    return (int32_t)y;
}

/* Simulate(x) of Table 1: simulate every condition, then score. */
int32_t orc_objective(const orc_net *net, const orc_tc *tc, const int8_t *x, uint8_t *traj)
{
    const int32_t N = net->n_nodes, T = tc->n_times, C = tc->n_cond;
    size_t n = (size_t)C * T * N;
    uint8_t *buf = traj ? traj : calloc(n ? n : 1, 1);
    if (!buf) return ORC_ENOMEM;
    for (int32_t c = 0; c < C; c++) {
        int32_t rc = orc_simulate(net, tc, x, c, buf + (size_t)c * T * N);
        if (rc != ORC_OK) {
            if (!traj) free(buf);
            return rc;
        }
    }
    int32_t y = orc_score_trajectory(net, tc, buf);
    if (!traj) free(buf);
    return y;
}

/* ---------------------------------------------------------- constraints -- */

/* Section 2.5.3: (a) every node has an outgoing edge with w != 0; (b) every
 * node has an incoming edge with p = +1 and w != 0. */
static int constraints_hold(const orc_net *net, const int8_t *x)
{
    const int32_t N = net->n_nodes, E = net->n_edges;
    int ok = 1;
    for (int32_t i = 0; i < N && ok; i++) {
        int out_nz = 0, pos_in = 0;
        for (int32_t e = 0; e < E; e++) {
            if (net->src[e] == i && x[e] != 0) out_nz++;
            if (net->dst[e] == i && x[e] != 0 && x[E + e] == 1) pos_in++;
        }
        ok = out_nz >= 1 && pos_in >= 1;
    }
    return ok;
}

/* Domains, fixed parameters and both constraints. */
int32_t orc_check_params(const orc_net *net, const int8_t *x)
{
    const int32_t P = orc_n_params(net);
    for (int32_t j = 0; j < P; j++) {
        int8_t vals[6];
        int32_t n = orc_domain(net, j, vals), in = 0;
        for (int32_t k = 0; k < n; k++) in |= (vals[k] == x[j]);
        if (!in) return ORC_EINVAL;
        if (is_frozen(net, j) && x[j] != net->frozen_val[j]) return ORC_EINVAL;
    }
    return constraints_hold(net, x) ? ORC_OK : ORC_ECONSTRAINT;
}

/* GetCandidate (Table 1; constraints of Section 2.5.3 enforced "by
 * conditionals"): index j = the pick(r0)-th free parameter; alternatives are
 * the domain values != x_j whose single change keeps both constraints; the new
 * value is the pick(r1)-th alternative.  Returns 1 and (j, v) for a move, 0
 * for a null move (j is still reported when there is a free parameter). */
int32_t orc_propose(const orc_net *net, const int8_t *x, uint32_t r0, uint32_t r1,
                    int32_t *j_out, int8_t *v_out)
{
    const int32_t P = orc_n_params(net);
    int32_t n_free = 0;
    for (int32_t j = 0; j < P; j++) n_free += is_proposable(net, j);
    *j_out = -1;
    if (n_free == 0) return 0;
    int32_t want = (int32_t)pick(r0, (uint32_t)n_free), j = -1;
    for (int32_t k = 0, seen = 0; k < P; k++) {
        if (!is_proposable(net, k)) continue;
        if (seen++ == want) { j = k; break; }
    }
    *j_out = j;

    int8_t *y = malloc((size_t)P);
    if (!y) return 0;
    memcpy(y, x, (size_t)P);
    int8_t vals[6], alts[6];
    int32_t n = orc_domain(net, j, vals), n_alt = 0;
    for (int32_t k = 0; k < n; k++) {
        if (vals[k] == x[j]) continue;
        y[j] = vals[k];
        if (constraints_hold(net, y)) alts[n_alt++] = vals[k];
    }
    free(y);
    if (n_alt == 0) return 0;
    *v_out = alts[pick(r1, (uint32_t)n_alt)];
    return 1;
}

/* ------------------------------------------------------ initialisation -- */

/* A valid random x0 for one chain (the paper draws it with a constraint
 * solver; here it is a seeded sample-and-repair, valid by construction):
 *   1. each free x_j = dom_j[pick(r, |dom_j|)], r = word (j & 3) of
 *      Philox(seed; j >> 2, 0, chain, 1); fixed parameters keep their value;
 *   2. for each node i in order with no incoming edge of p = +1, w != 0: among
 *      its in-edges (edge order) whose p may be +1 and whose w may be nonzero,
 *      take the pick(r0)-th, set p = +1 and w = 1 + (r1 & 1) where free, with
 *      r = Philox(seed; i, 0, chain, 3);
 *   3. then for each node i in order with no outgoing edge of w != 0: among
 *      its out-edges with free w take the pick(r0)-th and set w = 1 + (r1 & 1),
 *      r = Philox(seed; i, 1, chain, 3).
 * Step 2 only raises counts that step 3 needs, and step 3 never lowers a
 * count that step 2 established. */
int32_t orc_init_chain(const orc_net *net, uint64_t seed, int32_t chain, int8_t *x)
{
    const int32_t N = net->n_nodes, E = net->n_edges, P = orc_n_params(net);
    for (int32_t j = 0; j < P; j++) {
        if (is_frozen(net, j)) { x[j] = net->frozen_val[j]; continue; }
        uint32_t r[4];
        draw(seed, (uint32_t)(j >> 2), 0u, (uint32_t)chain, 1u, r);
        int8_t vals[6];
        int32_t n = orc_domain(net, j, vals);
        x[j] = vals[pick(r[j & 3], (uint32_t)n)];
    }
    for (int32_t i = 0; i < N; i++) {
        int has = 0, n_cand = 0;
        for (int32_t e = 0; e < E; e++)
            if (net->dst[e] == i && x[e] != 0 && x[E + e] == 1) has = 1;
        if (has) continue;
        for (int32_t e = 0; e < E; e++) {
            if (net->dst[e] != i) continue;
            int p_ok = !is_frozen(net, E + e) || net->frozen_val[E + e] == 1;
            int w_ok = !is_frozen(net, e) || net->frozen_val[e] != 0;
            n_cand += p_ok && w_ok;
        }
        if (n_cand == 0) return ORC_ECONSTRAINT;
        uint32_t r[4];
        draw(seed, (uint32_t)i, 0u, (uint32_t)chain, 3u, r);
        int32_t want = (int32_t)pick(r[0], (uint32_t)n_cand);
        for (int32_t e = 0, seen = 0; e < E; e++) {
            if (net->dst[e] != i) continue;
            int p_ok = !is_frozen(net, E + e) || net->frozen_val[E + e] == 1;
            int w_ok = !is_frozen(net, e) || net->frozen_val[e] != 0;
            if (!(p_ok && w_ok)) continue;
            if (seen++ != want) continue;
            if (!is_frozen(net, E + e)) x[E + e] = 1;
            if (!is_frozen(net, e)) x[e] = (int8_t)(1 + (r[1] & 1u));
            break;
        }
    }
    for (int32_t i = 0; i < N; i++) {
        int has = 0, n_cand = 0;
        for (int32_t e = 0; e < E; e++)
            if (net->src[e] == i && x[e] != 0) has = 1;
        if (has) continue;
        for (int32_t e = 0; e < E; e++)
            n_cand += net->src[e] == i && !is_frozen(net, e);
        if (n_cand == 0) return ORC_ECONSTRAINT;
        uint32_t r[4];
        draw(seed, (uint32_t)i, 1u, (uint32_t)chain, 3u, r);
        int32_t want = (int32_t)pick(r[0], (uint32_t)n_cand);
        for (int32_t e = 0, seen = 0; e < E; e++) {
            if (net->src[e] != i || is_frozen(net, e)) continue;
            if (seen++ != want) continue;
            x[e] = (int8_t)(1 + (r[1] & 1u));
            break;
        }
    }
    return constraints_hold(net, x) ? ORC_OK : ORC_ECONSTRAINT;
}

/* ------------------------------------------------------------ annealing -- */

/* Acceptance threshold of Table 1 as a 32-bit word: the candidate with
 * dE = delta_cand - delta_cur > 0 is accepted iff r < floor(A * 2^32) with
 * A = exp(-dE / T) and r a uniform 32-bit word; capped at 2^32 - 1. */
uint32_t orc_threshold(double T, int64_t dE)
{
    double a = exp(-(double)dE / T) * 4294967296.0;
    double f = floor(a);
    if (f >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)f;
}

/* Temperature of level l: T <- rho * T once per level (Table 1), starting at
 * T0, by repeated multiplication. */
double orc_level_temperature(double T0, double alpha, int64_t level)
{
    double T = T0;
    for (int64_t l = 0; l < level; l++) T *= alpha;
    return T;
}

/* Number of passes of "while T > T_min" in Table 1. */
int32_t orc_count_levels(double T, double T_min, double rho)
{
    int32_t n = 0;
    while (T > T_min) {
        n++;
        T *= rho;
    }
    return n;
}

/* The parallel annealing loop of Table 1 for global steps g0 .. g0+sweeps-1.
 * Step g of chain k draws r = Philox(seed; g_lo, g_hi, k, 0): r0 picks the
 * parameter, r1 its new value, r2 decides acceptance.  Level l = g / n_iter
 * runs at T_l; with reset_to_best the level starts from x_best; with
 * global_sync the level ends by copying the best x_best (lowest chain index on
 * ties) to every chain.  Chains are independent unless global_sync is set, so
 * any subset (chain_ids) may be run on its own. */
int32_t orc_anneal(const orc_net *net, const orc_tc *tc, const orc_schedule *sched,
                   uint64_t seed, int32_t n_chains, const int32_t *chain_ids,
                   int64_t g0, int64_t sweeps, orc_chains *st)
{
    const int32_t P = orc_n_params(net);
    const int64_t n_iter = sched->iters_per_level;
    if (n_iter <= 0 || n_chains < 0 || sweeps < 0 || g0 < 0) return ORC_EINVAL;
    if (sched->global_sync && chain_ids) return ORC_EINVAL;
    if (sched->sync_group < 0) return ORC_EINVAL;
    int64_t level = g0 / n_iter;
    double T = orc_level_temperature(sched->T0, sched->alpha, level);

    for (int64_t g = g0; g < g0 + sweeps; g++) {
        while (level < g / n_iter) {
            T *= sched->alpha;
            level++;
        }
        for (int32_t k = 0; k < n_chains; k++) {
            int32_t chain = chain_ids ? chain_ids[k] : k;
            int8_t *xc = st->x_cur + (size_t)k * P, *xb = st->x_best + (size_t)k * P;
            if (sched->reset_to_best && g % n_iter == 0) {
                memcpy(xc, xb, (size_t)P);
                st->d_cur[k] = st->d_best[k];
            }
            uint32_t r[4];
            draw(seed, (uint32_t)g, (uint32_t)((uint64_t)g >> 32), (uint32_t)chain, 0u, r);
            int32_t j;
            int8_t v;
            if (!orc_propose(net, xc, r[0], r[1], &j, &v)) {
                st->n_null[k]++;
                continue;
            }
            int8_t old = xc[j];
            xc[j] = v;
            int32_t d_cand = orc_objective(net, tc, xc, NULL);
            if (d_cand < 0) return d_cand;
            int64_t dE = (int64_t)d_cand - st->d_cur[k];
            int accept = dE <= 0 || r[2] < orc_threshold(T, dE);
            if (!accept) {
                xc[j] = old;
                continue;
            }
            st->d_cur[k] = d_cand;
            st->n_accept[k]++;
            if (dE > 0) st->n_uphill[k]++;
            if (d_cand < st->d_best[k]) {
                st->d_best[k] = d_cand;
                memcpy(xb, xc, (size_t)P);
            }
        }
        if (sched->global_sync && (g + 1) % n_iter == 0 && n_chains > 0) {
            /* one argmin over all chains, or one per group of sync_group
             * consecutive chains (Section 4.5) */
            const int32_t G = sched->sync_group > 0 ? sched->sync_group : n_chains;
            for (int32_t first = 0; first < n_chains; first += G) {
                const int32_t end = first + G < n_chains ? first + G : n_chains;
                int32_t b = first;
                for (int32_t k = first + 1; k < end; k++)
                    if (st->d_best[k] < st->d_best[b]) b = k;
                for (int32_t k = first; k < end; k++) {
                    if (k == b) continue;
                    memcpy(st->x_best + (size_t)k * P, st->x_best + (size_t)b * P, (size_t)P);
                    st->d_best[k] = st->d_best[b];
                }
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------ screening MLP -- */

/* One-hot input of the learned proposal screen: parameter j occupies
 * |dom_j| consecutive positions from off[j]; value dom_j[i] sets position
 * off[j] + i.  Returns D = off[P], the input width. */
int32_t orc_onehot_offsets(const orc_net *net, int32_t *off)
{
    const int32_t P = orc_n_params(net);
    off[0] = 0;
    for (int32_t j = 0; j < P; j++) {
        int8_t vals[6];
        off[j + 1] = off[j] + orc_domain(net, j, vals);
    }
    return off[P];
}

static int32_t onehot_pos(const orc_net *net, const int32_t *off, int32_t j, int8_t v)
{
    int8_t vals[6];
    int32_t n = orc_domain(net, j, vals);
    for (int32_t k = 0; k < n; k++)
        if (vals[k] == v) return off[j] + k;
    return -1;
}

/* The screening MLP in FP64 over a batch of B vectors X[B][P]:
 *   a1 = b1 + W1^T onehot(x)      h1 = relu(a1)          W1 [D][H1]
 *   a2 = b2 + W2^T h1             h2 = relu(a2)          W2 [H1][H2]
 *   y  = b3 + w3 . h2                                     w3 [H2]
 * y[B] out.  With target t: loss = (1/B) sum_b (y_b - t_b)^2 and, where the
 * output pointers are not NULL, its gradients (relu'(a) = [a > 0]). */
int32_t orc_mlp(const orc_net *net, int32_t B, const int8_t *X, const double *target,
                int32_t H1, int32_t H2, const double *W1, const double *b1, const double *W2,
                const double *b2, const double *w3, double b3, double *y, double *loss,
                double *gW1, double *gb1, double *gW2, double *gb2, double *gw3, double *gb3)
{
    const int32_t P = orc_n_params(net);
    int32_t *off = malloc(sizeof(int32_t) * (size_t)(P + 1));
    double *a1 = malloc(sizeof(double) * (size_t)H1), *a2 = malloc(sizeof(double) * (size_t)H2);
    double *d2 = malloc(sizeof(double) * (size_t)H2), *d1 = malloc(sizeof(double) * (size_t)H1);
    if (!off || !a1 || !a2 || !d2 || !d1) {
        free(off); free(a1); free(a2); free(d2); free(d1);
        return ORC_ENOMEM;
    }
    const int32_t D = orc_onehot_offsets(net, off);
    const int grads = target != NULL;
    if (grads) {
        if (gW1) memset(gW1, 0, sizeof(double) * (size_t)D * H1);
        if (gb1) memset(gb1, 0, sizeof(double) * (size_t)H1);
        if (gW2) memset(gW2, 0, sizeof(double) * (size_t)H1 * H2);
        if (gb2) memset(gb2, 0, sizeof(double) * (size_t)H2);
        if (gw3) memset(gw3, 0, sizeof(double) * (size_t)H2);
        if (gb3) *gb3 = 0.0;
        if (loss) *loss = 0.0;
    }
    int32_t rc = ORC_OK;
    for (int32_t b = 0; b < B && rc == ORC_OK; b++) {
        const int8_t *x = X + (size_t)b * P;
        for (int32_t i = 0; i < H1; i++) a1[i] = b1[i];
        for (int32_t j = 0; j < P; j++) {
            int32_t r = onehot_pos(net, off, j, x[j]);
            if (r < 0) { rc = ORC_EINVAL; break; }
            for (int32_t i = 0; i < H1; i++) a1[i] += W1[(size_t)r * H1 + i];
        }
        if (rc != ORC_OK) break;
        for (int32_t k = 0; k < H2; k++) {
            double s = b2[k];
            for (int32_t i = 0; i < H1; i++)
                s += (a1[i] > 0.0 ? a1[i] : 0.0) * W2[(size_t)i * H2 + k];
            a2[k] = s;
        }
        double out = b3;
        for (int32_t k = 0; k < H2; k++) out += w3[k] * (a2[k] > 0.0 ? a2[k] : 0.0);
        y[b] = out;
        if (!grads) continue;
        const double diff = out - target[b];
        if (loss) *loss += diff * diff / B;
        const double dy = 2.0 * diff / B;
        if (gb3) *gb3 += dy;
        for (int32_t k = 0; k < H2; k++) {
            const double h2 = a2[k] > 0.0 ? a2[k] : 0.0;
            if (gw3) gw3[k] += dy * h2;
            d2[k] = a2[k] > 0.0 ? dy * w3[k] : 0.0;
            if (gb2) gb2[k] += d2[k];
        }
        for (int32_t i = 0; i < H1; i++) {
            const double h1 = a1[i] > 0.0 ? a1[i] : 0.0;
            double s = 0.0;
            for (int32_t k = 0; k < H2; k++) {
                if (gW2) gW2[(size_t)i * H2 + k] += h1 * d2[k];
                s += d2[k] * W2[(size_t)i * H2 + k];
            }
            d1[i] = a1[i] > 0.0 ? s : 0.0;
            if (gb1) gb1[i] += d1[i];
        }
        if (gW1)
            for (int32_t j = 0; j < P; j++) {
                const int32_t r = onehot_pos(net, off, j, x[j]);
                for (int32_t i = 0; i < H1; i++) gW1[(size_t)r * H1 + i] += d1[i];
            }
    }
    free(off); free(a1); free(a2); free(d2); free(d1);
    return rc;
}

/* ---------------------------------------------------------- brute force -- */

/* Minimum of y over every assignment of the free parameters that satisfies
 * both constraints (enumerated in mixed radix, first free index fastest).
 * Returns the number of valid assignments; best_score/best_x receive the
 * first minimiser found. */
int64_t orc_bruteforce(const orc_net *net, const orc_tc *tc, int32_t *best_score, int8_t *best_x)
{
    const int32_t P = orc_n_params(net);
    int32_t *free_idx = malloc(sizeof(int32_t) * (size_t)(P ? P : 1));
    int32_t *digit = calloc((size_t)(P ? P : 1), sizeof(int32_t));
    int8_t *x = malloc((size_t)(P ? P : 1));
    if (!free_idx || !digit || !x) {
        free(free_idx); free(digit); free(x);
        return ORC_ENOMEM;
    }
    int32_t n_free = 0;
    for (int32_t j = 0; j < P; j++) {
        int8_t vals[6];
        orc_domain(net, j, vals);
        if (is_frozen(net, j)) x[j] = net->frozen_val[j];
        else { x[j] = vals[0]; free_idx[n_free++] = j; }
    }
    int64_t n_valid = 0;
    *best_score = -1;
    for (;;) {
        if (constraints_hold(net, x)) {
            int32_t y = orc_objective(net, tc, x, NULL);
            if (y < 0) { n_valid = y; break; }
            n_valid++;
            if (*best_score < 0 || y < *best_score) {
                *best_score = y;
                if (best_x) memcpy(best_x, x, (size_t)P);
            }
        }
        int32_t k = 0;
        for (; k < n_free; k++) {
            int8_t vals[6];
            int32_t n = orc_domain(net, free_idx[k], vals);
            if (++digit[k] < n) { x[free_idx[k]] = vals[digit[k]]; break; }
            digit[k] = 0;
            x[free_idx[k]] = vals[0];
        }
        if (k == n_free) break;
    }
    free(free_idx); free(digit); free(x);
    return n_valid;
}
