/*
 * oracle.h -- declarations of the plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This header belongs to the oracle and to nothing
 * else: the CUDA library under paper_2506_19866_gb300/csrc neither includes it
 * nor links the oracle.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load liboracle.so.
 *
 * Model (arXiv 2506.19866, Sections 2.1-2.3 and Table 1):
 *   nodes i = 0..N-1 with state s_i in {0,1,2};
 *   edges e = 0..E-1, src[e] -> dst[e], with weight w, polarity p, threshold t;
 *   node kinetics u (speed), m (memory), d (step size);
 *   parameter vector x = [w(E), p(E), t(E), u(N), m(N), d(N)], P = 3E + 3N.
 */
#ifndef RN_ORACLE_H
#define RN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ECONSTRAINT (-2)
#define ORC_ENOMEM (-3)

typedef struct {
    int32_t n_nodes;            /* N */
    int32_t n_edges;            /* E */
    const int32_t *src;         /* [E] source node of edge e */
    const int32_t *dst;         /* [E] target node of edge e */
    const uint8_t *fast;        /* [N] 1 = fast node (u in {10,11,12}) */
    const uint8_t *frozen;      /* [P] 1 = parameter is fixed, or NULL */
    const int8_t *frozen_val;   /* [P] value of each fixed parameter, or NULL */
    int32_t sync;               /* 1: synchronous update scheme (Section 2.2's
                                   alternative to priority updating): every
                                   eligible node moves at every step; u has no
                                   effect and is never proposed */
    int32_t n_cond_sel, n_times_sel;   /* shape of async_sel */
    const int32_t *async_sel;   /* [C][T] or NULL: asynchronous update scheme
                                   (Section 2.2's other alternative): at step tau
                                   of condition c only node async_sel[c][tau]
                                   (-1: none) may move, if eligible; u has no
                                   effect and is never proposed */
} orc_net;

typedef struct {
    int32_t n_cond;             /* C */
    int32_t n_times;            /* T, time points including t0 */
    const uint8_t *init;        /* [C][N] initial state per condition */
    const uint8_t *knockout;    /* [C][N] 1 = node held at 0, or NULL */
    const uint8_t *ref;         /* [C][T][N] reference data R, values 0..2 */
    const uint8_t *observed;    /* [C][T][N] 1 = entry observed */
} orc_tc;

typedef struct {
    double T0;                  /* initial temperature */
    double alpha;               /* cooling factor rho */
    int64_t iters_per_level;    /* proposals per temperature level */
    int32_t reset_to_best;      /* Table 1: each level restarts from x_best */
    int32_t global_sync;        /* Table 1: argmin over chains + broadcast */
    int32_t sync_group;         /* Section 4.5: argmin within groups of this many
                                   consecutive chains (0: one group of all) */
} orc_schedule;

typedef struct {
    int8_t *x_cur;              /* [n][P] */
    int8_t *x_best;             /* [n][P] */
    int32_t *d_cur;             /* [n] objective of x_cur */
    int32_t *d_best;            /* [n] objective of x_best */
    int64_t *n_accept;          /* [n] accepted moves */
    int64_t *n_uphill;          /* [n] accepted moves with dE > 0 */
    int64_t *n_null;            /* [n] steps with no valid alternative */
} orc_chains;

int32_t orc_n_params(const orc_net *net);
int32_t orc_domain(const orc_net *net, int32_t j, int8_t vals[6]);
void orc_philox4x32_10(uint32_t k0, uint32_t k1, const uint32_t ctr[4], uint32_t out[4]);
uint32_t orc_threshold(double T, int64_t dE);
double orc_level_temperature(double T0, double alpha, int64_t level);
int32_t orc_count_levels(double T, double T_min, double rho);

void orc_weights(const orc_net *net, const orc_tc *tc, uint8_t *W);
int32_t orc_simulate(const orc_net *net, const orc_tc *tc, const int8_t *x, int32_t c, uint8_t *S);
int32_t orc_score_trajectory(const orc_net *net, const orc_tc *tc, const uint8_t *traj);
int32_t orc_objective(const orc_net *net, const orc_tc *tc, const int8_t *x, uint8_t *traj);

int32_t orc_check_params(const orc_net *net, const int8_t *x);
int32_t orc_propose(const orc_net *net, const int8_t *x, uint32_t r0, uint32_t r1,
                    int32_t *j_out, int8_t *v_out);
int32_t orc_init_chain(const orc_net *net, uint64_t seed, int32_t chain, int8_t *x);
int32_t orc_anneal(const orc_net *net, const orc_tc *tc, const orc_schedule *sched,
                   uint64_t seed, int32_t n_chains, const int32_t *chain_ids,
                   int64_t g0, int64_t sweeps, orc_chains *st);
int64_t orc_bruteforce(const orc_net *net, const orc_tc *tc, int32_t *best_score,
                       int8_t *best_x);

int32_t orc_onehot_offsets(const orc_net *net, int32_t *off);
int32_t orc_mlp(const orc_net *net, int32_t B, const int8_t *X, const double *target,
                int32_t H1, int32_t H2, const double *W1, const double *b1, const double *W2,
                const double *b2, const double *w3, double b3, double *y, double *loss,
                double *gW1, double *gb1, double *gW2, double *gb2, double *gw3, double *gb3);

#ifdef __cplusplus
}
#endif
#endif
