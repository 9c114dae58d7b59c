/*
 * qv_oracle.h -- plain FP64 CPU reference for QV-Tree Search (test infrastructure).
 *
 * This is the oracle that the CUDA library is checked against.  Only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg may use
 * it; the product path never links, loads or calls it.  It shares no code, no
 * header and no table with the CUDA library.
 *
 * Layout: unpadded row-major grids, cell x = r*W + c.  Actions 0=N (row-1),
 * 1=E (col+1), 2=S (row+1), 3=W (col-1), 4=stay.
 */
#ifndef QV_ORACLE_H
#define QV_ORACLE_H
#include <stdint.h>

#define OR_NUM_ACTIONS 5
#define OR_MAX_DEPTH 6
#define OR_WEIGHT_FREQ 0
#define OR_WEIGHT_MARGINAL 1

typedef struct {
    int H, W;
    const unsigned char *occ;  /* [H*W] m(x): 1 occupied, 0 free            */
    int B;                     /* number of beacons; |Z| = B + 1            */
    const int *beacon;         /* [B] flat cell of each beacon              */
    int range;                 /* Manhattan sensing range                   */
    int goal;                  /* flat goal cell                            */
    double slip;               /* epsilon, per perpendicular side           */
    double acc;                /* alpha                                     */
    double gamma;              /* discount                                  */
    const double *cost;        /* [H*W] per-cell cost c(y), or NULL (c = 0) */
} or_problem;

/* Observation label of every cell: nearest beacon id within range, else B. */
void or_labels(const or_problem *p, int *label);
/* Row x of T(x, a, .): returns the number of distinct targets (<= 3).      */
int or_transition_row(const or_problem *p, int x, int a, int *y, double *pr);
/* R(x, a) for every x, a: R[a*n + x].                                      */
void or_reward_table(const or_problem *p, double *R);
/* O(x', z).                                                                */
double or_obs_lik(const or_problem *p, const int *label, int x, int z);

/* MDP value iteration (Jacobi).  truncated > 0: run exactly that many
 * sweeps; else stop at the first sweep whose max-abs change < tol (or after
 * max_sweeps).  V[n], Q[5*n]; residual_hist[k] = |V_{k+1} - V_k|_inf.
 * Returns 0 when converged (or truncated), 1 when max_sweeps was reached.  */
int or_value_iteration(const or_problem *p, double tol, int max_sweeps, int truncated,
                       double *V, double *Q, int *sweeps, double *residual,
                       double *residual_hist);

void or_predict(const or_problem *p, const double *b, int a, double *bbar);
void or_obs_marginal(const or_problem *p, const int *label, const double *bbar, double *P);
double or_correct(const or_problem *p, const int *label, const double *bbar, int z, double *bout);
double or_belief_reward(const or_problem *p, const double *R, const double *b, int a);
double or_leaf_value(const or_problem *p, const double *Q, const double *b, double *qa);

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* The k-th uniform of the (level, path) sample stream.                     */
float or_uniform(uint64_t seed, uint32_t episode, int level, uint64_t path, int k);
/* Inverse-CDF decision, taken in FP32 like the CUDA path: first z with
 * u * C(B) < C(z), C the FP32 running sum of (float)P in ascending z.      */
int or_sample_obs(const double *P, int nz, float u);
/* 1 when u lies within 1e-6 of an FP64 CDF boundary C(z)/C(B), z < B.      */
int or_is_boundary(const double *P, int nz, float u);

/* Level-synchronous tree of depth d.  Level l nodes occupy the flat slots
 * [off[l], off[l] + n_level[l]) of every per-node array; capacity
 * off[l+1]-off[l]; off has depth+2 entries.
 * Per-(node, action) arrays use index (slot*5 + a), per-sample ones
 * ((slot*5 + a)*K + k).  belief (nullable) holds levels 0..store_levels in
 * slots [off[l]..] of n cells each.  replay (nullable) replaces the Philox
 * draws with given observation samples, same indexing as samples.
 * Returns 0, or -1 when a level exceeds its capacity.                      */
int or_tree_plan(const or_problem *p, const double *Q, const double *b0,
                 int depth, int K, uint64_t seed, uint32_t episode, int weight_mode,
                 const int *replay, const long *off, int store_levels,
                 int *n_level, int *parent, int *action, int *obs,
                 double *weight, double *pz, double *value,
                 double *R, double *UQ, int *samples, unsigned char *boundary,
                 double *belief, int *root_action, double *root_value,
                 double *root_q, long *boundary_count);

/* ---- reverse mode (FREQ weights; samples and every argmax held fixed) ---- */
/* d T(x, a, .) / d eps on the targets of or_transition_row.                */
int or_transition_row_dslip(const or_problem *p, int x, int a, int *y, double *dpr);
/* Adjoint of the root value of an or_tree_plan tree (its flat arrays, with
 * belief holding levels 0..depth-1).  Accumulates (+=) into Qbar[5n] (dL/dQ),
 * Rbar[5n] (dL/dR(x, a) of the internal nodes' R(b, a)), *dslip (through T
 * in every prediction), *dacc (through O in every correction) and db0[n]
 * (nullable).                                                              */
int or_tree_backward(const or_problem *p, const double *Q, int depth, int K, const long *off,
                     const int *n_level, const int *parent, const int *action, const int *obs,
                     const double *weight, const double *UQ, const double *belief, double dL_dV,
                     double *Qbar, double *Rbar, double *dslip, double *dacc, double *db0);
/* Adjoint of `sweeps` truncated Jacobi sweeps from V_0 = 0 and of
 * Q = R + gamma T V_sweeps and R(x, a) = sum_y T r: given Qbar and Rbar
 * (Rbar updated in place), accumulates *dslip and dcost[n] (nullable).     */
int or_vi_backward(const or_problem *p, int sweeps, const double *Qbar, double *Rbar,
                   double *dslip, double *dcost);

/* ---- Fast Informed Bound (Sec. IV-A, Eq. 6-7) ---- */
/* One application of Eq. 7 to alpha [5*n] -> out [5*n]; R from
 * or_reward_table, label from or_labels.  Returns max |out - alpha|.       */
double or_fib_sweep(const or_problem *p, const int *label, const double *R, const double *alpha,
                    double *out);
/* Jacobi iteration of Eq. 7 from alpha_0 = 0 (same stopping rule as
 * or_value_iteration).  alpha [5*n]; residual_hist nullable.               */
int or_fib_iteration(const or_problem *p, double tol, int max_sweeps, int truncated, double *alpha,
                     int *sweeps, double *residual, double *residual_hist);

/* ---- Point-based value iteration (Sec. IV-B, Eq. 8) ---- */
/* Pessimistic alpha_0 = R_min / (1 - gamma) on free, non-goal cells.       */
void or_pbvi_init(const or_problem *p, double *alpha0);
/* One round of belief set expansion: a new point from every point.        */
int or_pbvi_expand(const or_problem *p, const double *B, int nB, int round, uint64_t seed, double *out,
                   int *action, int *obs, int *boundary);
/* One Eq. 8 backup at every point of B given Gamma [nG][n].                */
int or_pbvi_backup(const or_problem *p, const double *B, int nB, const double *G, int nG, double *Gout,
                   double *value, int *astar, int *best, double *q, double *score);

/* ---- AEMS bookkeeping (Alg. 5-7, Eq. 9) ---- */
int or_tree_bounds(int depth, const long *off, const int *n_level, const int *parent, const int *action,
                   const double *weight, const double *R, const double *UQ, const double *value,
                   const double *Lleaf, double gamma, double *LV, double *HV, int *EV, double *LQ,
                   double *HQ, int *EQ);

/* ---- Best-first QV-Tree Search (Alg. 1 inner loop) ---- */
int or_bestfirst(const or_problem *p, const double *Qu, const double *G, int nG, const double *b0, int K,
                 uint64_t seed, uint32_t episode, int iters, int max_depth, int max_nodes, double *belief,
                 int *n_nodes, int *expanded, int *vparent, int *vaction, int *vobs, int *vdepth, double *vweight,
                 double *U, double *L, double *Hh, int *E, double *Rq, double *UQ, double *LQ, double *HQ, int *EQ,
                 int *cbeg, int *ccnt, long *boundary, double *margin);

/* ---- Closed-loop episodes (Alg. 1 outer loop, Eq. 1) ---- */
int or_env_step(const or_problem *p, const int *label, int x, int a, uint64_t seed, uint32_t e, int step, int *z_out);
int or_closed_loop(const or_problem *p, const double *Q, int E, const double *b0s, const int *x0s, int depth, int K,
                   uint64_t seed, int max_steps, int *actions, int *obs, int *states, int *steps, int *success,
                   double *ret, double *root_gap, long *boundary);

/* ---- Ancestral forward sampling (Alg. 4) ---- */
void or_forward_sample(const or_problem *p, const double *b, int a, int K, uint64_t seed, uint32_t episode,
                       int level, uint64_t path, int *z, int *boundary);

int or_num_threads(void);
void or_set_threads(int n);

#endif
