/*
 * qv_oracle9.h -- plain FP64 CPU reference for the paper's experimental model
 * (Sec. V): nine actions, four occupancy sensors, the paper's stage reward.
 * Test infrastructure, like qv_oracle.h: only the test suite, the package
 * smoke check and the benchmark's CPU-baseline leg use it.
 *
 * Layout: unpadded row-major grids, cell x = r*W + c.  Action a moves to the
 * neighbour N_a(x) at (row + a/3 - 1, col + a%3 - 1), so N_4(x) = x.  Sensor
 * j = 0..3 reads the occupancy of N_1, N_3, N_5, N_7 (up, left, right, down)
 * and is bit j of the measurement z (|Z| = 16).
 */
#ifndef QV_ORACLE9_H
#define QV_ORACLE9_H
#include <stdint.h>

#define OR9_NUM_ACTIONS 9
#define OR9_NUM_OBS 16

typedef struct {
    int H, W;
    const unsigned char *occ;  /* [H*W] m(x): 1 occupied, 0 free                 */
    int goal;                  /* flat goal cell (free)                          */
    double slip;               /* epsilon: probability of each 45-degree slip    */
    double p_sensor;           /* P(z_s = m(N_s(x)) | x) of every sensor (0.95)  */
    double gamma;              /* discount                                       */
} or9_problem;

/* T'(x, a, .) before occupied targets are folded back (Fig. 2 reading):
 * returns the number of targets (1 or 3); cells may lie outside the grid
 * (reported as -1 with their row/col in rr/cc).                             */
int or9_tprime_row(const or9_problem *p, int x, int a, int *rr, int *cc, double *pr);
/* Row x of T(x, a, .) (the Sec. V equation: occupied or outside targets give
 * their mass to x): distinct targets (<= 3).                                */
int or9_transition_row(const or9_problem *p, int x, int a, int *y, double *pr);
/* R(x, a) for every x, a: R[a*n + x].                                       */
void or9_reward_table(const or9_problem *p, double *R);
/* Sensor pattern of x (bit j = occupancy of sensor j's cell) and O(x, z).   */
int or9_pattern(const or9_problem *p, int x);
double or9_obs_lik(const or9_problem *p, int x, int z);

int or9_value_iteration(const or9_problem *p, double tol, int max_sweeps, int truncated,
                        double *V, double *Q, int *sweeps, double *residual);
void or9_predict(const or9_problem *p, const double *b, int a, double *bbar);
void or9_obs_marginal(const or9_problem *p, const double *bbar, double *P);
double or9_correct(const or9_problem *p, const double *bbar, int z, double *bout);
double or9_belief_reward(const or9_problem *p, const double *R, const double *b, int a);
double or9_leaf_value(const or9_problem *p, const double *Q, const double *b, double *qa);

/* The sampled tree of Alg. 2-7 on this model, full width to `depth`
 * (<= 3), K samples per (V-node, action), FREQ weights f/K.  Node arrays
 * are indexed by off[l] + i; R and UQ by node * 9 + a; samples and boundary
 * flags by (node * 9 + a) * K + k.  belief (optional) receives the stored
 * beliefs of levels 0 .. min(store_levels, depth - 1).  Returns 0, or -1 when
 * a level outgrows the capacities in off.                                   */
int or9_tree_plan(const or9_problem *p, const double *Q, const double *b0, int depth, int K, uint64_t seed,
                  uint32_t episode, const long *off, int store_levels, int *n_level, int *parent, int *action,
                  int *obs, double *weight, double *pz, double *value, double *R, double *UQ, int *samples,
                  unsigned char *boundary, double *belief, int *root_action, double *root_value, double *root_q,
                  long *boundary_count);

#endif
