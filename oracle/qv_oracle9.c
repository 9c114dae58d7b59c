/*
 * qv_oracle9.c -- plain, slow FP64 CPU reference for the paper's
 * experimental model (Sec. V) and the sampled tree search on it.
 *
 * Test infrastructure: only the test suite, the package smoke check and the
 * benchmark's CPU-baseline leg use this file.  Every function follows one
 * passage of the paper, cited beside it; where the paper is silent the
 * reading taken is stated in the comment.
 */
#include "qv_oracle9.h"
#include "qv_oracle.h"  /* the sample streams and the inverse-CDF decision */

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Neighbours in clockwise order starting at N_1 (straight up): a 45-degree
 * slip of action a moves one step along this ring.                          */
static const int RING[8] = {1, 2, 5, 8, 7, 6, 3, 0};
static const int SENSOR[4] = {1, 3, 5, 7};

static int occupied(const or9_problem *p, int r, int c) {
    return r < 0 || r >= p->H || c < 0 || c >= p->W || p->occ[r * p->W + c];
}

/* Fig. 2 (T' with every neighbour free) is not in the text; the reading:
 * the stay action keeps the robot in place; any other action reaches N_a(x)
 * with probability 1 - 2 eps and slips 45 degrees to either side (the two
 * ring neighbours of N_a) with probability eps each.                       */
int or9_tprime_row(const or9_problem *p, int x, int a, int *rr, int *cc, double *pr) {
    const int r = x / p->W, c = x % p->W;
    if (a == 4) {
        rr[0] = r; cc[0] = c; pr[0] = 1.0;
        return 1;
    }
    int i = 0;
    while (RING[i] != a) ++i;
    const int t[3] = {a, RING[(i + 1) % 8], RING[(i + 7) % 8]};
    const double w[3] = {1.0 - 2.0 * p->slip, p->slip, p->slip};
    for (int j = 0; j < 3; ++j) {
        rr[j] = r + t[j] / 3 - 1;
        cc[j] = c + t[j] % 3 - 1;
        pr[j] = w[j];
    }
    return 3;
}

/* The true transition of Sec. V: mass T' puts on an occupied cell (the grid's
 * outside counts as occupied) goes to x.  Readings: the goal is absorbing
 * and an occupied cell keeps its (never used) mass.                         */
int or9_transition_row(const or9_problem *p, int x, int a, int *y, double *pr) {
    if (p->occ[x] || x == p->goal) {
        y[0] = x; pr[0] = 1.0;
        return 1;
    }
    int rr[3], cc[3];
    double w[3];
    const int m = or9_tprime_row(p, x, a, rr, cc, w);
    /* slot 0 collects the mass that stays on x */
    int ty[4];
    double tp[4];
    int n = 1;
    ty[0] = x; tp[0] = 0.0;
    for (int j = 0; j < m; ++j) {
        const int t = occupied(p, rr[j], cc[j]) ? x : rr[j] * p->W + cc[j];
        int k = 0;
        while (k < n && ty[k] != t) ++k;
        if (k == n) { ty[n] = t; tp[n] = 0.0; ++n; }
        tp[k] += w[j];
    }
    int out = 0;
    for (int k = 0; k < n; ++k)
        if (tp[k] != 0.0 || (k == 0 && n == 1)) { y[out] = ty[k]; pr[out] = tp[k]; ++out; }
    return out;
}

/* r(y) of Sec. V: -2 occupied (the outside included), 0 at the goal, -1
 * elsewhere; R(x, a) = -2 for the stay action off the goal, else
 * sum_y r(y) T'(x, a, y) (T', so that moves into obstacles cost more).
 * Readings: R = 0 at the (absorbing) goal and at occupied cells.           */
void or9_reward_table(const or9_problem *p, double *R) {
    const int n = p->H * p->W;
    for (int a = 0; a < OR9_NUM_ACTIONS; ++a)
        for (int x = 0; x < n; ++x) {
            double v = 0.0;
            if (!p->occ[x] && x != p->goal) {
                if (a == 4) v = -2.0;
                else {
                    int rr[3], cc[3];
                    double w[3];
                    const int m = or9_tprime_row(p, x, a, rr, cc, w);
                    for (int j = 0; j < m; ++j) {
                        double ry;
                        if (occupied(p, rr[j], cc[j])) ry = -2.0;
                        else if (rr[j] * p->W + cc[j] == p->goal) ry = 0.0;
                        else ry = -1.0;
                        v += ry * w[j];
                    }
                }
            }
            R[a * n + x] = v;
        }
}

/* The four sensors of Sec. V read the occupancy of N_1, N_3, N_5, N_7. */
int or9_pattern(const or9_problem *p, int x) {
    const int r = x / p->W, c = x % p->W;
    int m = 0;
    for (int j = 0; j < 4; ++j)
        if (occupied(p, r + SENSOR[j] / 3 - 1, c + SENSOR[j] % 3 - 1)) m |= 1 << j;
    return m;
}

/* Each sensor is right with probability p_sensor, independently. */
double or9_obs_lik(const or9_problem *p, int x, int z) {
    const int m = or9_pattern(p, x);
    double v = 1.0;
    for (int j = 0; j < 4; ++j) v *= (((z >> j) & 1) == ((m >> j) & 1)) ? p->p_sensor : 1.0 - p->p_sensor;
    return v;
}

/* MDP value iteration (the Bellman equation of Eq. 2 on a known state):
 * Jacobi sweeps from V = 0, stop at the first sweep whose max-abs change is
 * below tol (or run exactly `truncated` sweeps); Q = R + gamma T V.        */
int or9_value_iteration(const or9_problem *p, double tol, int max_sweeps, int truncated,
                        double *V, double *Q, int *sweeps, double *residual) {
    const int n = p->H * p->W, A = OR9_NUM_ACTIONS;
    double *R = (double *)malloc(sizeof(double) * A * n);
    double *Vn = (double *)malloc(sizeof(double) * n);
    or9_reward_table(p, R);
    for (int x = 0; x < n; ++x) V[x] = 0.0;
    int k = 0, status = 1;
    double res = 0.0;
    const int limit = truncated > 0 ? truncated : max_sweeps;
    while (k < limit) {
        res = 0.0;
        for (int x = 0; x < n; ++x) {
            if (p->occ[x] || x == p->goal) { Vn[x] = 0.0; continue; }
            double best = -HUGE_VAL;
            for (int a = 0; a < A; ++a) {
                int y[3];
                double pr[3];
                const int m = or9_transition_row(p, x, a, y, pr);
                double s = 0.0;
                for (int j = 0; j < m; ++j) s += pr[j] * V[y[j]];
                const double q = R[a * n + x] + p->gamma * s;
                if (q > best) best = q;
            }
            Vn[x] = best;
            const double d = fabs(Vn[x] - V[x]);
            if (d > res) res = d;
        }
        memcpy(V, Vn, sizeof(double) * n);
        ++k;
        if (truncated <= 0 && res < tol) { status = 0; break; }
    }
    if (truncated > 0) status = 0;
    for (int a = 0; a < A; ++a)
        for (int x = 0; x < n; ++x) {
            int y[3];
            double pr[3];
            const int m = or9_transition_row(p, x, a, y, pr);
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += pr[j] * V[y[j]];
            Q[a * n + x] = R[a * n + x] + p->gamma * s;
        }
    *sweeps = k;
    *residual = res;
    free(R); free(Vn);
    return status;
}

/* Numerator of Eq. 3: bbar(y) = sum_x T(x, a, y) b(x), scattered row by row. */
void or9_predict(const or9_problem *p, const double *b, int a, double *bbar) {
    const int n = p->H * p->W;
    for (int y = 0; y < n; ++y) bbar[y] = 0.0;
    for (int x = 0; x < n; ++x) {
        if (b[x] == 0.0) continue;
        int y[3];
        double pr[3];
        const int m = or9_transition_row(p, x, a, y, pr);
        for (int j = 0; j < m; ++j) bbar[y[j]] += pr[j] * b[x];
    }
}

/* Denominator of Eq. 3 for every z: P(z) = sum_y O(y, z) bbar(y). */
void or9_obs_marginal(const or9_problem *p, const double *bbar, double *P) {
    const int n = p->H * p->W;
    for (int z = 0; z < OR9_NUM_OBS; ++z) {
        double s = 0.0;
        for (int y = 0; y < n; ++y) s += or9_obs_lik(p, y, z) * bbar[y];
        P[z] = s;
    }
}

/* Eq. 3: b'(y) = O(y, z) bbar(y) / P(z); returns P(z). */
double or9_correct(const or9_problem *p, const double *bbar, int z, double *bout) {
    const int n = p->H * p->W;
    double s = 0.0;
    for (int y = 0; y < n; ++y) s += or9_obs_lik(p, y, z) * bbar[y];
    for (int y = 0; y < n; ++y) bout[y] = or9_obs_lik(p, y, z) * bbar[y] / s;
    return s;
}

/* R(b, a) = sum_x b(x) R(x, a). */
double or9_belief_reward(const or9_problem *p, const double *R, const double *b, int a) {
    const int n = p->H * p->W;
    double s = 0.0;
    for (int x = 0; x < n; ++x) s += b[x] * R[a * n + x];
    return s;
}

/* Alg. 5 / Eq. 4 with Gamma = {Q(., a')}: max_a' sum_y b(y) Q(a', y). */
double or9_leaf_value(const or9_problem *p, const double *Q, const double *b, double *qa) {
    const int n = p->H * p->W;
    double best = -HUGE_VAL;
    for (int a = 0; a < OR9_NUM_ACTIONS; ++a) {
        double s = 0.0;
        for (int y = 0; y < n; ++y) s += b[y] * Q[a * n + y];
        if (qa) qa[a] = s;
        if (s > best) best = s;
    }
    return best;
}

/* The tree of Alg. 2-7 on this model, as or_tree_plan does it on the beacon
 * model: every V-node above depth d expanded over the nine actions, K
 * samples of z from P(z | b, a) per (node, action) by the FP32 inverse CDF
 * of the uniform stream (level, path = code * 9 + a), one child per unique
 * z in ascending order with weight f/K, leaves valued by Alg. 5, Q-nodes
 * backed up with the discount of Eq. 2, the root action the lowest index
 * among the maxima.                                                          */
int or9_tree_plan(const or9_problem *p, const double *Q, const double *b0, int depth, int K, uint64_t seed,
                  uint32_t episode, const long *off, int store_levels, int *n_level, int *parent, int *action,
                  int *obs, double *weight, double *pz, double *value, double *R, double *UQ, int *samples,
                  unsigned char *boundary, double *belief, int *root_action, double *root_value, double *root_q,
                  long *boundary_count) {
    const int n = p->H * p->W, A = OR9_NUM_ACTIONS, nz = OR9_NUM_OBS;
    double *Rt = (double *)malloc(sizeof(double) * A * n);
    or9_reward_table(p, Rt);
    double **lev_b = (double **)calloc(depth + 1, sizeof(double *));
    uint64_t **code = (uint64_t **)calloc(depth + 1, sizeof(uint64_t *));
    long bcount = 0;
    int status = 0;
    n_level[0] = 1;
    lev_b[0] = (double *)malloc(sizeof(double) * n);
    for (int x = 0; x < n; ++x) lev_b[0][x] = p->occ[x] ? 0.0 : b0[x];
    code[0] = (uint64_t *)malloc(sizeof(uint64_t));
    code[0][0] = 0;
    parent[off[0]] = -1; action[off[0]] = -1; obs[off[0]] = -1;
    weight[off[0]] = 1.0; pz[off[0]] = 1.0;
    double *bbar = (double *)malloc(sizeof(double) * n);
    double *bn = (double *)malloc(sizeof(double) * n);
    for (int l = 0; l < depth && status == 0; ++l) {
        const int nl = n_level[l];
        const long base = off[l];
        const int leaf = (l + 1 == depth);
        long c = 0;
        /* count the children first (capacity check), then build them */
        int *uz = (int *)malloc(sizeof(int) * (size_t)nl * A * K);
        int *uf = (int *)malloc(sizeof(int) * (size_t)nl * A * K);
        double *up = (double *)malloc(sizeof(double) * (size_t)nl * A * K);
        int *un = (int *)calloc((size_t)nl * A, sizeof(int));
        for (int i = 0; i < nl; ++i) {
            const double *b = lev_b[l] + (size_t)i * n;
            for (int a = 0; a < A; ++a) {
                const long s = (base + i) * A + a;
                double P[OR9_NUM_OBS];
                int cnt[OR9_NUM_OBS] = {0};
                R[s] = or9_belief_reward(p, Rt, b, a);
                or9_predict(p, b, a, bbar);
                or9_obs_marginal(p, bbar, P);
                const uint64_t path = code[l][i] * A + (uint64_t)a;
                for (int k = 0; k < K; ++k) {
                    const float u = or_uniform(seed, episode, l, path, k);
                    const int z = or_sample_obs(P, nz, u);
                    const unsigned char bd = (unsigned char)or_is_boundary(P, nz, u);
                    samples[s * K + k] = z;
                    boundary[s * K + k] = bd;
                    bcount += bd;
                    cnt[z] += 1;
                }
                int m = 0;
                for (int z = 0; z < nz; ++z)
                    if (cnt[z]) {
                        uz[((size_t)i * A + a) * K + m] = z;
                        uf[((size_t)i * A + a) * K + m] = cnt[z];
                        up[((size_t)i * A + a) * K + m] = P[z];
                        ++m;
                    }
                un[(size_t)i * A + a] = m;
                c += m;
            }
        }
        if (off[l] + nl > off[l + 1] || off[l + 1] + c > off[l + 2]) status = -1;
        if (status == 0) {
            n_level[l + 1] = (int)c;
            code[l + 1] = (uint64_t *)malloc(sizeof(uint64_t) * (c > 0 ? c : 1));
            if (!leaf) lev_b[l + 1] = (double *)malloc(sizeof(double) * (size_t)(c > 0 ? c : 1) * n);
            long j = 0;
            for (int i = 0; i < nl; ++i)
                for (int a = 0; a < A; ++a) {
                    const int m = un[(size_t)i * A + a];
                    if (m) or9_predict(p, lev_b[l] + (size_t)i * n, a, bbar);
                    for (int q = 0; q < m; ++q, ++j) {
                        const long t = off[l + 1] + j;
                        parent[t] = i;
                        action[t] = a;
                        obs[t] = uz[((size_t)i * A + a) * K + q];
                        pz[t] = up[((size_t)i * A + a) * K + q];
                        weight[t] = (double)uf[((size_t)i * A + a) * K + q] / (double)K;
                        code[l + 1][j] = (code[l][i] * A + (uint64_t)a) * (uint64_t)nz + (uint64_t)obs[t];
                        double *dst = leaf ? bn : lev_b[l + 1] + (size_t)j * n;
                        or9_correct(p, bbar, obs[t], dst);                 /* Eq. 3 */
                        if (leaf) value[t] = or9_leaf_value(p, Q, dst, NULL); /* Alg. 5 */
                    }
                }
        }
        free(uz); free(uf); free(up); free(un);
    }
    if (depth == 0) value[off[0]] = or9_leaf_value(p, Q, lev_b[0], NULL);
    /* Alg. 6 / 7 from the deepest internal level up to the root */
    for (int l = depth - 1; l >= 0 && status == 0; --l) {
        const long cb = off[l + 1];
        long c = 0;
        for (int i = 0; i < n_level[l]; ++i) {
            double best = -HUGE_VAL;
            for (int a = 0; a < A; ++a) {
                double s = 0.0;
                while (c < n_level[l + 1] && parent[cb + c] == i && action[cb + c] == a) {
                    s += weight[cb + c] * value[cb + c];
                    ++c;
                }
                const double uq = R[(off[l] + i) * A + a] + p->gamma * s;
                UQ[(off[l] + i) * A + a] = uq;
                if (uq > best) best = uq;
            }
            value[off[l] + i] = best;
        }
    }
    if (status == 0) {
        int best = 0;
        if (depth == 0) {
            double qa[OR9_NUM_ACTIONS];
            *root_value = or9_leaf_value(p, Q, lev_b[0], qa);
            for (int a = 0; a < A; ++a) root_q[a] = qa[a];
        } else {
            for (int a = 0; a < A; ++a) root_q[a] = UQ[off[0] * A + a];
            *root_value = value[off[0]];
        }
        for (int a = 1; a < A; ++a) if (root_q[a] > root_q[best]) best = a;
        *root_action = best;
        *boundary_count = bcount;
        if (belief)
            for (int l = 0; l < depth && l <= store_levels; ++l)
                if (lev_b[l])
                    memcpy(belief + (size_t)off[l] * n, lev_b[l], sizeof(double) * (size_t)n_level[l] * n);
    }
    for (int l = 0; l <= depth; ++l) { free(lev_b[l]); free(code[l]); }
    free(lev_b); free(code); free(Rt); free(bbar); free(bn);
    return status;
}
